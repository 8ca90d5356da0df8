// ew_mapped.cu -- a single curvilinear grid by the mapping method (Section
// "Discrete approximations": a smooth invertible map x = G(r) from the unit
// square; the equations transformed by the chain rule and discretised by
// conservative centred differences).  Two dimensions, second order, u = 0 on
// every boundary vertex.
//
// Operator.  In the r coordinates (r, s) with the metric of the vertex
// coordinates (centred differences, second-order one-sided ones on the
// boundary vertices):
//   J = x_r y_s - x_s y_r,  A11 = (x_s^2 + y_s^2)/J,  A22 = (x_r^2 + y_r^2)/J,
//   A12 = -(x_r x_s + y_r y_s)/J,
//   J L u = d_r(A11 u_r + A12 u_s) + d_s(A12 u_r + A22 u_s),
// discretised with the diagonal fluxes at half points (A averaged over the two
// vertices) and the cross fluxes by centred differences.  The result is a
// 9-point stencil whose coefficients, multiplied by J, are symmetric: the
// coupling of a vertex to its east neighbour equals the east neighbour's
// coupling back, and likewise north, north-east and south-east.  So per
// active vertex the library stores the centre and the E, N, NE, SE couplings
// of J L (the W, S, SW, NW ones are the neighbours' E, N, NE, SE) and 1/J, as
// one 4-wide record (E, N, NE, SE) and one 2-wide record (centre, 1/J) per vertex.
// The off-diagonal couplings are rounded to a common grid and the centre is
// minus their exact sum, so L 1 = 0 holds exactly in the stored precision
// (the same consistency as the box stencils).
//
// Symmetry.  L is symmetric in the J-weighted sums (the discrete L2 inner
// product of the map), which ew_rayleigh and the Krylov solver use through the
// weights sqrt(J) (launch_wsqrt).
//
// Kernels: one fused leapfrog + filter step per launch (summed form, as the
// box kernels), the first step, and L alone.  Per point and step the step kernel
// moves W^n, D^n and the filter sum in, the five couplings and 1/J in, and
// D^{n+1}, W^{n+1} and the filter sum out: 48 B in FP32 (the neighbours' W and
// couplings come through L1/L2).
#include <math.h>

#include <algorithm>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "ew_internal.h"

namespace ew {

namespace {

// metric of the vertex lattice (p1 x p2 vertices, r index fastest)
struct Metric {
    std::vector<double> J, A11, A12, A22;
};

double dline(const double* xy, int64_t base, int64_t stride, int64_t p, int64_t t, int c, double d) {
    auto F = [&](int64_t k) { return xy[2 * (base + k * stride) + c]; };
    if (t == 0) return (-3.0 * F(0) + 4.0 * F(1) - F(2)) / (2.0 * d);
    if (t == p - 1) return (3.0 * F(p - 1) - 4.0 * F(p - 2) + F(p - 3)) / (2.0 * d);
    return (F(t + 1) - F(t - 1)) / (2.0 * d);
}

}  // namespace

ew_status mapped_build(int64_t n1, int64_t n2, const double* xy, MappedData* m) {
    const int64_t p1 = n1 + 2, p2 = n2 + 2;
    const double dr = 1.0 / (double)(n1 + 1), ds = 1.0 / (double)(n2 + 1);
    const size_t np = (size_t)(p1 * p2);
    Metric g;
    g.J.resize(np);
    g.A11.resize(np);
    g.A12.resize(np);
    g.A22.resize(np);
    for (int64_t J = 0; J < p2; ++J)
        for (int64_t I = 0; I < p1; ++I) {
            const size_t q = (size_t)(J * p1 + I);
            const double xr = dline(xy, J * p1, 1, p1, I, 0, dr), yr = dline(xy, J * p1, 1, p1, I, 1, dr);
            const double xs = dline(xy, I, p1, p2, J, 0, ds), ys = dline(xy, I, p1, p2, J, 1, ds);
            const double jac = xr * ys - xs * yr;
            if (!(jac > 0.0) || !std::isfinite(jac))
                return set_error(EW_EINVAL, "mapped grid: the map must be orientation preserving (J > 0 at every vertex)");
            g.J[q] = jac;
            g.A11[q] = (xs * xs + ys * ys) / jac;
            g.A22[q] = (xr * xr + yr * yr) / jac;
            g.A12[q] = -(xr * xs + yr * ys) / jac;
        }
    auto at = [&](const std::vector<double>& a, int64_t I, int64_t J) { return a[(size_t)(J * p1 + I)]; };
    // couplings of vertex (I, J) to (I+1, J), (I, J+1), (I+1, J+1), (I+1, J-1), on the lattice
    m->E.assign(np, 0.0);
    m->N.assign(np, 0.0);
    m->NE.assign(np, 0.0);
    m->SE.assign(np, 0.0);
    const double cx = 1.0 / (dr * dr), cy = 1.0 / (ds * ds), cxy = 1.0 / (4.0 * dr * ds);
    for (int64_t J = 0; J < p2; ++J)
        for (int64_t I = 0; I < p1; ++I) {
            const size_t q = (size_t)(J * p1 + I);
            if (I + 1 < p1) m->E[q] = 0.5 * (at(g.A11, I, J) + at(g.A11, I + 1, J)) * cx;
            if (J + 1 < p2) m->N[q] = 0.5 * (at(g.A22, I, J) + at(g.A22, I, J + 1)) * cy;
            if (I + 1 < p1 && J + 1 < p2) m->NE[q] = (at(g.A12, I + 1, J) + at(g.A12, I, J + 1)) * cxy;
            if (I + 1 < p1 && J >= 1) m->SE[q] = -(at(g.A12, I + 1, J) + at(g.A12, I, J - 1)) * cxy;
        }
    m->n1 = n1;
    m->n2 = n2;
    m->xy.assign(xy, xy + 2 * np);
    m->J.resize((size_t)(n1 * n2));
    for (int64_t j = 0; j < n2; ++j)
        for (int64_t i = 0; i < n1; ++i) m->J[(size_t)(j * n1 + i)] = at(g.J, i + 1, j + 1);
    // Gershgorin bound of rho(-L) for the explicit step limit
    double rho = 0.0;
    for (int64_t J = 1; J <= n2; ++J)
        for (int64_t I = 1; I <= n1; ++I) {
            auto c = [&](const std::vector<double>& a, int64_t i, int64_t j) { return a[(size_t)(j * p1 + i)]; };
            const double off[8] = {c(m->E, I, J),      c(m->E, I - 1, J),      c(m->N, I, J),
                                   c(m->N, I, J - 1),  c(m->NE, I, J),         c(m->NE, I - 1, J - 1),
                                   c(m->SE, I, J),     c(m->SE, I - 1, J + 1)};
            double centre = 0.0, row = 0.0;
            for (double o : off) {
                centre -= o;
                row += fabs(o);
            }
            rho = std::max(rho, (fabs(centre) + row) / at(g.J, I, J));
        }
    m->rho = rho;
    return EW_OK;
}

// stored couplings in T: the off-diagonals rounded to a common grid q/2, the
// centre minus their exact sum (L 1 = 0 exactly in T)
template <typename T>
static void mapped_round(const MappedData& m, std::vector<T>& out) {
    const int64_t n1 = m.n1, n2 = m.n2, p1 = n1 + 2, N = n1 * n2;
    double mx = 0.0;
    for (size_t q = 0; q < m.E.size(); ++q)
        mx = std::max(std::max(mx, fabs(m.E[q])), std::max(fabs(m.N[q]), std::max(fabs(m.NE[q]), fabs(m.SE[q]))));
    const int mant = std::numeric_limits<T>::digits;
    int e = 0;
    frexp(16.0 * mx, &e);
    double q2 = 0.5 * ldexp(1.0, e - mant);
    auto rnd = [&](double c) { return nearbyint(c / q2) * q2; };
    // layout: N records (E, N, NE, SE) then N records (centre, 1/J), so a point's
    // own couplings are one 4-wide and one 2-wide load
    out.assign((size_t)(6 * N), T(0));
    T* quad = out.data();
    T* pair = quad + 4 * N;
    auto c = [&](const std::vector<double>& a, int64_t i, int64_t j) { return rnd(a[(size_t)(j * p1 + i)]); };
    for (int64_t J = 1; J <= n2; ++J)
        for (int64_t I = 1; I <= n1; ++I) {
            const size_t q = (size_t)((J - 1) * n1 + (I - 1));
            const double off[8] = {c(m.E, I, J),     c(m.E, I - 1, J),      c(m.N, I, J),  c(m.N, I, J - 1),
                                   c(m.NE, I, J),    c(m.NE, I - 1, J - 1), c(m.SE, I, J), c(m.SE, I - 1, J + 1)};
            double centre = 0.0;
            for (double o : off) centre -= o;  // exact: multiples of q/2 far below 2^53 q/2
            quad[4 * q + 0] = T(off[0]);
            quad[4 * q + 1] = T(off[2]);
            quad[4 * q + 2] = T(off[4]);
            quad[4 * q + 3] = T(off[6]);
            pair[2 * q + 0] = T(centre);
            pair[2 * q + 1] = T(1.0 / m.J[q]);
        }
}

// device copies in the field precision (and sqrt J in FP64), made on first use
template <typename T>
static ew_status mapped_device(const GridGeom& g, const T** coef, const double** sqrtJ) {
    MappedData* m = g.map;
    std::lock_guard<std::mutex> lk(m->mu);
    const int k = sizeof(T) == 4 ? 0 : 1;
    const int64_t N = m->n1 * m->n2;
    if (!m->dev[k]) {
        std::vector<T> h;
        mapped_round<T>(*m, h);
        void* d = nullptr;
        EW_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(T)));
        cudaError_t ce = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            cudaFree(d);
            return cuda_error(ce, "upload of the mapped-grid couplings");
        }
        m->dev[k] = d;
    }
    if (!m->sqrtJ) {
        std::vector<double> h((size_t)N);
        for (int64_t q = 0; q < N; ++q) h[(size_t)q] = sqrt(m->J[(size_t)q]);
        void* d = nullptr;
        EW_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(double)));
        cudaError_t ce = cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            cudaFree(d);
            return cuda_error(ce, "upload of the mapped-grid weights");
        }
        m->sqrtJ = (double*)d;
    }
    if (coef) *coef = (const T*)m->dev[k];
    if (sqrtJ) *sqrtJ = m->sqrtJ;
    return EW_OK;
}

void mapped_release(MappedData* m) {
    if (!m) return;
    for (void*& d : m->dev)
        if (d) {
            cudaFree(d);
            d = nullptr;
        }
    if (m->sqrtJ) cudaFree(m->sqrtJ);
    m->sqrtJ = nullptr;
}

// a point's own couplings: (E, N, NE, SE) and (centre, 1/J)
template <typename T>
struct Own {
    T e, n, ne, se, c, rj;
};
__device__ __forceinline__ Own<float> own_couplings(const float* __restrict__ c, int64_t N, int64_t q) {
    const float4 a = reinterpret_cast<const float4*>(c)[q];
    const float2 b = reinterpret_cast<const float2*>(c + 4 * N)[q];
    return Own<float>{a.x, a.y, a.z, a.w, b.x, b.y};
}
__device__ __forceinline__ Own<double> own_couplings(const double* __restrict__ c, int64_t N, int64_t q) {
    const double2 a = reinterpret_cast<const double2*>(c)[2 * q];
    const double2 a2 = reinterpret_cast<const double2*>(c)[2 * q + 1];
    const double2 b = reinterpret_cast<const double2*>(c + 4 * N)[q];
    return Own<double>{a.x, a.y, a2.x, a2.y, b.x, b.y};
}

// J L u at active vertex (i, j) (0-based), x fastest, and 1/J there; neighbours
// beyond the active set are boundary vertices (u = 0)
template <typename T>
__device__ __forceinline__ T mapped_jlap(const T* __restrict__ u, const T* __restrict__ c, int64_t N, int nx,
                                         int ny, int i, int j, int64_t q, T& rj) {
    const Own<T> o = own_couplings(c, N, q);
    rj = o.rj;
    const bool w = i > 0, e = i + 1 < nx, s = j > 0, n = j + 1 < ny;
    T r = o.c * u[q];
    if (e) r += o.e * u[q + 1];
    if (w) r += c[4 * (q - 1) + 0] * u[q - 1];
    if (n) r += o.n * u[q + nx];
    if (s) r += c[4 * (q - nx) + 1] * u[q - nx];
    if (e && n) r += o.ne * u[q + 1 + nx];
    if (w && s) r += c[4 * (q - 1 - nx) + 2] * u[q - 1 - nx];
    if (e && s) r += o.se * u[q + 1 - nx];
    if (w && n) r += c[4 * (q - 1 + nx) + 3] * u[q - 1 + nx];
    return r;
}

// one thread per point: x from the block's threads, y from grid.y, the vector from grid.z
template <typename T>
__global__ void __launch_bounds__(128) k_mapped_apply(int nx, int ny, const T* __restrict__ u, T* __restrict__ Lu,
                                                      const T* __restrict__ c, T scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const int64_t N = (int64_t)nx * ny, q = (int64_t)j * nx + i, v = blockIdx.z;
    T rj;
    const T jl = mapped_jlap<T>(u + v * N, c, N, nx, ny, i, j, q, rj);
    Lu[v * N + q] = scale * rj * jl;
}

// first step: D^1 = (dt^2/2) L V, W^1 = V + D^1, out = c0 V + c1 W^1
template <typename T>
__global__ void __launch_bounds__(128) k_mapped_first(int nx, int ny, const T* __restrict__ vin, T* __restrict__ D1,
                                                      T* __restrict__ W1, T* __restrict__ vout,
                                                      const T* __restrict__ c, T half_dt2, T c0, T c1,
                                                      int64_t fstride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const int64_t N = (int64_t)nx * ny, q = (int64_t)j * nx + i, v = blockIdx.z;
    const T x = vin[v * N + q];
    T rj;
    const T jl = mapped_jlap<T>(vin + v * N, c, N, nx, ny, i, j, q, rj);
    const T d = half_dt2 * rj * jl;
    const T w1 = x + d;
    D1[v * fstride + q] = d;
    W1[v * fstride + q] = w1;
    vout[v * N + q] = c0 * x + c1 * w1;
}

// D <- D + dt^2 L W (in place), Wout <- W + D, acc += cn Wout
template <typename T>
__global__ void __launch_bounds__(128) k_mapped_step(int nx, int ny, const T* __restrict__ W, T* __restrict__ D,
                                                     T* __restrict__ Wout, T* __restrict__ acc,
                                                     const T* __restrict__ c, T dt2, T cn, int64_t fstride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const int64_t N = (int64_t)nx * ny, q = (int64_t)j * nx + i, v = blockIdx.z;
    const int64_t f = v * fstride + q;
    T rj;
    const T jl = mapped_jlap<T>(W + v * fstride, c, N, nx, ny, i, j, q, rj);
    const T d = D[f] + dt2 * rj * jl;
    const T wn = W[f] + d;
    D[f] = d;
    Wout[f] = wn;
    acc[v * N + q] += cn * wn;
}

static dim3 mgrid(const GridGeom& g, int nvec) {
    return dim3((unsigned)((g.n[0] + 127) / 128), (unsigned)g.n[1], (unsigned)nvec);
}

static ew_status mapped_check(const GridGeom& g, int nvec) {
    if (g.n[1] > 65535 || nvec > 65535) return set_error(EW_EUNSUPPORTED, "mapped grid: more than 65535 rows or vectors");
    return EW_OK;
}

template <typename T>
ew_status mapped_apply_L(const GridGeom& g, const T* u, T* Lu, int nvec, double scale, cudaStream_t st) {
    EW_TRY(mapped_check(g, nvec));
    const T* c = nullptr;
    EW_TRY(mapped_device<T>(g, &c, nullptr));
    k_mapped_apply<T><<<mgrid(g, nvec), 128, 0, st>>>((int)g.n[0], (int)g.n[1], u, Lu, c, T(scale));
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}
template ew_status mapped_apply_L<float>(const GridGeom&, const float*, float*, int, double, cudaStream_t);
template ew_status mapped_apply_L<double>(const GridGeom&, const double*, double*, int, double, cudaStream_t);

template <typename T>
ew_status mapped_wave_solve(const GridGeom& g, const FilterPlan& plan, const T* vin, T* vout, int nvec, T* fields,
                            cudaStream_t st) {
    EW_TRY(mapped_check(g, nvec));
    const T* c = nullptr;
    EW_TRY(mapped_device<T>(g, &c, nullptr));
    const int64_t fstride = field_stride(g.N);
    T* F[3];
    for (int q = 0; q < 3; ++q) F[q] = fields + (int64_t)q * nvec * fstride;
    const int nx = (int)g.n[0], ny = (int)g.n[1];
    const dim3 grid = mgrid(g, nvec);
    k_mapped_first<T><<<grid, 128, 0, st>>>(nx, ny, vin, F[0], F[1], vout, c, T(0.5 * plan.dt * plan.dt),
                                            T(plan.cn(0)), T(plan.cn(1)), fstride);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    const T dt2 = T(plan.dt * plan.dt);
    int cur = 1, nxt = 2;
    for (int64_t L = 1; L < plan.Nt; ++L) {
        cudaEvent_t ev = fused_begin(st);
        k_mapped_step<T><<<grid, 128, 0, st>>>(nx, ny, F[cur], F[0], F[nxt], vout, c, dt2, T(plan.cn(L + 1)), fstride);
        EW_CUDA_TRY(cudaGetLastError());
        fused_end(ev, st, g.N * nvec, g.N * nvec);
        std::swap(cur, nxt);
    }
    return EW_OK;
}
template ew_status mapped_wave_solve<float>(const GridGeom&, const FilterPlan&, const float*, float*, int, float*,
                                            cudaStream_t);
template ew_status mapped_wave_solve<double>(const GridGeom&, const FilterPlan&, const double*, double*, int,
                                             double*, cudaStream_t);

// out = sqrt(J)^e in, in == out allowed
template <typename T>
__global__ void k_wsqrt_mapped(const T* __restrict__ in, T* __restrict__ out, const double* __restrict__ sj, int64_t N,
                               int64_t total, int e) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const double s = sj[q % N];
        out[q] = T(e > 0 ? (double)in[q] * s : (double)in[q] / s);
    }
}

template <typename T>
ew_status mapped_wsqrt(const GridGeom& g, const T* in, T* out, int nvec, int e, cudaStream_t st) {
    const double* sj = nullptr;
    EW_TRY(mapped_device<T>(g, nullptr, &sj));
    k_wsqrt_mapped<T><<<kReduceBlocks * 4, 256, 0, st>>>(in, out, sj, g.N, g.N * (int64_t)nvec, e);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}
template ew_status mapped_wsqrt<float>(const GridGeom&, const float*, float*, int, int, cudaStream_t);
template ew_status mapped_wsqrt<double>(const GridGeom&, const double*, double*, int, int, cudaStream_t);

}  // namespace ew

using namespace ew;

extern "C" ew_status ew_grid_create_mapped(const int64_t n_interior[2], const double* xy_host, ew_prec prec,
                                           ew_grid** out) try {
    clear_error();
    if (!out || !n_interior || !xy_host) return set_error(EW_EINVAL, "null argument");
    *out = nullptr;
    if (prec == EW_FP32X2) return set_error(EW_EUNSUPPORTED, "mapped grids: FP32 or FP64 fields");
    if (prec != EW_FP32 && prec != EW_FP64) return set_error(EW_EINVAL, "bad precision");
    const int64_t n1 = n_interior[0], n2 = n_interior[1];
    if (n1 < 1 || n2 < 1) return set_error(EW_EINVAL, "n_interior must be >= 1");
    if (n1 > (1 << 20) || n2 > (1 << 20) || (n1 + 2) * (n2 + 2) > ((int64_t)1 << 31))
        return set_error(EW_EINVAL, "mapped grid too large");
    std::unique_ptr<MappedData> m(new (std::nothrow) MappedData());
    if (!m) return set_error(EW_ENOMEM, "host allocation failed");
    EW_TRY(mapped_build(n1, n2, xy_host, m.get()));
    int64_t n3[3] = {n1, n2, 1};
    double len[3] = {1.0, 1.0, 1.0};  // the unit square of the r coordinates
    ew_grid* g = nullptr;
    EW_TRY(ew_grid_create(2, n3, len, 2, nullptr, prec, &g));
    g->geom.map = m.release();
    *out = g;
    return EW_OK;
} catch (...) {
    return abi_exception();
}
