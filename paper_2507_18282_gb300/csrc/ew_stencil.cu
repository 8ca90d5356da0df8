// ew_stencil.cu -- fused leapfrog + filter kernels for the explicit wave-solve.
//
// One wave-solve (Algorithm matVec with the explicit scheme):
//   W^0 = V,  W^1 = V + (dt^2/2) L_h V                       (eq. explicitStep1)
//   W^{n+1} = 2 W^n - W^{n-1} + dt^2 L_h W^n                 (eq. explicitScheme)
//   V_out  = sum_{n=0}^{N_t} c_n W^n                          (eq. filterQuadrature)
// The filter sum is accumulated inside the time loop, as the paper notes for
// Algorithm EigenWave, so no time history is stored.
//
// Summed (velocity-difference) form.  Every kernel carries D^n = W^n - W^{n-1}
// instead of W^{n-1}:
//   D^1 = (dt^2/2) L_h V,  W^1 = V + D^1
//   D^{n+1} = D^n + dt^2 L_h W^n,  W^{n+1} = W^n + D^{n+1}
// which is the same recurrence.  In FP32 it matters: dt^2 L_h W^n is about
// (lambda dt)^2 |W| (1e-5 .. 1e-3 of |W| for the low and middle modes of fine
// grids), and added to 2 W^n - W^{n-1} it keeps only eps32 / (lambda dt)^2 of
// its relative precision; added to D^n (about lambda dt |W|) it keeps
// eps32 / (lambda dt).  The low modes of a 2047 x 3071 grid lose a factor
// 30 .. 300 of accuracy in the first form.
//
// Fields are stored in the active-point layout (x fastest, no padding): the
// box closure is applied on the fly.  Beyond a Dirichlet face the point one
// step outside is the wall (value 0) and the point two steps outside a ghost
// holding the odd reflection -u(mirror); a Neumann face's wall point is
// active and the points beyond it hold the even reflection u(mirror)
// (ew_bc_dev.cuh).
//
// Kernels:
//   k_first_step      : a3, writes D^1, W^1 and V_out = c_0 W^0 + c_1 W^1
//                       (3D; k_first_step2d: the same, tiled in shared memory).
//   k_step_simple     : one time step per launch (any dim), reads W^n and its
//                       neighbours from global memory, updates D in place,
//                       writes W^{n+1} to a second W buffer and
//                       V_out += c W^{n+1}.
//   k_step_tb2d       : (ew_tb2d.cu) b time steps per launch on overlapped
//                       tiles staged in shared memory (temporal blocking).
//   k_resident2d      : the whole wave-solve of a small 2D grid inside one CTA
//                       (grid + ghosts resident in shared memory).
#include <algorithm>
#include <cmath>
#include <limits>
#include <type_traits>
#include <utility>

#include "ew_dd.cuh"
#include "ew_internal.h"
#include "ew_stencil_dev.cuh"

namespace ew {

// Stencil coefficients, pre-multiplied by `scale` (dt^2 or dt^2/2) and stored
// in T.  Rounded one by one they would no longer sum to zero: the discrete
// operator would gain a mass term of about eps_T |c0| -- for FP32 on a
// 2047 x 3071 grid about 1e-7 of W per step against a force of 1e-5 .. 1e-3
// of W for the low and middle modes, i.e. a frequency error of up to 1e-2
// that builds up as phase drift over the wave-solve.  So the off-centre
// coefficients are rounded to a common grid q/2 (q = the ulp of T at twice
// their total weight) and c0 is minus their exact sum: the stencil stays
// exactly consistent (L_h 1 = 0 in the stored coefficients), the
// coefficients move by at most about 4 ulps relative.
template <typename T>
Stencil<T> make_stencil(const GridGeom& g, double scale) {
    Stencil<T> s;
    s.bc = g.bc;
    double a1[3] = {0, 0, 0}, a2[3] = {0, 0, 0};
    double tot = 0.0;
    for (int a = 0; a < g.dim; ++a) {
        double ih2 = 1.0 / (g.h[a] * g.h[a]);
        if (g.order == 2) {
            a1[a] = scale * ih2;
        } else {
            a1[a] = scale * 16.0 / 12.0 * ih2;
            a2[a] = -scale / 12.0 * ih2;
        }
        tot += 2.0 * (fabs(a1[a]) + fabs(a2[a]));
    }
    const int mant = MantBits<T>::value;  // 24, 53, or 48 for double-FP32 pairs
    int e = 0;
    frexp(2.0 * tot, &e);                               // 2 tot < 2^e
    double q = ldexp(1.0, e - mant);                    // ulp of T just below 2^e
    for (;;) {
        double c1[3], c2[3], sum = 0.0;
        for (int a = 0; a < 3; ++a) {
            c1[a] = nearbyint(a1[a] / (0.5 * q)) * (0.5 * q);
            c2[a] = nearbyint(a2[a] / (0.5 * q)) * (0.5 * q);
            sum += 2.0 * (c1[a] + c2[a]);
        }
        const double c0 = -sum;
        bool exact = (double)(T)c0 == c0;
        for (int a = 0; a < 3; ++a) exact = exact && (double)(T)c1[a] == c1[a] && (double)(T)c2[a] == c2[a];
        if (exact || q > 1.0) {
            for (int a = 0; a < 3; ++a) {
                s.c1[a] = T(c1[a]);
                s.c2[a] = T(c2[a]);
            }
            s.c0 = T(c0);
            return s;
        }
        q *= 2.0;
    }
}
template Stencil<float> make_stencil<float>(const GridGeom&, double);
template Stencil<double> make_stencil<double>(const GridGeom&, double);
template Stencil<dd> make_stencil<dd>(const GridGeom&, double);


template <typename T, int DIM, int ORDER>
__global__ void k_apply_L(int64_t nx, int64_t ny, int64_t nz, const T* __restrict__ u,
                          T* __restrict__ Lu, Stencil<T> s) {
    const int64_t N = nx * ny * nz;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int64_t v = blockIdx.z / nz, k = blockIdx.z - v * nz, j = blockIdx.y, q = (k * ny + j) * nx + i;
    u += v * N;
    Lu += v * N;
    Lu[q] = lap_global<T, DIM, ORDER>(u, s, q, i, j, k, nx, ny, nz);
}

// a3: D^1 = (dt^2/2) L V, W^1 = V + D^1, V_out = c0 W^0 + c1 W^1.  `s`
// carries the dt^2/2 scale.
// D1 and W1 have row pitch fpitch (>= nx: the padded layout of the
// TMA-staged 2D step, or nx)
template <typename T, int DIM, int ORDER>
__global__ void k_first_step(int64_t nx, int64_t ny, int64_t nz, const T* __restrict__ vin,
                             T* __restrict__ D1, T* __restrict__ W1, T* __restrict__ vout,
                             Stencil<T> s, T c0, T c1, int64_t fstride, int64_t fpitch) {
    const int64_t N = nx * ny * nz;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int64_t v = blockIdx.z / nz, k = blockIdx.z - v * nz, j = blockIdx.y, q = (k * ny + j) * nx + i;
    const int64_t qf = (k * ny + j) * fpitch + i;
    vin += v * N;
    vout += v * N;
    D1 += v * fstride;
    W1 += v * fstride;
    T x = vin[q];
    T d = lap_global<T, DIM, ORDER>(vin, s, q, i, j, k, nx, ny, nz);
    T w1 = x + d;
    D1[qf] = d;
    W1[qf] = w1;
    vout[q] = c0 * x + c1 * w1;
}

// The same first step on 2D grids, tiled: a CTA stages its 32 x 32 outputs
// and a halo of ORDER / 2 (with the box closure) in shared memory once,
// so each value of V is read from memory about once instead of once per
// stencil point; 32 x 8 threads, four rows each.  The Laplacian sums its
// terms in the order of lap_global.
constexpr int kFsTX = 32, kFsTY = 32;

template <typename T, int ORDER>
__global__ void __launch_bounds__(256)
    k_first_step2d(int nx, int ny, const T* __restrict__ vin, T* __restrict__ D1, T* __restrict__ W1,
                   T* __restrict__ vout, Stencil<T> s, T c0, T c1, int64_t fstride, int64_t fpitch) {
    constexpr int R = ORDER / 2, SX = kFsTX + 2 * R, SY = kFsTY + 2 * R;
    __shared__ __align__(16) unsigned char sv_raw[sizeof(T) * SY * SX];  // raw: T may be a pair type
    T* sv = reinterpret_cast<T*>(sv_raw);
    const int64_t N = (int64_t)nx * ny, v = blockIdx.z;
    vin += v * N;
    vout += v * N;
    D1 += v * fstride;
    W1 += v * fstride;
    const int x0 = blockIdx.x * kFsTX, y0 = blockIdx.y * kFsTY;
    const int cbx = axis_bc(s.bc, 0), cby = axis_bc(s.bc, 1);
    const int tid = threadIdx.y * kFsTX + threadIdx.x;
    for (int c = tid; c < SX * SY; c += 256) {
        const int sy = c / SX, sx = c - sy * SX;
        const int gx = x0 - R + sx, gy = y0 - R + sy;
        int sgx = 1, sgy = 1;
        const int ix = (gx >= 0 && gx < nx) ? gx : ext_axis<int>(gx, nx, cbx, sgx);
        const int iy = (gy >= 0 && gy < ny) ? gy : ext_axis<int>(gy, ny, cby, sgy);
        T val = T(0);
        if (ix >= 0 && iy >= 0) {
            val = vin[(int64_t)iy * nx + ix];
            if (sgx * sgy < 0) val = -val;
        }
        sv[c] = val;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kFsTY / 8; ++r) {
        const int yy = threadIdx.y + 8 * r, gx = x0 + threadIdx.x, gy = y0 + yy;
        if (gx >= nx || gy >= ny) continue;
        const int q = (yy + R) * SX + threadIdx.x + R;
        const T x = sv[q];
        T d = s.c0 * x;
        d += s.c1[0] * (sv[q - 1] + sv[q + 1]);
        d += s.c1[1] * (sv[q - SX] + sv[q + SX]);
        if (ORDER == 4) {
            d += s.c2[0] * (sv[q - 2] + sv[q + 2]);
            d += s.c2[1] * (sv[q - 2 * SX] + sv[q + 2 * SX]);
        }
        const T w1 = x + d;
        const int64_t qf = (int64_t)gy * fpitch + gx;
        D1[qf] = d;
        W1[qf] = w1;
        vout[(int64_t)gy * nx + gx] = c0 * x + c1 * w1;
    }
}

// one step: D <- D + dt^2 L W (in place), Wout <- W + D, acc += c Wout
template <typename T, int DIM, int ORDER>
__global__ void k_step_simple(int64_t nx, int64_t ny, int64_t nz, const T* __restrict__ W,
                              T* __restrict__ D, T* __restrict__ Wout, T* __restrict__ acc, Stencil<T> s, T c,
                              int64_t fstride) {
    const int64_t N = nx * ny * nz;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int64_t v = blockIdx.z / nz, k = blockIdx.z - v * nz, j = blockIdx.y, q = (k * ny + j) * nx + i;
    W += v * fstride;
    D += v * fstride;
    Wout += v * fstride;
    acc += v * N;
    T d = D[q] + lap_global<T, DIM, ORDER>(W, s, q, i, j, k, nx, ny, nz);
    T wn = W[q] + d;
    D[q] = d;
    Wout[q] = wn;
    acc[q] += c * wn;
}

// ---------------------------------------------------------------------------
// whole wave-solve of a small 2D grid in one CTA
// ---------------------------------------------------------------------------
// boundary and ghost layers of a whole padded 2D grid (pitch PX, G = 2
// layers on every side) from the box closure: Dirichlet walls 0, beyond them
// the odd reflection, Neumann ghosts the even reflection.  The cross-shaped
// stencils never read the corner blocks.
template <typename T, int R>
__device__ __forceinline__ void resident_fix(T* buf, int nx, int ny, int PX, int bc, int tid, int nthr) {
    constexpr int G = 2;
    if (R != 2 && bc == 0) return;  // order 2 with Dirichlet walls reads only the zero wall layer
    const int bx = axis_bc(bc, 0), by = axis_bc(bc, 1);
    for (int q = tid; q < 2 * G * (ny + nx); q += nthr) {
        const int layer = q % G + 1, side = (q / G) & 1, r = q / (2 * G);
        int sg = 1;
        if (r < ny) {  // x-ghost of row r
            const int gx = side ? nx - 1 + layer : -layer;
            const int ix = ext_axis<int>(gx, nx, bx, sg);
            const T v = ix < 0 ? T(0) : buf[(r + G) * PX + ix + G];
            buf[(r + G) * PX + gx + G] = sg < 0 ? -v : v;
        } else {  // y-ghost of column x
            const int x = r - ny;
            const int gy = side ? ny - 1 + layer : -layer;
            const int iy = ext_axis<int>(gy, ny, by, sg);
            const T v = iy < 0 ? T(0) : buf[(iy + G) * PX + x + G];
            buf[(gy + G) * PX + x + G] = sg < 0 ? -v : v;
        }
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(1024)
    k_resident2d(int nx, int ny, const T* __restrict__ vin, T* __restrict__ vout,
                 const T* __restrict__ cw, int64_t Nt, Stencil<T> st, Stencil<T> st_half) {
    constexpr int G = 2;
    const int PX = nx + 2 * G, PY = ny + 2 * G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sA = reinterpret_cast<T*>(smem_raw);
    T* sB = sA + PX * PY;
    T* sAcc = sB + PX * PY;
    const int64_t N = (int64_t)nx * ny;
    vin += blockIdx.x * N;
    vout += blockIdx.x * N;
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;

    auto fix = [&](T* buf) { resident_fix<T, R>(buf, nx, ny, PX, st.bc, tid, nthr); };
    auto lap = [&](const T* c, int p, const Stencil<T>& s) {
        T r = s.c0 * c[p] + s.c1[0] * (c[p - 1] + c[p + 1]) + s.c1[1] * (c[p - PX] + c[p + PX]);
        if (R == 2) r += s.c2[0] * (c[p - 2] + c[p + 2]) + s.c2[1] * (c[p - 2 * PX] + c[p + 2 * PX]);
        return r;
    };

    // sA: W^n with its boundary and ghost layers; sB: D^n (same layout)
    for (int q = tid; q < PX * PY; q += nthr) {
        sA[q] = T(0);
        sB[q] = T(0);
    }
    __syncthreads();
    for (int q = tid; q < N; q += nthr) {
        int x = q % nx, y = q / nx;
        sA[(y + G) * PX + x + G] = vin[q];
    }
    __syncthreads();
    fix(sA);
    __syncthreads();
    // first step (eq. explicitStep1): D^1 = (dt^2/2) L W^0, then W^1 = W^0 + D^1
    const T c0 = cw[0], c1 = cw[1];
    for (int q = tid; q < N; q += nthr) {
        int x = q % nx, y = q / nx;
        int p = (y + G) * PX + x + G;
        sB[p] = lap(sA, p, st_half);
    }
    __syncthreads();
    for (int q = tid; q < N; q += nthr) {
        int x = q % nx, y = q / nx;
        int p = (y + G) * PX + x + G;
        T x0 = sA[p];
        T w1 = x0 + sB[p];
        sA[p] = w1;
        sAcc[q] = c0 * x0 + c1 * w1;
    }
    __syncthreads();
    fix(sA);
    __syncthreads();
    for (int64_t n = 1; n < Nt; ++n) {
        const T cn = cw[n + 1];
        // D^{n+1} = D^n + dt^2 L W^n everywhere, then W^{n+1} = W^n + D^{n+1} pointwise
        for (int q = tid; q < N; q += nthr) {
            int x = q % nx, y = q / nx;
            int p = (y + G) * PX + x + G;
            sB[p] = sB[p] + lap(sA, p, st);
        }
        __syncthreads();
        for (int q = tid; q < N; q += nthr) {
            int x = q % nx, y = q / nx;
            int p = (y + G) * PX + x + G;
            T wn = sA[p] + sB[p];
            sA[p] = wn;
            sAcc[q] += cn * wn;
        }
        __syncthreads();
        fix(sA);
        __syncthreads();
    }
    for (int q = tid; q < N; q += nthr) vout[q] = sAcc[q];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// one thread per point: x from the block's threads, y from grid.y, z and the
// vector from grid.z (no integer division by the grid shape in the kernels)
static int pt_threads(int64_t nx) { return nx >= 128 ? 128 : (int)(((nx + 31) / 32) * 32); }
static dim3 pt_grid(const GridGeom& g, int nvec) {
    const int t = pt_threads(g.n[0]);
    const int64_t nz = g.dim == 3 ? g.n[2] : 1;
    return dim3((unsigned)((g.n[0] + t - 1) / t), (unsigned)g.n[1], (unsigned)(nz * nvec));
}

static ew_status pt_check(const GridGeom& g, int nvec) {
    const int64_t nz = g.dim == 3 ? g.n[2] : 1;
    if (g.n[1] > 65535 || nz * nvec > 65535)
        return set_error(EW_EUNSUPPORTED, "grid too long in y, or z x vectors too many (at most 65535)");
    return EW_OK;
}


template <typename T>
ew_status launch_apply_L(const GridGeom& g, const T* u, T* Lu, int nvec, double scale,
                         cudaStream_t st) {
    if (g.map) return mapped_apply_L<T>(g, u, Lu, nvec, scale, st);
    Stencil<T> s = make_stencil<T>(g, scale);
    EW_TRY(pt_check(g, nvec));
    dim3 grid = pt_grid(g, nvec), blk(pt_threads(g.n[0]));
    if (g.dim == 2 && g.order == 2)
        k_apply_L<T, 2, 2><<<grid, blk, 0, st>>>(g.n[0], g.n[1], 1, u, Lu, s);
    else if (g.dim == 2)
        k_apply_L<T, 2, 4><<<grid, blk, 0, st>>>(g.n[0], g.n[1], 1, u, Lu, s);
    else if (g.order == 2)
        k_apply_L<T, 3, 2><<<grid, blk, 0, st>>>(g.n[0], g.n[1], g.n[2], u, Lu, s);
    else
        k_apply_L<T, 3, 4><<<grid, blk, 0, st>>>(g.n[0], g.n[1], g.n[2], u, Lu, s);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}
template ew_status launch_apply_L<float>(const GridGeom&, const float*, float*, int, double,
                                         cudaStream_t);
template ew_status launch_apply_L<double>(const GridGeom&, const double*, double*, int, double,
                                          cudaStream_t);

template <typename T>
static size_t resident_smem(const GridGeom& g) {
    return sizeof(T) * ((size_t)2 * (g.n[0] + 4) * (g.n[1] + 4) + (size_t)g.n[0] * g.n[1]);
}

template <typename T>
ew_status step3d(const GridGeom& g, const T* W, T* D, T* Wout, T* acc, T c, const Stencil<T>& s, int nvec,
                 int64_t fstride, cudaStream_t st);

template <typename T>
ew_status first_step(const GridGeom& g, const T* vin, T* D1, T* W1, T* vout,
                            const FilterPlan& plan, int nvec, int64_t fstride, cudaStream_t st, int64_t fpitch) {
    if (fpitch < g.n[0] || (g.dim == 3 && fpitch != g.n[0])) return set_error(EW_EINVAL, "first step: bad field pitch");
    Stencil<T> s = make_stencil<T>(g, 0.5 * plan.dt * plan.dt);
    EW_TRY(pt_check(g, nvec));
    dim3 grid = pt_grid(g, nvec), blk(pt_threads(g.n[0]));
    T c0 = T(plan.cn(0)), c1 = T(plan.cn(1));
    if (g.dim == 2) {
        const dim3 g2((unsigned)((g.n[0] + kFsTX - 1) / kFsTX), (unsigned)((g.n[1] + kFsTY - 1) / kFsTY),
                      (unsigned)nvec);
        if (g.order == 2)
            k_first_step2d<T, 2><<<g2, dim3(kFsTX, 8), 0, st>>>((int)g.n[0], (int)g.n[1], vin, D1, W1, vout, s, c0,
                                                                c1, fstride, fpitch);
        else
            k_first_step2d<T, 4><<<g2, dim3(kFsTX, 8), 0, st>>>((int)g.n[0], (int)g.n[1], vin, D1, W1, vout, s, c0,
                                                                c1, fstride, fpitch);
    } else if (g.order == 2)
        k_first_step<T, 3, 2><<<grid, blk, 0, st>>>(g.n[0], g.n[1], g.n[2], vin, D1, W1, vout, s, c0, c1, fstride, fpitch);
    else
        k_first_step<T, 3, 4><<<grid, blk, 0, st>>>(g.n[0], g.n[1], g.n[2], vin, D1, W1, vout, s, c0, c1, fstride, fpitch);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}

template <typename T>
static ew_status step_simple(const GridGeom& g, const T* W, T* D, T* Wout, T* acc, T c, const Stencil<T>& s,
                             int nvec, int64_t fstride, cudaStream_t st) {
    EW_TRY(pt_check(g, nvec));
    dim3 grid = pt_grid(g, nvec), blk(pt_threads(g.n[0]));
    cudaEvent_t ev = fused_begin(st);
    if (g.dim == 2 && g.order == 2)
        k_step_simple<T, 2, 2><<<grid, blk, 0, st>>>(g.n[0], g.n[1], 1, W, D, Wout, acc, s, c, fstride);
    else if (g.dim == 2)
        k_step_simple<T, 2, 4><<<grid, blk, 0, st>>>(g.n[0], g.n[1], 1, W, D, Wout, acc, s, c, fstride);
    else if (g.order == 2)
        k_step_simple<T, 3, 2><<<grid, blk, 0, st>>>(g.n[0], g.n[1], g.n[2], W, D, Wout, acc, s, c, fstride);
    else
        k_step_simple<T, 3, 4><<<grid, blk, 0, st>>>(g.n[0], g.n[1], g.n[2], W, D, Wout, acc, s, c, fstride);
    EW_CUDA_TRY(cudaGetLastError());
    fused_end(ev, st, g.N * nvec, g.N * nvec);
    return EW_OK;
}

template <typename T>
static ew_status resident(const GridGeom& g, const T* vin, T* vout, const T* cw, const FilterPlan& plan,
                          int nvec, cudaStream_t st) {
    Stencil<T> s = make_stencil<T>(g, plan.dt * plan.dt);
    Stencil<T> sh = make_stencil<T>(g, 0.5 * plan.dt * plan.dt);
    size_t smem = resident_smem<T>(g);
    int threads = (int)std::min<int64_t>(1024, ((g.N + 31) / 32) * 32);
    cudaEvent_t ev = fused_begin(st);
    if (g.order == 2) {
        EW_CUDA_TRY(cudaFuncSetAttribute(k_resident2d<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        k_resident2d<T, 1><<<nvec, threads, smem, st>>>((int)g.n[0], (int)g.n[1], vin, vout, cw, plan.Nt, s, sh);
    } else {
        EW_CUDA_TRY(cudaFuncSetAttribute(k_resident2d<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        k_resident2d<T, 2><<<nvec, threads, smem, st>>>((int)g.n[0], (int)g.n[1], vin, vout, cw, plan.Nt, s, sh);
    }
    EW_CUDA_TRY(cudaGetLastError());
    fused_end(ev, st, g.N * nvec, g.N * nvec * plan.Nt);
    return EW_OK;
}

// Resident path: small 2D grids whose three fields fit in one CTA's shared
// memory and would leave most SMs idle anyway.
template <typename T>
static bool use_resident(const GridGeom& g, int nvec) {
    return g.dim == 2 && resident_smem<T>(g) <= 200 * 1024 && g.N <= 16384 && nvec <= 4 * 152;
}

template <typename T>
ew_status explicit_wave_solve(const GridGeom& g, const FilterPlan& plan, const T* cdev, const T* vin, T* vout,
                              int nvec, T* fields, int temporal_block, cudaStream_t st) {
    if (temporal_block < 0) return set_error(EW_EINVAL, "temporal_block < 0");
    if constexpr (std::is_same<T, dd>::value) {
        // double-FP32 pairs: 2D boxes only (the blocked 2D, one-CTA and one-step kernels)
        if (g.map || g.dim != 2) return set_error(EW_EUNSUPPORTED, "double-FP32 fields: 2D boxes only");
    } else {
        if (g.map) return mapped_wave_solve<T>(g, plan, vin, vout, nvec, fields, st);  // one step per launch
    }
    // the variant override EW_TB2D_VARIANT (a tuning and testing hook) selects a
    // blocked kernel, so it also bypasses the one-CTA path of small grids
    if (use_resident<T>(g, nvec) && temporal_block == 0 && !getenv("EW_TB2D_VARIANT"))
        return resident<T>(g, vin, vout, cdev, plan, nvec, st);
    // fields are laid out [field][vector][point]; 2D rows may be padded (pitch2d)
    const int64_t fstride = wave_field_stride(g);
    T* F[4];
    for (int q = 0; q < 4; ++q) F[q] = fields + (int64_t)q * nvec * fstride;
    const bool blocked = g.dim == 2 && temporal_block != 1;
    // the tuner writes the spare fields and the filter sum, so it runs before the first step
    if (blocked && temporal_block == 0) EW_TRY(tb2d_tune<T>(g, plan, cdev, F, vout, nvec, fstride, st));
    if constexpr (!std::is_same<T, dd>::value)
        if (g.dim == 3 && g.order == 2 && temporal_block == 0)
            EW_TRY(tb3d_tune<T>(g, plan, cdev, F, vout, nvec, fstride, st));
    // F[0] = D^n, F[1] = W^n; the unblocked steps write W^{n+1} to F[2] and swap
    const int64_t fpitch =
        blocked ? tb2d_field_pitch<T>(g, plan, cdev, F, vout, nvec, fstride, temporal_block, st) : g.n[0];
    EW_TRY(first_step<T>(g, vin, F[0], F[1], vout, plan, nvec, fstride, st, fpitch));
    if (blocked) {
        int prv = 0, cur = 1;
        return tb2d_advance<T>(g, plan, cdev, F, &prv, &cur, 1, vout, nvec, fstride, temporal_block, st);
    }
    if constexpr (!std::is_same<T, dd>::value)
        if (g.dim == 3 && g.order == 2 && temporal_block != 1) {
            int prv = 0, cur = 1;
            return tb3d_advance<T>(g, plan, cdev, F, &prv, &cur, 1, vout, nvec, fstride, temporal_block, st);
        }
    Stencil<T> s = make_stencil<T>(g, plan.dt * plan.dt);
    int cur = 1, nxt = 2;
    for (int64_t L = 1; L < plan.Nt; ++L) {
        if constexpr (!std::is_same<T, dd>::value) {
            if (g.dim == 3) {
                EW_TRY(step3d<T>(g, F[cur], F[0], F[nxt], vout, T(plan.cn(L + 1)), s, nvec, fstride, st));
                std::swap(cur, nxt);
                continue;
            }
        }
        EW_TRY(step_simple<T>(g, F[cur], F[0], F[nxt], vout, T(plan.cn(L + 1)), s, nvec, fstride, st));
        std::swap(cur, nxt);
    }
    return EW_OK;
}
template ew_status explicit_wave_solve<float>(const GridGeom&, const FilterPlan&, const float*, const float*,
                                              float*, int, float*, int, cudaStream_t);
template ew_status explicit_wave_solve<double>(const GridGeom&, const FilterPlan&, const double*,
                                               const double*, double*, int, double*, int, cudaStream_t);
template ew_status explicit_wave_solve<dd>(const GridGeom&, const FilterPlan&, const dd*,
                                               const dd*, dd*, int, dd*, int, cudaStream_t);

}  // namespace ew

namespace ew {
template ew_status first_step<float>(const GridGeom&, const float*, float*, float*, float*, const FilterPlan&, int,
                                     int64_t, cudaStream_t, int64_t);
template ew_status first_step<double>(const GridGeom&, const double*, double*, double*, double*, const FilterPlan&,
                                      int, int64_t, cudaStream_t, int64_t);
}  // namespace ew
