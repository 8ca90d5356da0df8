// ew_mg.cu -- geometric multigrid for the implicit time-step systems and the
// implicit wave-solve (eqs. implicitScheme, impMatrix, implicitStep1).
//
//   M x = b,   M = I - a L_h,   a = dt^2 / 2
//
// One V(pre, post) cycle (the paper solves these systems with its multigrid
// solver and names red-black / line smoothers; this is the plain geometric
// cycle for Cartesian boxes):
//   levels      n_c = (n - 1) / 2 per axis while every axis has odd n >= 5
//               (coarse point I on fine point 2I + 1, h_c = 2 h)
//   smoother    damped Jacobi x <- x + w (b - M x) / D with the constant
//               interior diagonal D = 1 + a sum_i d0 / h_i^2 (d0 = 2 or 5/2),
//               or multi-colour Gauss-Seidel with the same diagonal (two
//               colours at second order, three at fourth), or the learned
//               correction x <- x + N(b - M x) on the finest `learned_levels`
//               levels (ew_smoother.cu, applied as its composed stencil in
//               FP32, ew_smoother_comp.cu)
//   restriction full weighting, tensor product of (1/4, 1/2, 1/4)
//   prolongation (multi)linear interpolation, zero on the boundary
//   coarsest    conjugate gradients in one CTA (M is SPD)
//
// Implicit wave-solve (one application of S):
//   M W^1 = W^0;  M y = 2 W^n, W^{n+1} = y - W^{n-1};  V_out = sum c_n W^n
// Each system gets `max_cycles` V-cycles (or stops at `rtol`) from the
// initial guess y = 2 W^n (W^1 = W^0 for the first step) or, with
// guess = 1, from the previous system's solution.
// Kernels: 3D levels run their stencil operations 2.5D blocked
// (k_mg_plane3d), 2D levels one thread per point.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "ew_internal.h"
#include "ew_stencil_dev.cuh"

namespace ew {

// learned correction x += N(r) (ew_smoother.cu)
template <typename T>
ew_status smoother_apply(const GridGeom& g, const float* weights, const T* r, T* x, cudaStream_t st);

struct MGLevel {
    GridGeom geom;
};

int mg_levels(const GridGeom& g, GridGeom* lv, int maxlev) {
    int L = 0;
    lv[0] = g;
    for (;;) {
        bool ok = L + 1 < maxlev;
        for (int a = 0; a < g.dim; ++a)
            if (lv[L].n[a] < 5 || (lv[L].n[a] % 2) == 0) ok = false;
        if (!ok) break;
        GridGeom c = lv[L];
        c.N = 1;
        for (int a = 0; a < 3; ++a) {
            if (a < g.dim) {
                c.n[a] = (lv[L].n[a] - 1) / 2;
                c.h[a] = 2.0 * lv[L].h[a];
            }
            c.N *= c.n[a];
        }
        lv[++L] = c;
    }
    return L + 1;
}

static int grid_blocks(int64_t N, int threads) {
    int64_t b = (N + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// one thread per point: x from the block's threads, y and z from the grid (no
// integer division in the kernels)
static int pt_threads(int64_t nx) { return nx >= 128 ? 128 : (int)(((nx + 31) / 32) * 32); }
static dim3 pt_grid(int64_t nx, int64_t ny, int64_t nz) {
    const int t = pt_threads(nx);
    return dim3((unsigned)((nx + t - 1) / t), (unsigned)ny, (unsigned)nz);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// r = b - M x = b - x + a L x   (sa carries the scale a)
template <typename T, int DIM, int ORDER>
__global__ void k_mg_resid(int64_t nx, int64_t ny, int64_t nz, const T* __restrict__ x, const T* __restrict__ b,
                           T* __restrict__ r, Stencil<T> sa) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int64_t j = blockIdx.y, k = blockIdx.z, q = (k * ny + j) * nx + i;
    r[q] = (b[q] - x[q]) + lap_global<T, DIM, ORDER>(x, sa, q, i, j, k, nx, ny, nz);
}

// x_out = x_in + wd (b - M x_in), wd = w / D
template <typename T, int DIM, int ORDER>
__global__ void k_mg_jacobi(int64_t nx, int64_t ny, int64_t nz, const T* __restrict__ x, const T* __restrict__ b,
                            T* __restrict__ xo, Stencil<T> sa, T wd) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int64_t j = blockIdx.y, k = blockIdx.z, q = (k * ny + j) * nx + i;
    T r = (b[q] - x[q]) + lap_global<T, DIM, ORDER>(x, sa, q, i, j, k, nx, ny, nz);
    xo[q] = x[q] + wd * r;
}

// multi-colour Gauss-Seidel, in place: the points of one colour take
// x += (b - M x) * inv_d, M_ii = 1 / inv_d.  Second order: red-black, colour
// (i + j + k) & 1.  Fourth order (offsets of 1 and 2 along one axis): three
// colours, (i + j + k) mod 3; an offset changes the colour by +-1 or +-2, never
// 0 mod 3.  So no point of a colour reads another point of its colour, the
// colour's updates are independent, and the sweep is exact Gauss-Seidel in
// colour order
template <int ORDER>
__device__ __forceinline__ int mg_colour(int64_t i, int64_t j, int64_t k) {
    return ORDER == 2 ? (int)((i + j + k) & 1) : (int)((i + j + k) % 3);
}

template <typename T, int ORDER>
__global__ void k_mg_rbgs(int64_t nx, int64_t ny, T* __restrict__ x, const T* __restrict__ b, Stencil<T> sa, T inv_d,
                          int colour) {  // 2D levels (3D: k_mg_plane3d, MODE 2)
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int64_t j = blockIdx.y, q = j * nx + i;
    if (mg_colour<ORDER>(i, j, 0) != colour) return;
    const T r = (b[q] - x[q]) + lap_global<T, 2, ORDER>(x, sa, q, i, j, 0, nx, ny, 1);
    x[q] = x[q] + inv_d * r;
}

// ---------------------------------------------------------------------------
// 3D stencil operations of the cycle, 2.5D blocked: a CTA owns 64 x 8 columns
// and a chunk of planes and streams along z through a ring of kPlS staged
// planes (each with a halo of R = ORDER / 2 in x and y).  The planes are
// filled by asynchronous copies kPlD planes ahead of the one the stencil needs
// next, so the loads of several planes are in flight while a plane is
// computed, and every value of x is read from memory about once.  b goes
// through a ring of its own (no halo).  Dirichlet box closure (the multigrid
// levels have no Neumann faces): a wall point is 0, a point beyond it the
// negated mirror; each staged cell is either 0 or a copy of one point of the
// box, negated by the thread that copied it once the copy has landed.
// MODE 0: out = r = b - M x; MODE 1: out = x + wd (b - M x) (Jacobi); MODE 2:
// the colour sweep in place (out == x), x += wd (b - M x) at the points of
// colour `colour` (mg_colour).  The Laplacian sums its terms in the order of
// lap_global.
constexpr int kPlBX = 64, kPlBY = 8, kPlNT = 256, kPlD = 2;

// index of coordinate i on an axis of n points under the odd closure
// (|i - clamp| <= 2): -1 for a wall point, else the mirror with sg negated
__device__ __forceinline__ int mg_ext(int i, int n, int& sg) {
    if (i >= 0 && i < n) return i;
    if (i == -1 || i == n) return -1;
    sg = -sg;
    return i < 0 ? -2 - i : 2 * n - i;
}

template <typename T>
__device__ __forceinline__ void mg_cp_async(T* dst, const T* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void mg_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void mg_cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T, int ORDER>
struct PlaneRing {
    static constexpr int R = ORDER == 2 ? 1 : 2;
    static constexpr int SX = kPlBX + 2 * R, SY = kPlBY + 2 * R, CELLS = SX * SY;
    static constexpr int S = 2 * R + 1 + kPlD;                 // planes z - R .. z + R + kPlD
    static constexpr int PER = (CELLS + kPlNT - 1) / kPlNT;    // staged cells per thread and plane
    static constexpr int BPER = kPlBX * kPlBY / kPlNT;         // b cells per thread and plane
    static constexpr size_t SMEM = sizeof(T) * (size_t)S * (CELLS + kPlBX * kPlBY);
    static_assert(PER * S <= 32, "negation flags of the ring fit one word");
};

template <typename T, int ORDER, int MODE>
__global__ void __launch_bounds__(kPlNT)
    k_mg_plane3d(int nx, int ny, int nz, int zc, const T* x, const T* __restrict__ b, T* out, Stencil<T> sa, T wd,
                 int colour) {
    using PR = PlaneRing<T, ORDER>;
    constexpr int R = PR::R, SX = PR::SX, CELLS = PR::CELLS, S = PR::S, PER = PR::PER, BPER = PR::BPER;
    extern __shared__ __align__(16) unsigned char mg_smem[];
    T* ring = reinterpret_cast<T*>(mg_smem);  // [S][CELLS]
    T* bring = ring + (size_t)S * CELLS;      // [S][kPlBX * kPlBY]
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kPlBX, y0 = blockIdx.y * kPlBY;
    const int z0 = blockIdx.z * zc, z1 = min(nz, z0 + zc);
    const int64_t plane = (int64_t)nx * ny;
    unsigned neg = 0;  // bit (slot * PER + u): this thread's cell u of ring slot `slot` awaits negation
    // the thread's staged cells, the same in every plane: offset of the source
    // column in a plane (-1: 0 for every plane), and which are negated mirrors
    int coff[PER];
    unsigned cneg = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int c = tid + kPlNT * u;
        const int sy = c / SX, sx = c - sy * SX;
        const int hx = x0 - R + sx, hy = y0 - R + sy;
        int sg = 1;
        const int ex = hx < nx + R ? mg_ext(hx, nx, sg) : -1;  // past a ragged tile's reach: never read
        const int ey = hy < ny + R ? mg_ext(hy, ny, sg) : -1;
        coff[u] = (c < CELLS && ex >= 0 && ey >= 0) ? ey * nx + ex : -1;
        if (sg < 0) cneg |= 1u << u;
    }
    int boff[BPER];
#pragma unroll
    for (int u = 0; u < BPER; ++u) {
        const int c = tid + kPlNT * u;
        const int cy = c / kPlBX, cx = c - cy * kPlBX;
        boff[u] = (x0 + cx < nx && y0 + cy < ny) ? (y0 + cy) * nx + x0 + cx : -1;
    }
    // stage plane p (any integer in [z0 - R, z1 + R)) into its slot, and b of plane p (when inside [z0, z1))
    auto issue = [&](int p) {
        if (p >= z1 + R) {  // past the chunk's last stencil plane: an empty group keeps the count
            mg_cp_commit();
            return;
        }
        const int slot = ((p % S) + S) % S;
        T* dst = ring + (size_t)slot * CELLS;
        int sgz = 1;
        const int ez = mg_ext(p, nz, sgz);
        const T* xp = x + (int64_t)(ez < 0 ? 0 : ez) * plane;
        const unsigned flip = sgz < 0 ? (1u << PER) - 1 : 0u;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int c = tid + kPlNT * u;
            if (c >= CELLS) break;
            if (ez < 0 || coff[u] < 0) {
                dst[c] = T(0);
            } else {
                mg_cp_async(dst + c, xp + coff[u]);
                if (((cneg ^ flip) >> u) & 1u) neg |= 1u << (slot * PER + u);
            }
        }
        if (p >= z0 && p < z1) {
            T* bd = bring + (size_t)slot * (kPlBX * kPlBY);
            const T* bp = b + (int64_t)p * plane;
#pragma unroll
            for (int u = 0; u < BPER; ++u)
                if (boff[u] >= 0) mg_cp_async(bd + tid + kPlNT * u, bp + boff[u]);
        }
        mg_cp_commit();
    };
    auto negate = [&](int p) {  // after its copies landed: this thread's negated cells of plane p
        const int slot = ((p % S) + S) % S;
        T* dst = ring + (size_t)slot * CELLS;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const unsigned bit = 1u << (slot * PER + u);
            if (neg & bit) {
                dst[tid + kPlNT * u] = -dst[tid + kPlNT * u];
                neg &= ~bit;
            }
        }
    };
    // prologue: planes z0 - R .. z0 + R + kPlD - 1, one group each
    for (int p = z0 - R; p < z0 + R + kPlD; ++p) issue(p);
    const T c1x = sa.c1[0], c1y = sa.c1[1], c1z = sa.c1[2], c2x = sa.c2[0], c2y = sa.c2[1], c2z = sa.c2[2];
    const int tx = tid % kPlBX, ty0 = tid / kPlBX;  // rows ty0 and ty0 + 4
    for (int z = z0; z < z1; ++z) {
        // plane z + R's group and every older one have landed (kPlD - 1 younger groups may be in flight)
        mg_cp_wait<kPlD - 1>();
        if (z == z0)
            for (int p = z0 - R; p <= z0 + R; ++p) negate(p);
        else
            negate(z + R);
        __syncthreads();  // plane z + R visible to all; every read of iteration z - 1 done
        issue(z + R + kPlD);  // into the slot of plane z - R - 1, last read in iteration z - 1
        const T* pc = ring + (size_t)(z % S) * CELLS;
        const T* bz = bring + (size_t)(z % S) * (kPlBX * kPlBY);
#pragma unroll
        for (int rr = 0; rr < kPlBY / 4; ++rr) {
            const int ty = ty0 + 4 * rr;
            const int gx = x0 + tx, gy = y0 + ty;
            if (gx >= nx || gy >= ny) continue;
            const int cc = (ty + R) * SX + tx + R;
            const T xc = pc[cc];
            T lap = sa.c0 * xc;
            lap += c1x * (pc[cc - 1] + pc[cc + 1]);
            lap += c1y * (pc[cc - SX] + pc[cc + SX]);
            lap += c1z * (ring[(size_t)((z - 1 + S) % S) * CELLS + cc] + ring[(size_t)((z + 1) % S) * CELLS + cc]);
            if (ORDER == 4) {
                lap += c2x * (pc[cc - 2] + pc[cc + 2]);
                lap += c2y * (pc[cc - 2 * SX] + pc[cc + 2 * SX]);
                lap += c2z * (ring[(size_t)((z - 2 + S) % S) * CELLS + cc] + ring[(size_t)((z + 2) % S) * CELLS + cc]);
            }
            const T r = (bz[ty * kPlBX + tx] - xc) + lap;
            const int64_t qi = (int64_t)z * plane + (int64_t)gy * nx + gx;
            if (MODE == 0) out[qi] = r;
            if (MODE == 1) out[qi] = xc + wd * r;
            if (MODE == 2 && mg_colour<ORDER>(gx, gy, z) == colour) out[qi] = xc + wd * r;
        }
    }
    mg_cp_wait<0>();  // no copy outlives the CTA
}

template <typename T>
__device__ __forceinline__ T get0(const T* __restrict__ v, int64_t i, int64_t j, int64_t k, int64_t nx, int64_t ny,
                                  int64_t nz) {
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return T(0);
    return v[(k * ny + j) * nx + i];
}

// full weighting: bc(I) = sum_o w(o) r(2I + 1 + o); x_c = 0
template <typename T, int DIM>
__global__ void k_mg_restrict(int64_t fx, int64_t fy, int64_t fz, int64_t cx, int64_t cy, int64_t cz,
                              const T* __restrict__ r, T* __restrict__ bc, T* __restrict__ xc) {
    const T w[3] = {T(0.25), T(0.5), T(0.25)};
    {
        const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (I >= cx) return;
        const int64_t J = blockIdx.y, K = blockIdx.z, q = (K * cy + J) * cx + I;
        int64_t fi = 2 * I + 1, fj = 2 * J + 1, fk = DIM == 3 ? 2 * K + 1 : 0;
        T s = T(0);
        for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    T wt = w[ox + 1] * w[oy + 1] * (DIM == 3 ? w[oz + 1] : T(1));
                    s += wt * get0(r, fi + ox, fj + oy, fk + oz, fx, fy, fz);
                }
        bc[q] = s;
        xc[q] = T(0);
    }
}

// x_f += P e_c (linear interpolation per axis)
template <typename T, int DIM>
__global__ void k_mg_prolong(int64_t fx, int64_t fy, int64_t fz, int64_t cx, int64_t cy, int64_t cz,
                             const T* __restrict__ ec, T* __restrict__ xf) {
    {
        const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i >= fx) return;
        const int64_t j = blockIdx.y, k = blockIdx.z, q = (k * fy + j) * fx + i;
        // per axis the coarse neighbours c, c + 1 and their weights: an odd fine index lies on
        // coarse point (i - 1) / 2 (weight 1, the second weight 0), an even one between two
        // (1/2 each); fixed trip counts keep everything in registers, and skipping the zero
        // weights leaves the same terms in the same order
        const int64_t ci = (i & 1) ? (i - 1) / 2 : i / 2 - 1;
        const int64_t cj = (j & 1) ? (j - 1) / 2 : j / 2 - 1;
        const int64_t ck = DIM == 2 ? 0 : ((k & 1) ? (k - 1) / 2 : k / 2 - 1);
        const T wi[2] = {(i & 1) ? T(1) : T(0.5), (i & 1) ? T(0) : T(0.5)};
        const T wj[2] = {(j & 1) ? T(1) : T(0.5), (j & 1) ? T(0) : T(0.5)};
        const T wk[2] = {(DIM == 2 || (k & 1)) ? T(1) : T(0.5), (DIM == 2 || (k & 1)) ? T(0) : T(0.5)};
        T s = T(0);
#pragma unroll
        for (int c3 = 0; c3 < (DIM == 3 ? 2 : 1); ++c3)
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
                for (int c1 = 0; c1 < 2; ++c1)
                    if (wi[c1] != T(0) && wj[c2] != T(0) && wk[c3] != T(0))
                        s += wi[c1] * wj[c2] * wk[c3] * get0(ec, ci + c1, cj + c2, ck + c3, cx, cy, cz);
        xf[q] += s;
    }
}

// coarsest level: CG in one CTA, all vectors in shared memory (N <= kCoarseMax)
constexpr int kCoarseMax = 2048;
constexpr int kCoarseThreads = 512;

template <typename T>
__device__ T block_dot(const T* a, const T* b, int N, T* red) {
    T s = T(0);
    for (int q = threadIdx.x; q < N; q += blockDim.x) s += a[q] * b[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    T t = T(0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

template <typename T, int DIM, int ORDER>
__global__ void __launch_bounds__(kCoarseThreads)
    k_mg_coarse_cg(int nx, int ny, int nz, const T* __restrict__ b, T* __restrict__ x, Stencil<T> sa, T rtol,
                   int maxit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = nx * ny * nz;
    T* sx = reinterpret_cast<T*>(smem_raw);
    T* sr = sx + N;
    T* sp = sr + N;
    T* sq = sp + N;
    T* red = sq + N;
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
        sx[q] = T(0);
        sr[q] = b[q];
        sp[q] = b[q];
    }
    __syncthreads();
    T rr = block_dot(sr, sr, N, red);
    const T stop = rtol * rtol * rr;
    for (int it = 0; it < maxit && rr > stop && rr > T(0); ++it) {
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
            int i = q % nx, t = q / nx, j = t % ny, k = t / ny;
            sq[q] = sp[q] - lap_global<T, DIM, ORDER>(sp, sa, q, i, j, k, nx, ny, nz);  // M p
        }
        __syncthreads();
        T pq = block_dot(sp, sq, N, red);
        if (!(pq > T(0))) break;
        T alpha = rr / pq;
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
            sx[q] += alpha * sp[q];
            sr[q] -= alpha * sq[q];
        }
        __syncthreads();
        T rr2 = block_dot(sr, sr, N, red);
        T beta = rr2 / rr;
        rr = rr2;
        for (int q = threadIdx.x; q < N; q += blockDim.x) sp[q] = sr[q] + beta * sp[q];
        __syncthreads();
    }
    for (int q = threadIdx.x; q < N; q += blockDim.x) x[q] = sx[q];
}

template <typename T>
__global__ void k_guess_rhs(int64_t N, const T* __restrict__ w, T* __restrict__ b, T* __restrict__ x, T sc) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        T v = sc * w[q];
        b[q] = v;
        if (x) x[q] = v;  // x == nullptr: keep the iterate as the guess
    }
}

// W^{n+1} = y - W^{n-1} (stored over W^{n-1}); acc += c W^{n+1}; first: acc = c0 W^0 + c1 W^1
template <typename T>
__global__ void k_implicit_update(int64_t N, const T* __restrict__ y, T* __restrict__ wprev, T* __restrict__ acc, T c) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        T wn = y[q] - wprev[q];
        wprev[q] = wn;
        acc[q] += c * wn;
    }
}
template <typename T>
__global__ void k_implicit_first(int64_t N, const T* __restrict__ w0, const T* __restrict__ w1, T* __restrict__ acc,
                                 T c0, T c1) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        acc[q] = c0 * w0[q] + c1 * w1[q];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
struct MGSolver {
    GridGeom lv[16];
    int nlev = 0;
    T* X[16];  // iterate (two buffers per level, X points at the current one)
    T* Tm[16];
    T* B[16];
    T* R[16];
    double a = 0.0;
    ew_grid* gr = nullptr;
    const ew_mg_params* p = nullptr;
    double wJ = 0.8;
    cudaStream_t st = nullptr;
    // FP32 fields: the learned levels' smoother as its composed stencil (one
    // build per solver set-up); EW_SMOOTHER_TWO_LAYER=1 keeps the two-layer
    // tensor-core form instead (a comparison hook)
    ComposedSmoother comp[16];
    bool use_comp = false;

    ew_status setup(ew_grid* g, double a_, const ew_mg_params* params, cudaStream_t s) {
        gr = g;
        a = a_;
        p = params;
        st = s;
        wJ = params->jacobi_weight > 0 ? params->jacobi_weight : 0.8;
        if (g->geom.bc)
            return set_error(EW_EUNSUPPORTED, "multigrid: boxes with Neumann faces are not implemented");
        if (g->geom.map) return set_error(EW_EUNSUPPORTED, "multigrid: mapped grids are not implemented");
        if (g->prec == EW_FP32X2) return set_error(EW_EUNSUPPORTED, "multigrid: FP32 or FP64 grids only");
        nlev = mg_levels(g->geom, lv, 16);
        {
            int dev = 0;
            EW_CUDA_TRY(cudaGetDevice(&dev));
            EW_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            const int s2 = (int)PlaneRing<T, 2>::SMEM, s4 = (int)PlaneRing<T, 4>::SMEM;
            const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
            EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_plane3d<T, 2, 0>, A, s2));
            EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_plane3d<T, 2, 1>, A, s2));
            EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_plane3d<T, 2, 2>, A, s2));
            EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_plane3d<T, 4, 0>, A, s4));
            EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_plane3d<T, 4, 1>, A, s4));
            EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_plane3d<T, 4, 2>, A, s4));
            // resident CTAs a SM (the fewest over the modes): the z chunks fill them once
            int o = 0;
            pl_occ[0] = pl_occ[1] = 1 << 20;
            EW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mg_plane3d<T, 2, 0>, kPlNT, s2));
            pl_occ[0] = std::min(pl_occ[0], o);
            EW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mg_plane3d<T, 2, 1>, kPlNT, s2));
            pl_occ[0] = std::min(pl_occ[0], o);
            EW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mg_plane3d<T, 2, 2>, kPlNT, s2));
            pl_occ[0] = std::min(pl_occ[0], o);
            EW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mg_plane3d<T, 4, 0>, kPlNT, s4));
            pl_occ[1] = std::min(pl_occ[1], o);
            EW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mg_plane3d<T, 4, 1>, kPlNT, s4));
            pl_occ[1] = std::min(pl_occ[1], o);
            EW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mg_plane3d<T, 4, 2>, kPlNT, s4));
            pl_occ[1] = std::min(pl_occ[1], o);
            pl_occ[0] = std::max(pl_occ[0], 1);
            pl_occ[1] = std::max(pl_occ[1], 1);
        }
        if (g->geom.n[1] > 65535 || g->geom.n[2] > 65535)
            return set_error(EW_EUNSUPPORTED, "multigrid: axes longer than 65535 points");
        if (lv[nlev - 1].N > kCoarseMax)
            return set_error(EW_EUNSUPPORTED, "multigrid needs axes that halve down to at most 2048 coarse points "
                                              "(n = 2^k - 1 per axis, for example)");
        if (params->learned_levels > 0 && g->geom.dim != 3)
            return set_error(EW_EUNSUPPORTED, "the learned smoother is three-dimensional");
        if (params->learned_levels > 0 && !params->weights_dev)
            return set_error(EW_EINVAL, "learned_levels > 0 needs weights_dev");
        use_comp = sizeof(T) == 4 && params->learned_levels > 0 && !getenv("EW_SMOOTHER_TWO_LAYER");
        if (use_comp)
            for (int L = 0; L < std::min(params->learned_levels, nlev); ++L)
                EW_TRY(comp[L].build(params->weights_dev + (size_t)L * 432, st));
        size_t total = 0;
        for (int L = 0; L < nlev; ++L) total += 4 * (size_t)lv[L].N;
        EW_TRY(g->mgh.reserve(total * sizeof(T)));
        T* base = (T*)g->mgh.ptr;
        for (int L = 0; L < nlev; ++L) {
            X[L] = base;
            Tm[L] = base + lv[L].N;
            B[L] = base + 2 * lv[L].N;
            R[L] = base + 3 * lv[L].N;
            base += 4 * lv[L].N;
        }
        return EW_OK;
    }

    double diag(int L) const {
        double d0 = lv[L].order == 2 ? 2.0 : 2.5, s = 0.0;
        for (int q = 0; q < lv[L].dim; ++q) s += d0 / (lv[L].h[q] * lv[L].h[q]);
        return 1.0 + a * s;
    }

// 2D levels: one thread per point (3D levels go through k_mg_plane3d)
#define EW_MG_DISPATCH2D(KERN, GEOM, ...)                                                                \
    do {                                                                                                 \
        const GridGeom& g_ = (GEOM);                                                                     \
        dim3 grid_ = pt_grid(g_.n[0], g_.n[1], 1), blk_(pt_threads(g_.n[0]));                            \
        if (g_.order == 2)                                                                               \
            KERN<T, 2, 2><<<grid_, blk_, 0, st>>>(g_.n[0], g_.n[1], 1, __VA_ARGS__);                     \
        else                                                                                             \
            KERN<T, 2, 4><<<grid_, blk_, 0, st>>>(g_.n[0], g_.n[1], 1, __VA_ARGS__);                     \
        count_launch();                                                                                  \
    } while (0)

    // 3D levels: the 2.5D-blocked stencil kernel; 2D levels: one thread per point
    int nsm = 0, pl_occ[2] = {1, 1};  // SMs; resident plane-kernel CTAs a SM (order 2, order 4)
    template <int MODE>
    void plane3d(const GridGeom& g_, const T* x, const T* b, T* out, const Stencil<T>& sa, T wd, int colour) {
        const int nx = (int)g_.n[0], ny = (int)g_.n[1], nz = (int)g_.n[2];
        const int bx = (nx + kPlBX - 1) / kPlBX, by = (ny + kPlBY - 1) / kPlBY;
        // z chunks: enough CTAs to fill the resident slots once, at least 8 planes each
        const int nzc = std::max(1, (pl_occ[g_.order == 2 ? 0 : 1] * nsm) / std::max(1, bx * by));
        const int zc = std::max(std::min(8, nz), (nz + nzc - 1) / nzc);
        const dim3 grid((unsigned)bx, (unsigned)by, (unsigned)((nz + zc - 1) / zc));
        if (g_.order == 2)
            k_mg_plane3d<T, 2, MODE><<<grid, kPlNT, PlaneRing<T, 2>::SMEM, st>>>(nx, ny, nz, zc, x, b, out, sa, wd,
                                                                              colour);
        else
            k_mg_plane3d<T, 4, MODE><<<grid, kPlNT, PlaneRing<T, 4>::SMEM, st>>>(nx, ny, nz, zc, x, b, out, sa, wd,
                                                                              colour);
        count_launch();
    }
    void resid(int L, const Stencil<T>& sa) {
        if (lv[L].dim == 3)
            plane3d<0>(lv[L], X[L], B[L], R[L], sa, T(0), 0);
        else
            EW_MG_DISPATCH2D(k_mg_resid, lv[L], X[L], B[L], R[L], sa);
    }

    ew_status smooth(int L, int steps) {
        Stencil<T> sa = make_stencil<T>(lv[L], a);
        for (int s = 0; s < steps; ++s) {
            if (L < p->learned_levels) {
                resid(L, sa);
                if constexpr (sizeof(T) == 4) {
                    if (use_comp) {
                        EW_TRY(comp[L].apply(lv[L], R[L], X[L], st));
                        continue;
                    }
                }
                EW_TRY(smoother_apply<T>(lv[L], p->weights_dev + (size_t)L * 432, R[L], X[L], st));
            } else if (p->red_black) {
                // M_ii = 1 - c0 of the stored (consistent) stencil of a L_h
                const T inv_d = (T)(1.0 / (1.0 - (double)sa.c0));
                const GridGeom& g_ = lv[L];
                dim3 grid_ = pt_grid(g_.n[0], g_.n[1], 1), blk_(pt_threads(g_.n[0]));
                const int ncol = g_.order == 2 ? 2 : 3;
                for (int colour = 0; colour < ncol; ++colour) {
                    // one launch per colour: 3D levels the 2.5D kernel, 2D levels one thread per point
                    if (g_.dim == 3)
                        plane3d<2>(g_, X[L], B[L], X[L], sa, inv_d, colour);
                    else if (g_.order == 2)
                        k_mg_rbgs<T, 2><<<grid_, blk_, 0, st>>>(g_.n[0], g_.n[1], X[L], B[L], sa, inv_d, colour);
                    else
                        k_mg_rbgs<T, 4><<<grid_, blk_, 0, st>>>(g_.n[0], g_.n[1], X[L], B[L], sa, inv_d, colour);
                    if (g_.dim == 2) count_launch();
                }
            } else {
                T wd = (T)(wJ / diag(L));
                if (lv[L].dim == 3)
                    plane3d<1>(lv[L], X[L], B[L], Tm[L], sa, wd, 0);
                else
                    EW_MG_DISPATCH2D(k_mg_jacobi, lv[L], X[L], B[L], Tm[L], sa, wd);
                std::swap(X[L], Tm[L]);
            }
        }
        return EW_OK;
    }

    ew_status coarse(int L) {
        Stencil<T> sa = make_stencil<T>(lv[L], a);
        const GridGeom& c = lv[L];
        size_t smem = sizeof(T) * (4 * (size_t)c.N + 32);
        T rtol = sizeof(T) == 4 ? T(1e-7) : T(1e-14);
        int maxit = (int)std::min<int64_t>(4 * c.N + 10, 4000);
        if (c.dim == 2 && c.order == 2)
            k_mg_coarse_cg<T, 2, 2><<<1, kCoarseThreads, smem, st>>>((int)c.n[0], (int)c.n[1], 1, B[L], X[L], sa, rtol, maxit);
        else if (c.dim == 2)
            k_mg_coarse_cg<T, 2, 4><<<1, kCoarseThreads, smem, st>>>((int)c.n[0], (int)c.n[1], 1, B[L], X[L], sa, rtol, maxit);
        else if (c.order == 2)
            k_mg_coarse_cg<T, 3, 2><<<1, kCoarseThreads, smem, st>>>((int)c.n[0], (int)c.n[1], (int)c.n[2], B[L], X[L], sa, rtol, maxit);
        else
            k_mg_coarse_cg<T, 3, 4><<<1, kCoarseThreads, smem, st>>>((int)c.n[0], (int)c.n[1], (int)c.n[2], B[L], X[L], sa, rtol, maxit);
        count_launch();
        EW_CUDA_TRY(cudaGetLastError());
        return EW_OK;
    }

    ew_status vcycle(int L) {
        if (L == nlev - 1) return coarse(L);
        EW_TRY(smooth(L, p->pre));
        Stencil<T> sa = make_stencil<T>(lv[L], a);
        resid(L, sa);
        const GridGeom &f = lv[L], &c = lv[L + 1];
        const int fz = f.dim == 3 ? (int)f.n[2] : 1, cz = f.dim == 3 ? (int)c.n[2] : 1;
        if (f.dim == 2)
            k_mg_restrict<T, 2><<<pt_grid(c.n[0], c.n[1], cz), pt_threads(c.n[0]), 0, st>>>(
                f.n[0], f.n[1], fz, c.n[0], c.n[1], cz, R[L], B[L + 1], X[L + 1]);
        else
            k_mg_restrict<T, 3><<<pt_grid(c.n[0], c.n[1], cz), pt_threads(c.n[0]), 0, st>>>(
                f.n[0], f.n[1], fz, c.n[0], c.n[1], cz, R[L], B[L + 1], X[L + 1]);
        count_launch();
        EW_TRY(vcycle(L + 1));
        if (f.dim == 2)
            k_mg_prolong<T, 2><<<pt_grid(f.n[0], f.n[1], fz), pt_threads(f.n[0]), 0, st>>>(
                f.n[0], f.n[1], fz, c.n[0], c.n[1], cz, X[L + 1], X[L]);
        else
            k_mg_prolong<T, 3><<<pt_grid(f.n[0], f.n[1], fz), pt_threads(f.n[0]), 0, st>>>(
                f.n[0], f.n[1], fz, c.n[0], c.n[1], cz, X[L + 1], X[L]);
        count_launch();
        EW_TRY(smooth(L, p->post));
        EW_CUDA_TRY(cudaGetLastError());
        return EW_OK;
    }

    // the current top-level iterate lives in X[0]; callers load b into B[0]
    // and the initial guess into X[0]
    ew_status cycles(int ncyc) {
        for (int c = 0; c < ncyc; ++c) EW_TRY(vcycle(0));
        return EW_OK;
    }

    // ||v||_2 of a finest-level vector (FP64 reduction, synchronises)
    ew_status norm2(const T* v, double* out) {
        EW_TRY(gr->reduce.reserve(sizeof(double) * (kReduceBlocks + 8)));
        double* dpart = (double*)gr->reduce.ptr;
        double* dres = dpart + kReduceBlocks;
        EW_TRY(launch_dots<T>(v, v, lv[0].N, 1, dpart, dres, st));
        double h = 0.0;
        EW_CUDA_TRY(cudaMemcpyAsync(&h, dres, sizeof(double), cudaMemcpyDeviceToHost, st));
        EW_CUDA_TRY(cudaStreamSynchronize(st));
        *out = sqrt(h);
        return EW_OK;
    }

    // V-cycles until ||B - M X||_2 <= rtol ||B||_2, tested after every cycle,
    // or max_cycles; rtol <= 0 runs max_cycles without a test
    ew_status solve(int max_cycles, double rtol, int* used) {
        if (!(rtol > 0.0)) {
            *used = max_cycles;
            return cycles(max_cycles);
        }
        double bn = 0.0;
        EW_TRY(norm2(B[0], &bn));
        Stencil<T> sa = make_stencil<T>(lv[0], a);
        int c = 0;
        while (c < max_cycles) {
            EW_TRY(vcycle(0));
            ++c;
            resid(0, sa);
            double rk = 0.0;
            EW_TRY(norm2(R[0], &rk));
            if (rk <= rtol * bn) break;
        }
        *used = c;
        return EW_OK;
    }
};

template <typename T>
static ew_status coarse_smem_attr() {
    size_t smem = sizeof(T) * (4 * (size_t)kCoarseMax + 32);
    EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_coarse_cg<T, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_coarse_cg<T, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_coarse_cg<T, 3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EW_CUDA_TRY(cudaFuncSetAttribute(k_mg_coarse_cg<T, 3, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return EW_OK;
}

static ew_status check_mg(const ew_mg_params* mg) {
    if (!mg) return set_error(EW_EINVAL, "the implicit scheme needs multigrid parameters (params->mg)");
    if (mg->pre < 0 || mg->post < 0 || mg->pre + mg->post < 1) return set_error(EW_EINVAL, "bad smoothing counts");
    if (mg->max_cycles < 1) return set_error(EW_EINVAL, "max_cycles must be >= 1");
    if (mg->learned_levels < 0) return set_error(EW_EINVAL, "learned_levels < 0");
    if (mg->red_black != 0 && mg->red_black != 1) return set_error(EW_EINVAL, "red_black must be 0 or 1");
    if (mg->guess != 0 && mg->guess != 1) return set_error(EW_EINVAL, "guess must be 0 or 1");
    return EW_OK;
}

template <typename T>
static ew_status implicit_wave_solve_t(ew_grid* g, const FilterPlan& plan, const ew_filter_params* p, const T* vin,
                                       T* vout, int nvec, cudaStream_t st) {
    EW_TRY(check_mg(p->mg));
    EW_TRY(coarse_smem_attr<T>());
    const int64_t N = g->geom.N;
    MGSolver<T> mg;
    EW_TRY(mg.setup(g, 0.5 * plan.dt * plan.dt, p->mg, st));
    EW_TRY(g->fields.reserve(2 * (size_t)N * sizeof(T)));
    T* Wm = (T*)g->fields.ptr;  // W^{n-1}
    T* W0 = Wm + N;             // W^n
    const int blocks = grid_blocks(N, 256);
    for (int v = 0; v < nvec; ++v) {
        const T* x = vin + (size_t)v * N;
        T* acc = vout + (size_t)v * N;
        // W^0 = V; M W^1 = W^0 (initial guess W^0)
        EW_CUDA_TRY(cudaMemcpyAsync(Wm, x, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
        k_guess_rhs<T><<<blocks, 256, 0, st>>>(N, x, mg.B[0], mg.X[0], T(1));
        count_launch();
        int used = 0;
        EW_TRY(mg.solve(p->mg->max_cycles, p->mg->rtol, &used));
        count_mg_solve(used);
        EW_CUDA_TRY(cudaMemcpyAsync(W0, mg.X[0], N * sizeof(T), cudaMemcpyDeviceToDevice, st));
        k_implicit_first<T><<<blocks, 256, 0, st>>>(N, Wm, W0, acc, (T)plan.c[0], (T)plan.c[1]);
        count_launch();
        for (int64_t n = 1; n < plan.Nt; ++n) {
            // M y = 2 W^n from y = 2 W^n, or (guess 1, n >= 2) from the previous
            // system's solution, which X[0] still holds; W^{n+1} = y - W^{n-1} over W^{n-1}
            const bool keep = p->mg->guess == 1 && n >= 2;
            k_guess_rhs<T><<<blocks, 256, 0, st>>>(N, W0, mg.B[0], keep ? nullptr : mg.X[0], T(2));
            count_launch();
            EW_TRY(mg.solve(p->mg->max_cycles, p->mg->rtol, &used));
            count_mg_solve(used);
            k_implicit_update<T><<<blocks, 256, 0, st>>>(N, mg.X[0], Wm, acc, (T)plan.c[(size_t)n + 1]);
            count_launch();
            std::swap(Wm, W0);
        }
    }
    EW_CUDA_TRY(cudaGetLastError());
    return EW_OK;
}

ew_status implicit_wave_solve_any(ew_grid* g, const FilterPlan& plan, const ew_filter_params* p, const void* vin,
                                  void* vout, int nvec, cudaStream_t st) {
    if (g->prec == EW_FP32)
        return implicit_wave_solve_t<float>(g, plan, p, (const float*)vin, (float*)vout, nvec, st);
    return implicit_wave_solve_t<double>(g, plan, p, (const double*)vin, (double*)vout, nvec, st);
}

template <typename T>
ew_status launch_dots(const T* x, const T* y, int64_t N, int nvec, double* part, double* out, cudaStream_t st);

template <typename T>
static ew_status step_mg_t(ew_grid* g, double a, const T* rhs, T* x, const ew_mg_params* mp, double* conv,
                           int* cycles_done, cudaStream_t st) {
    EW_TRY(check_mg(mp));
    EW_TRY(coarse_smem_attr<T>());
    const int64_t N = g->geom.N;
    MGSolver<T> mg;
    EW_TRY(mg.setup(g, a, mp, st));
    EW_TRY(g->reduce.reserve(sizeof(double) * (kReduceBlocks + 8)));
    double* dpart = (double*)g->reduce.ptr;
    double* dres = dpart + kReduceBlocks;
    EW_CUDA_TRY(cudaMemcpyAsync(mg.B[0], rhs, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
    EW_CUDA_TRY(cudaMemcpyAsync(mg.X[0], x, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
    Stencil<T> sa = make_stencil<T>(g->geom, a);
    auto resid_norm = [&](double* out) -> ew_status {
        T* r = mg.R[0];
        {
            const GridGeom& gg = g->geom;
            dim3 grid_ = pt_grid(gg.n[0], gg.n[1], gg.dim == 3 ? gg.n[2] : 1), blk_(pt_threads(gg.n[0]));
            if (gg.dim == 3) {
                mg.template plane3d<0>(gg, mg.X[0], mg.B[0], r, sa, T(0), 0);
            } else {
                if (gg.order == 2)
                    k_mg_resid<T, 2, 2><<<grid_, blk_, 0, st>>>(gg.n[0], gg.n[1], 1, mg.X[0], mg.B[0], r, sa);
                else
                    k_mg_resid<T, 2, 4><<<grid_, blk_, 0, st>>>(gg.n[0], gg.n[1], 1, mg.X[0], mg.B[0], r, sa);
                count_launch();
            }
        }
        EW_TRY(launch_dots<T>(r, r, N, 1, dpart, dres, st));
        double h = 0.0;
        EW_CUDA_TRY(cudaMemcpyAsync(&h, dres, sizeof(double), cudaMemcpyDeviceToHost, st));
        EW_CUDA_TRY(cudaStreamSynchronize(st));
        *out = sqrt(h);
        return EW_OK;
    };
    double bnorm = 0.0, r0 = 0.0, rk = 0.0;
    EW_TRY(launch_dots<T>(rhs, rhs, N, 1, dpart, dres, st));
    EW_CUDA_TRY(cudaMemcpyAsync(&bnorm, dres, sizeof(double), cudaMemcpyDeviceToHost, st));
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    bnorm = sqrt(bnorm);
    EW_TRY(resid_norm(&r0));
    rk = r0;
    int c = 0;
    for (c = 0; c < mp->max_cycles; ++c) {
        if (mp->rtol > 0 && rk <= mp->rtol * bnorm) break;
        EW_TRY(mg.vcycle(0));
        if (mp->rtol > 0 || c + 1 == mp->max_cycles) EW_TRY(resid_norm(&rk));
    }
    EW_CUDA_TRY(cudaMemcpyAsync(x, mg.X[0], N * sizeof(T), cudaMemcpyDeviceToDevice, st));
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    if (conv) *conv = (c > 0 && r0 > 0) ? pow(rk / r0, 1.0 / c) : 0.0;
    if (cycles_done) *cycles_done = c;
    if (mp->rtol > 0 && rk > mp->rtol * bnorm) return set_error(EW_ENOCONV, "multigrid did not reach rtol");
    return EW_OK;
}

ew_status splitmix_uniform(int64_t n, uint64_t seed, double* out, cudaStream_t st);
template <typename S, typename D>
ew_status convert(int64_t n, const S* x, D* y, cudaStream_t st);

// Residual samples for training the learned smoother: for rhs number q
// (uniform [-1,1) from SplitMix64 stream seed + q) plain V-cycles run from
// x = 0, and the residual b - M x the finest-level smoother sees at the start
// of cycles 0, 1, 2 is recorded, until nsamples residuals (FP32) are stored.
ew_status mg_collect_residuals(ew_grid* g, double a, const ew_mg_params* mp, int nsamples, uint64_t seed, float* out,
                               cudaStream_t st) {
    EW_TRY(check_mg(mp));
    EW_TRY(coarse_smem_attr<float>());
    const int64_t N = g->geom.N;
    MGSolver<float> mg;
    EW_TRY(mg.setup(g, a, mp, st));
    DeviceBuffer tmp_buf;
    EW_TRY(tmp_buf.alloc(sizeof(double) * (size_t)N));
    double* tmp = tmp_buf.as<double>();
    Stencil<float> sa = make_stencil<float>(g->geom, a);
    ew_status s = EW_OK;
    int k = 0;
    for (uint64_t q = 0; k < nsamples && s == EW_OK; ++q) {
        s = splitmix_uniform(N, seed + q, tmp, st);
        if (s == EW_OK) s = convert<double, float>(N, tmp, mg.B[0], st);
        if (s != EW_OK) break;
        cudaMemsetAsync(mg.X[0], 0, sizeof(float) * N, st);
        for (int c = 0; c < 3 && k < nsamples && s == EW_OK; ++c) {
            float* r = out + (size_t)k * N;
            const GridGeom& gg = g->geom;
            mg.template plane3d<0>(gg, mg.X[0], mg.B[0], r, sa, 0.f, 0);
            ++k;
            s = mg.vcycle(0);
        }
    }
    cudaStreamSynchronize(st);
    return s;
}

// Convergence factor of ncycles V-cycles on M x = b, b uniform [-1,1) from
// stream seed, x = 0: (||r_n|| / ||r_1||)^(1 / (n - 1)), skipping the first
// cycle's transient.
ew_status mg_convergence(ew_grid* g, double a, const ew_mg_params* mp, int ncycles, uint64_t seed, double* rho,
                         cudaStream_t st) {
    const int64_t N = g->geom.N;
    DeviceBuffer tmp_buf, b_buf, x_buf;
    EW_TRY(tmp_buf.alloc(sizeof(double) * (size_t)N));
    EW_TRY(b_buf.alloc(sizeof(float) * (size_t)N));
    EW_TRY(x_buf.alloc(sizeof(float) * (size_t)N));
    double* tmp = tmp_buf.as<double>();
    float* b = b_buf.as<float>();
    float* x = x_buf.as<float>();
    ew_status s = splitmix_uniform(N, seed, tmp, st);
    if (s == EW_OK) s = convert<double, float>(N, tmp, b, st);
    cudaMemsetAsync(x, 0, sizeof(float) * N, st);
    ew_mg_params one = *mp;
    one.max_cycles = 1;
    one.rtol = 0.0;
    double c1 = 0.0;
    if (s == EW_OK) s = step_mg_t<float>(g, a, b, x, &one, &c1, nullptr, st);  // r_1 / r_0
    ew_mg_params rest = *mp;
    rest.max_cycles = std::max(1, ncycles - 1);
    rest.rtol = 0.0;
    double cr = 0.0;
    if (s == EW_OK) s = step_mg_t<float>(g, a, b, x, &rest, &cr, nullptr, st);
    cudaStreamSynchronize(st);
    *rho = cr;
    return s;
}

}  // namespace ew

using namespace ew;

extern "C" ew_status ew_implicit_step_mg(const ew_grid* grid, double half_dt2, const void* rhs, void* x,
                                         const ew_mg_params* mg, double* conv_factor, int* cycles_done,
                                         cudaStream_t stream) try {
    clear_error();
    if (!grid || !rhs || !x || !mg) return set_error(EW_EINVAL, "null argument");
    if (!(half_dt2 >= 0.0) || !std::isfinite(half_dt2)) return set_error(EW_EINVAL, "half_dt2 must be finite and >= 0");
    {
        const size_t bytes = (size_t)grid->geom.N * (grid->prec == EW_FP32 ? 4 : 8);
        const char* a = (const char*)rhs;
        const char* b = (const char*)x;
        if (a < b + bytes && b < a + bytes) return set_error(EW_EINVAL, "rhs and x overlap");
    }
    int dev = -1;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    if (grid->device >= 0 && grid->device != dev) return set_error(EW_EINVAL, "grid was created on another device");
    ew_grid* g = const_cast<ew_grid*>(grid);
    if (g->prec == EW_FP32)
        return step_mg_t<float>(g, half_dt2, (const float*)rhs, (float*)x, mg, conv_factor, cycles_done, stream);
    return step_mg_t<double>(g, half_dt2, (const double*)rhs, (double*)x, mg, conv_factor, cycles_done, stream);
} catch (...) {
    return abi_exception();
}
