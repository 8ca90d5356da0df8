// ew_tb2d.cu -- temporally blocked fused leapfrog + filter step for 2D grids.
//
// One launch advances every active point by b <= B time steps
// (eq. explicitScheme) and adds c_{n+1} W^{n+1} + ... + c_{n+b} W^{n+b} to the
// filter sum (eq. filterQuadrature) without leaving shared memory.
//
// Tiling.  A CTA owns a TX x TY tile.  It stages W^{n-1} and W^n over the tile
// plus a halo of H = R B points (R = stencil radius: 1 for order 2, 2 for
// order 4) in two shared-memory buffers, and updates the fixed "compute
// region" (the staged region minus an R-wide rim) B times.  Each step the
// valid part of the region shrinks by R, so after b steps the owned tile is
// exact; halo points are recomputed by several CTAs but only owned points are
// accumulated and stored.  W^{n+b-1}, W^{n+b} go to a second pair of global
// buffers because neighbouring CTAs still read the first pair.
//
// Threads.  A warp covers 32 consecutive columns of the compute region and
// each thread a column segment of KY rows, held as a sliding register window
// along y, so a point costs five shared-memory loads (centre column entry,
// x +- 1, x +- 2), the W^{n-1} load and one store per step, and the step needs
// one barrier.
//
// Boundary conditions without branches.  Points of the staged region outside
// the box are loaded with the odd extension of the grid function about the
// boundary lines (zero on the boundary lines, -u(mirror) beyond them, applied
// per axis and periodically with period 2(n+1) for tiny boxes).  The update
// is linear and uses the same instruction sequence at every point, and IEEE
// negation is exact, so the updated values stay the exact odd extension: the
// boundary lines stay 0 and the ghosts (two outside, read by the 4th-order
// stencil) stay -u(mirror), with no fix-up pass.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "ew_internal.h"

namespace ew {

// odd extension of an axis of length n about -1 and n: returns the interior
// index holding the value and its sign, or -1 for a zero (boundary line).
__device__ __forceinline__ int odd_ext(int p, int n, int& sign) {
    const int P = 2 * (n + 1);
    int q = (p + 1) % P;
    if (q < 0) q += P;
    q -= 1;  // q in [-1, 2n]
    if (q == -1 || q == n) return -1;
    if (q < n) {
        sign = 1;
        return q;
    }
    sign = -1;
    return 2 * n - q;
}

template <typename T>
__device__ __forceinline__ T load_ext(const T* __restrict__ u, int gx, int gy, int nx, int ny) {
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) return u[(int64_t)gy * nx + gx];
    int sx = 1, sy = 1;
    int ix = odd_ext(gx, nx, sx);
    int iy = odd_ext(gy, ny, sy);
    if (ix < 0 || iy < 0) return T(0);
    T v = u[(int64_t)iy * nx + ix];
    return (sx * sy < 0) ? -v : v;
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// Shape of one variant.  Each thread owns a PAIR of adjacent columns of the
// compute region (8- or 16-byte shared-memory accesses) and KY rows.
template <typename T, int R, int NWX, int NTY, int KY, int B>
struct Tb2dShape {
    static constexpr int CWX = 64 * NWX;      // compute-region width (two columns per lane)
    static constexpr int CWY = NTY * KY;      // compute-region height
    static constexpr int RX = CWX + 2 * R;    // staged width
    static constexpr int RY = CWY + 2 * R;    // staged height
    static constexpr int OFF = R & 1;         // shift so that column pairs start on an even index
    static constexpr int PX = RX + 2 * OFF;   // shared-memory row pitch (even)
    static constexpr int H = R * B;           // halo
    static constexpr int TX = RX - 2 * H;     // owned tile
    static constexpr int TY = RY - 2 * H;
    static constexpr int NT = 32 * NWX * NTY;
    static constexpr size_t SMEM = sizeof(T) * 2 * (size_t)PX * RY;
    static_assert(TX > 0 && TY > 0, "halo larger than the tile");
};

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Packed two-point arithmetic.  FP32 uses the sm_100+ paired instructions
// (one instruction for both points); FP64 does the same operations one lane
// at a time.  Explicit rounding-mode forms, so no operation is contracted
// differently between the two points of a pair.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float s_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double2 p_add(double2 a, double2 b) {
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) {
    return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c) {
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ double s_add(double a, double b) { return __dadd_rn(a, b); }

// MINB: CTAs per SM the register budget is sized for.
template <typename T, int R, int NWX, int NTY, int KY, int B, int MINB>
__global__ void __launch_bounds__(32 * NWX * NTY, MINB)
    k_step_tb2d(int nx, int ny, const T* __restrict__ Ain, const T* __restrict__ Bin, T* __restrict__ Aout,
                T* __restrict__ Bout, T* __restrict__ acc, const T* __restrict__ cw, int b, Stencil<T> st,
                int64_t fstride) {
    using S = Tb2dShape<T, R, NWX, NTY, KY, B>;
    using T2 = typename Vec2<T>::type;
    constexpr int RX = S::RX, RY = S::RY, PX = S::PX, OFF = S::OFF, H = S::H, TX = S::TX, TY = S::TY,
                  NT = S::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sP = reinterpret_cast<T*>(smem_raw);  // W^{n-1} at staging, then the level being written
    T* sC = sP + PX * RY;                    // W^n

    const int64_t N = (int64_t)nx * ny;
    const int64_t v = blockIdx.z;
    Ain += v * fstride;
    Bin += v * fstride;
    Aout += v * fstride;
    Bout += v * fstride;
    acc += v * N;

    const int x0 = blockIdx.x * TX - H;  // global coordinate of staged column 0
    const int y0 = blockIdx.y * TY - H;
    const int tid = threadIdx.x;

    // ---- stage W^{n-1}, W^n: asynchronous copies inside the box, the odd
    //      extension outside it ---------------------------------------------
    const bool inside = x0 >= 0 && y0 >= 0 && x0 + RX <= nx && y0 + RY <= ny;
    for (int q = tid; q < RX * RY; q += NT) {
        const int sy = q / RX, sx = q - sy * RX;
        const int gx = x0 + sx, gy = y0 + sy;
        const int d = sy * PX + sx + OFF;
        if (inside || (gx >= 0 && gx < nx && gy >= 0 && gy < ny)) {
            const int64_t g = (int64_t)gy * nx + gx;
            if (sizeof(T) == 8) {
                cp_async8(sP + d, Ain + g);
                cp_async8(sC + d, Bin + g);
            } else {
                cp_async4(sP + d, Ain + g);
                cp_async4(sC + d, Bin + g);
            }
        } else {
            sP[d] = load_ext(Ain, gx, gy, nx, ny);
            sC[d] = load_ext(Bin, gx, gy, nx, ny);
        }
    }

    const int lane = tid & 31;
    const int wx = (tid >> 5) % NWX;
    const int ty = (tid >> 5) / NWX;
    const int sx = R + 2 * (32 * wx + lane);  // first of the thread's two staged columns
    const int cx = sx + OFF;                  // its shared-memory column (even)
    const int sy0 = R + ty * KY;              // first staged row of its segment
    const int gx = x0 + sx;
    const int gy0 = y0 + sy0;
    const bool own_a = sx >= H && sx < H + TX && gx < nx;
    const bool own_b = sx + 1 >= H && sx + 1 < H + TX && gx + 1 < nx;
    const int klo = max(0, H - sy0);
    const int khi = min(min(KY, H + TY - sy0), ny - gy0);

    T2 accp[KY];  // filter sums of the thread's two columns
    {
        int64_t base = (int64_t)gy0 * nx + gx;
        asm volatile("" : "+l"(base));  // keep row addresses out of registers across the time loop
#pragma unroll
        for (int k = 0; k < KY; ++k) {
            const bool oy = k >= klo && k < khi;
            accp[k].x = (own_a && oy) ? acc[base + (int64_t)k * nx] : T(0);
            accp[k].y = (own_b && oy) ? acc[base + (int64_t)k * nx + 1] : T(0);
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // W^{n-1} of the thread's own points lives in registers from here on
    T2 pp[KY];
#pragma unroll
    for (int k = 0; k < KY; ++k) pp[k] = *reinterpret_cast<const T2*>(sP + (sy0 + k) * PX + cx);

    const T2 C0{st.c0, st.c0}, C1X{st.c1[0], st.c1[0]}, C1Y{st.c1[1], st.c1[1]};
    const T2 C2X{st.c2[0], st.c2[0]}, C2Y{st.c2[1], st.c2[1]};
    const T2 TWO{T(2), T(2)}, MONE{T(-1), T(-1)};
    T* cur = sC;
    T* nxt = sP;  // its old content (W^{n-1}) is only ever read by the owning thread
    for (int s = 0; s < b; ++s) {
        const T* col = cur + cx;
        // the order-2 stencil never reads rows sy0-2 and sy0+KY+1 (outside its staged region)
        T2 w0 = R == 2 ? *reinterpret_cast<const T2*>(col + (sy0 - 2) * PX) : T2{T(0), T(0)};
        T2 w1 = *reinterpret_cast<const T2*>(col + (sy0 - 1) * PX);
        T2 w2 = *reinterpret_cast<const T2*>(col + sy0 * PX);
        T2 w3 = *reinterpret_cast<const T2*>(col + (sy0 + 1) * PX);
        const T cs = cw[s];
        const T2 CS{cs, cs};
#pragma unroll
        for (int k = 0; k < KY; ++k) {
            const int row = (sy0 + k) * PX + cx;
            const T2 w4 = (R == 2 || k + 1 < KY) ? *reinterpret_cast<const T2*>(col + (sy0 + k + 2) * PX)
                                                 : T2{T(0), T(0)};
            const T2 L = *reinterpret_cast<const T2*>(cur + row - 2);  // columns x-2, x-1
            const T2 Q = *reinterpret_cast<const T2*>(cur + row + 2);  // columns x+2, x+3
            // point a at column x, point b at column x+1; every sum is (left + right)
            T2 sx1;
            sx1.x = s_add(L.y, w2.y);
            sx1.y = s_add(w2.x, Q.x);
            T2 lap = p_mul(C0, w2);
            lap = p_fma(C1X, sx1, lap);
            lap = p_fma(C1Y, p_add(w1, w3), lap);
            if (R == 2) {
                lap = p_fma(C2X, p_add(L, Q), lap);
                lap = p_fma(C2Y, p_add(w0, w4), lap);
            }
            const T2 nv = p_fma(TWO, w2, p_fma(MONE, pp[k], lap));  // 2 W^n + (dt^2 L W^n - W^{n-1})
            *reinterpret_cast<T2*>(nxt + row) = nv;
            pp[k] = w2;
            accp[k] = p_fma(CS, nv, accp[k]);  // only owned entries are stored
            w0 = w1;
            w1 = w2;
            w2 = w3;
            w3 = w4;
        }
        __syncthreads();
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    // cur = W^{n+b} (shared), pp = W^{n+b-1} (registers)
    int64_t base = (int64_t)gy0 * nx + gx;
    asm volatile("" : "+l"(base));
#pragma unroll
    for (int k = 0; k < KY; ++k) {
        if (k >= klo && k < khi) {
            const T2 c2 = *reinterpret_cast<const T2*>(cur + (sy0 + k) * PX + cx);
            const int64_t g = base + (int64_t)k * nx;
            if (own_a) {
                Bout[g] = c2.x;
                Aout[g] = pp[k].x;
                acc[g] = accp[k].x;
            }
            if (own_b) {
                Bout[g + 1] = c2.y;
                Aout[g + 1] = pp[k].y;
                acc[g + 1] = accp[k].y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// variant table
// ---------------------------------------------------------------------------
struct Tb2dVariant {
    int nwx, nty, ky, B;
    int TX, TY, threads;
    size_t smem;
    void* fn;  // kernel pointer
    int minb, fence;
};

#define EW_TB2D_VARIANT(T, R, NWX, NTY, KY, B, MINB)                                                  \
    Tb2dVariant {                                                                                     \
        NWX, NTY, KY, B, Tb2dShape<T, R, NWX, NTY, KY, B>::TX, Tb2dShape<T, R, NWX, NTY, KY, B>::TY,  \
            Tb2dShape<T, R, NWX, NTY, KY, B>::NT, Tb2dShape<T, R, NWX, NTY, KY, B>::SMEM,              \
            (void*)k_step_tb2d<T, R, NWX, NTY, KY, B, MINB>, MINB, 0                                   \
    }

template <typename T, int R>
static const std::vector<Tb2dVariant>& tb2d_variants();

// Index 0 of each list is the default used when the caller fixes the depth.
template <>
const std::vector<Tb2dVariant>& tb2d_variants<float, 2>() {
    static const std::vector<Tb2dVariant> v = {
        EW_TB2D_VARIANT(float, 2, 2, 8, 8, 4, 2),  EW_TB2D_VARIANT(float, 2, 2, 8, 8, 2, 2),
        EW_TB2D_VARIANT(float, 2, 2, 8, 8, 3, 2),  EW_TB2D_VARIANT(float, 2, 2, 16, 8, 4, 1),
        EW_TB2D_VARIANT(float, 2, 2, 16, 8, 6, 1), EW_TB2D_VARIANT(float, 2, 2, 4, 16, 4, 2),
        EW_TB2D_VARIANT(float, 2, 4, 4, 8, 4, 2),  EW_TB2D_VARIANT(float, 2, 2, 8, 12, 4, 1),
        EW_TB2D_VARIANT(float, 2, 2, 16, 8, 8, 1), EW_TB2D_VARIANT(float, 2, 1, 16, 8, 4, 2),
    };
    return v;
}
template <>
const std::vector<Tb2dVariant>& tb2d_variants<float, 1>() {
    static const std::vector<Tb2dVariant> v = {
        EW_TB2D_VARIANT(float, 1, 2, 8, 8, 4, 2),  EW_TB2D_VARIANT(float, 1, 2, 8, 8, 8, 2),
        EW_TB2D_VARIANT(float, 1, 2, 8, 8, 2, 2),  EW_TB2D_VARIANT(float, 1, 2, 16, 8, 8, 1),
        EW_TB2D_VARIANT(float, 1, 2, 16, 8, 12, 1), EW_TB2D_VARIANT(float, 1, 2, 4, 16, 8, 2),
        EW_TB2D_VARIANT(float, 1, 4, 4, 8, 8, 2),
    };
    return v;
}
template <>
const std::vector<Tb2dVariant>& tb2d_variants<double, 2>() {
    static const std::vector<Tb2dVariant> v = {
        EW_TB2D_VARIANT(double, 2, 2, 8, 8, 4, 1), EW_TB2D_VARIANT(double, 2, 2, 8, 8, 2, 1),
        EW_TB2D_VARIANT(double, 2, 2, 4, 8, 4, 2), EW_TB2D_VARIANT(double, 2, 1, 16, 8, 4, 1),
        // FP64 is ALU-bound on this part: shallow depths recompute fewer halo points
        EW_TB2D_VARIANT(double, 2, 2, 8, 8, 1, 1), EW_TB2D_VARIANT(double, 2, 2, 4, 8, 1, 2),
        EW_TB2D_VARIANT(double, 2, 2, 4, 8, 2, 2),
    };
    return v;
}
template <>
const std::vector<Tb2dVariant>& tb2d_variants<double, 1>() {
    static const std::vector<Tb2dVariant> v = {
        EW_TB2D_VARIANT(double, 1, 2, 8, 8, 4, 1), EW_TB2D_VARIANT(double, 1, 2, 8, 8, 2, 1),
        EW_TB2D_VARIANT(double, 1, 2, 4, 8, 4, 2), EW_TB2D_VARIANT(double, 1, 2, 8, 8, 8, 1),
        EW_TB2D_VARIANT(double, 1, 2, 8, 8, 1, 1), EW_TB2D_VARIANT(double, 1, 2, 4, 8, 1, 2),
    };
    return v;
}

template <typename T>
static const std::vector<Tb2dVariant>& variants_for(int order) {
    return order == 2 ? tb2d_variants<T, 1>() : tb2d_variants<T, 2>();
}

static std::mutex g_attr_mu;

template <typename T>
static ew_status launch_variant(const Tb2dVariant& var, const GridGeom& g, const T* Ain, const T* Bin, T* Aout,
                                T* Bout, T* acc, const T* cw, int b, const Stencil<T>& s, int nvec,
                                int64_t fstride, cudaStream_t st) {
    {
        // raise the dynamic shared-memory limit once per kernel and device
        static std::map<std::pair<void*, int>, bool> done;
        int dev = 0;
        EW_CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(g_attr_mu);
        auto key = std::make_pair(var.fn, dev);
        if (!done.count(key)) {
            EW_CUDA_TRY(cudaFuncSetAttribute(var.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)var.smem));
            done[key] = true;
        }
    }
    int nx = (int)g.n[0], ny = (int)g.n[1];
    dim3 grid((unsigned)((nx + var.TX - 1) / var.TX), (unsigned)((ny + var.TY - 1) / var.TY), (unsigned)nvec);
    void* args[] = {(void*)&nx, (void*)&ny, (void*)&Ain, (void*)&Bin, (void*)&Aout, (void*)&Bout,
                    (void*)&acc, (void*)&cw, (void*)&b, (void*)&s, (void*)&fstride};
    cudaEvent_t ev = fused_begin(st);
    EW_CUDA_TRY(cudaLaunchKernel(var.fn, grid, dim3(var.threads), args, var.smem, st));
    fused_end(ev, st, g.N * nvec, g.N * nvec * b);
    return EW_OK;
}

// ---------------------------------------------------------------------------
// autotuner: times every variant on the caller's buffers (before the real
// wave-solve overwrites them) and caches the fastest per grid shape.
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int64_t, int64_t, int, int, int, int>;  // nx, ny, order, elem, nvec, device
static std::map<TuneKey, int> g_tune_cache;
static std::mutex g_tune_mu;

template <typename T>
static ew_status autotune(const GridGeom& g, T* const* F, T* acc, const T* cw, const Stencil<T>& s, int nvec,
                          int64_t fstride, cudaStream_t st, int* out, bool lookup_only) {
    int dev = 0;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    TuneKey key{g.n[0], g.n[1], g.order, (int)sizeof(T), nvec, dev};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            return EW_OK;
        }
        if (lookup_only) {
            *out = 0;
            return EW_OK;
        }
    }
    const auto& vars = variants_for<T>(g.order);
    bool prof = g_profile_on;
    g_profile_on = false;  // tuning launches are not counted
    cudaEvent_t e0, e1;
    EW_CUDA_TRY(cudaEventCreate(&e0));
    EW_CUDA_TRY(cudaEventCreate(&e1));
    int best = 0;
    double best_rate = -1.0;
    ew_status status = EW_OK;
    for (size_t i = 0; i < vars.size() && status == EW_OK; ++i) {
        const auto& var = vars[i];
        int b = var.B;
        // one warm launch, then three timed ones
        for (int rep = 0; rep < 4 && status == EW_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            status = launch_variant<T>(var, g, F[0], F[1], F[2], F[3], acc, cw, b, s, nvec, fstride, st);
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        double rate = (double)b * 3.0 / std::max(ms, 1e-6f);  // time steps per ms
        if (getenv("EW_TUNE_LOG"))
            fprintf(stderr, "[ew tune] %lldx%lld order %d %s: variant %zu (warps %dx%d, rows %d, depth %d, "
                            "minb %d, fence %d, tile %dx%d): %.4f ms/step\n",
                    (long long)g.n[0], (long long)g.n[1], g.order, sizeof(T) == 4 ? "fp32" : "fp64", i, var.nwx,
                    var.nty, var.ky, var.B, var.minb, var.fence, var.TX, var.TY, 1.0 / rate);
        if (rate > best_rate) {
            best_rate = rate;
            best = (int)i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_profile_on = prof;
    EW_TRY(status);
    EW_CUDA_TRY(cudaGetLastError());
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    *out = best;
    return EW_OK;
}

template <typename T>
ew_status tb2d_tune(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, T* acc, int nvec,
                    int64_t fstride, cudaStream_t st) {
    Stencil<T> s = make_stencil<T>(g, plan.dt * plan.dt);
    int vi = 0;
    return autotune<T>(g, F, acc, cdev, s, nvec, fstride, st, &vi, false);
}
template ew_status tb2d_tune<float>(const GridGeom&, const FilterPlan&, const float*, float* const*, float*, int,
                                    int64_t, cudaStream_t);
template ew_status tb2d_tune<double>(const GridGeom&, const FilterPlan&, const double*, double* const*, double*,
                                     int, int64_t, cudaStream_t);

// Advance the explicit scheme from level L (F[cur]) with F[prv] = level L-1
// to level Nt, accumulating into acc.  `variant` < 0: autotune.  `tb` > 0
// caps the steps per launch.
template <typename T>
ew_status tb2d_advance(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, int* prv, int* cur,
                       int64_t L, T* acc, int nvec, int64_t fstride, int tb, cudaStream_t st) {
    Stencil<T> s = make_stencil<T>(g, plan.dt * plan.dt);
    int vi = 0;
    if (tb == 0) EW_TRY(autotune<T>(g, F, acc, cdev, s, nvec, fstride, st, &vi, true));
    const auto& vars = variants_for<T>(g.order);
    const Tb2dVariant& var = vars[(size_t)vi];
    int bmax = var.B;
    if (tb > 0) bmax = std::min(bmax, tb);  // tb > 0 runs the default variant (index 0)
    int p = *prv, c = *cur;
    int a = -1, d = -1;  // the two spare buffers
    for (int q = 0; q < 4; ++q)
        if (q != p && q != c) (a < 0 ? a : d) = q;
    while (L < plan.Nt) {
        int b = (int)std::min<int64_t>(bmax, plan.Nt - L);
        EW_TRY(launch_variant<T>(var, g, F[p], F[c], F[a], F[d], acc, cdev + L + 1, b, s, nvec, fstride, st));
        L += b;
        int op = p, oc = c;
        p = a;
        c = d;
        a = op;
        d = oc;
    }
    *prv = p;
    *cur = c;
    return EW_OK;
}
template ew_status tb2d_advance<float>(const GridGeom&, const FilterPlan&, const float*, float* const*, int*, int*,
                                       int64_t, float*, int, int64_t, int, cudaStream_t);
template ew_status tb2d_advance<double>(const GridGeom&, const FilterPlan&, const double*, double* const*, int*,
                                        int*, int64_t, double*, int, int64_t, int, cudaStream_t);

// description of the tuned choice (for reports)
template <typename T>
int tb2d_choice(const GridGeom& g, int nvec, int* B, int* TX, int* TY) {
    int dev = 0;
    cudaGetDevice(&dev);
    TuneKey key{g.n[0], g.n[1], g.order, (int)sizeof(T), nvec, dev};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it == g_tune_cache.end()) return -1;
    const auto& var = variants_for<T>(g.order)[(size_t)it->second];
    *B = var.B;
    *TX = var.TX;
    *TY = var.TY;
    return it->second;
}
template int tb2d_choice<float>(const GridGeom&, int, int*, int*, int*);
template int tb2d_choice<double>(const GridGeom&, int, int*, int*, int*);

}  // namespace ew
