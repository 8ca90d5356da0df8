// ew_tb2d_dev.cuh -- device side of the temporally blocked 2D fused step:
// the per-tile computation (shared by the single-grid and the batched kernels)
// and the single-grid kernel.  See ew_tb2d.cu for the design.
#pragma once

#include "ew_bc_dev.cuh"
#include "ew_dd.cuh"
#include "ew_internal.h"

namespace ew {

// odd extension of an axis of length n about -1 and n (two Dirichlet faces):
// the interior index holding the value and its sign, or -1 for a zero (wall)
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

// The 2D blocked kernels come in two instantiations: GEN = false for boxes
// with Dirichlet faces only (the odd extension above) and GEN = true for any
// faces (ew_bc_dev.cuh: ext_axis).  The general code in the staging loop of
// every tile made the Dirichlet kernels 10-20 % slower on 2047 x 3071
// (measured), so the Dirichlet instantiation keeps the plain form.
template <bool GEN>
__device__ __forceinline__ int ext2(int p, int n, int code, int& sign) {
    if constexpr (GEN) return ext_axis<int>(p, n, code, sign);
    else return odd_ext(p, n, sign);
}

// value of point (gx, gy) of the box closure's extension
template <typename T, bool GEN>
__device__ __forceinline__ T load_ext(const T* __restrict__ u, int gx, int gy, int nx, int ny, int bc) {
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) return u[(int64_t)gy * nx + gx];
    int sx = 1, sy = 1;
    int ix = ext2<GEN>(gx, nx, axis_bc(bc, 0), sx);
    int iy = ext2<GEN>(gy, ny, axis_bc(bc, 1), sy);
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
template <>
struct Vec2<dd> {
    using type = dd2;
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
// double-FP32 pairs: the same operations in the pair arithmetic of ew_dd.cuh
__device__ __forceinline__ dd2 p_add(dd2 a, dd2 b) { return dd2{dd_add(a.x, b.x), dd_add(a.y, b.y)}; }
__device__ __forceinline__ dd2 p_mul(dd2 a, dd2 b) { return dd2{dd_mul(a.x, b.x), dd_mul(a.y, b.y)}; }
__device__ __forceinline__ dd2 p_fma(dd2 a, dd2 b, dd2 c) { return dd2{dd_fma(a.x, b.x, c.x), dd_fma(a.y, b.y, c.y)}; }
__device__ __forceinline__ dd s_add(dd a, dd b) { return dd_add(a, b); }

// One tile (tile_x, tile_y) of one grid: b <= B steps.  Called by the
// single-grid kernel below and by the batched persistent kernel.
template <typename T, int R, int NWX, int NTY, int KY, int B, bool GEN>
__device__ __forceinline__ void tb2d_tile(int nx, int ny, const T* __restrict__ Ain, const T* __restrict__ Bin,
                                          T* __restrict__ Aout, T* __restrict__ Bout, T* __restrict__ acc,
                                          const T* __restrict__ cw, int b, const Stencil<T>& st, int tile_x,
                                          int tile_y) {
    using S = Tb2dShape<T, R, NWX, NTY, KY, B>;
    using T2 = typename Vec2<T>::type;
    constexpr int RX = S::RX, RY = S::RY, PX = S::PX, OFF = S::OFF, H = S::H, TX = S::TX, TY = S::TY,
                  NT = S::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sP = reinterpret_cast<T*>(smem_raw);  // D^n at staging, then the level being written
    T* sC = sP + PX * RY;                    // W^n

    const int x0 = tile_x * TX - H;  // global coordinate of staged column 0
    const int y0 = tile_y * TY - H;
    const int tid = threadIdx.x;

    // ---- stage D^n, W^n: asynchronous copies inside the box, the box
    //      closure's extension outside it -----------------------------------
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
            sP[d] = load_ext<T, GEN>(Ain, gx, gy, nx, ny, st.bc);
            sC[d] = load_ext<T, GEN>(Bin, gx, gy, nx, ny, st.bc);
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

    // D^n = W^n - W^{n-1} of the thread's own points lives in registers from here on
    T2 dd[KY];
#pragma unroll
    for (int k = 0; k < KY; ++k) dd[k] = *reinterpret_cast<const T2*>(sP + (sy0 + k) * PX + cx);

    const T2 C0{st.c0, st.c0}, C1X{st.c1[0], st.c1[0]}, C1Y{st.c1[1], st.c1[1]};
    const T2 C2X{st.c2[0], st.c2[0]}, C2Y{st.c2[1], st.c2[1]};
    T* cur = sC;
    T* nxt = sP;  // its old content (D^n) is only ever read by the owning thread
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
            const T2 d = p_add(dd[k], lap);  // D^{n+1} = D^n + dt^2 L W^n
            const T2 nv = p_add(w2, d);      // W^{n+1} = W^n + D^{n+1}
            *reinterpret_cast<T2*>(nxt + row) = nv;
            dd[k] = d;
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
    // cur = W^{n+b} (shared), dd = D^{n+b} (registers)
    int64_t base = (int64_t)gy0 * nx + gx;
    asm volatile("" : "+l"(base));
#pragma unroll
    for (int k = 0; k < KY; ++k) {
        if (k >= klo && k < khi) {
            const T2 c2 = *reinterpret_cast<const T2*>(cur + (sy0 + k) * PX + cx);
            const int64_t g = base + (int64_t)k * nx;
            if (own_a) {
                Bout[g] = c2.x;
                Aout[g] = dd[k].x;
                acc[g] = accp[k].x;
            }
            if (own_b) {
                Bout[g + 1] = c2.y;
                Aout[g + 1] = dd[k].y;
                acc[g + 1] = accp[k].y;
            }
        }
    }
}

// MINB: CTAs per SM the register budget is sized for.
template <typename T, int R, int NWX, int NTY, int KY, int B, int MINB, bool GEN>
__global__ void __launch_bounds__(32 * NWX * NTY, MINB)
    k_step_tb2d(int nx, int ny, const T* __restrict__ Ain, const T* __restrict__ Bin, T* __restrict__ Aout,
                T* __restrict__ Bout, T* __restrict__ acc, const T* __restrict__ cw, int b, Stencil<T> st,
                int64_t fstride) {
    const int64_t N = (int64_t)nx * ny;
    const int64_t v = blockIdx.z;
    tb2d_tile<T, R, NWX, NTY, KY, B, GEN>(nx, ny, Ain + v * fstride, Bin + v * fstride, Aout + v * fstride,
                                     Bout + v * fstride, acc + v * N, cw, b, st, blockIdx.x, blockIdx.y);
}

}  // namespace ew
