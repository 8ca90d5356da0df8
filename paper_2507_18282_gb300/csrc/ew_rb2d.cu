// ew_rb2d.cu -- register-blocked, persistent form of the temporally blocked
// 2D fused step (eqs. explicitScheme, filterQuadrature), FP32.
//
// The shared-memory form (ew_tb2d_dev.cuh) keeps W^n in shared memory and
// re-reads every point's column window and its x-neighbours from there each
// step; it is bound by shared-memory wavefronts and it stages, computes and
// stores one tile after the other.  Here:
//
//  * W^n, D^n = W^n - W^{n-1} (the summed form of the recurrence, see
//    ew_stencil.cu) and the filter sum of a thread's KY x 4 points stay in
//    registers for the whole tile.  A warp covers one row band of 128
//    columns (4 per lane), so the x-neighbours come from the adjacent lanes
//    by warp shuffles and the y-neighbours from the thread's own registers;
//    only the R top and R bottom rows of each band cross warps, through a
//    small double-buffered shared-memory exchange (one barrier per step).
//  * The CTA is persistent (one per SM) and walks a static list of tiles.
//    While it advances tile t, the bulk-copy engine (cp.async.bulk with an
//    mbarrier) fills the staging buffer with D^n, W^n of tile t+1, so the
//    HBM reads overlap the arithmetic.
//
// The compute region is the whole staged 128 x (NTY KY) region: lanes at the
// left/right edge and warps at the top/bottom edge see wrong neighbours, and
// the wrong values spread R points per step, so after b <= B steps the tile
// minus a rim of H = R B points is exact; that TX x TY interior is the owned
// tile.  Points outside the box are staged with the box closure's extension of
// the grid function (ew_bc_dev.cuh), which the linear update keeps exact, as in
// the shared-memory form.  Every point performs the
// same operations in the same order as in the shared-memory form, so both
// forms give bit-identical results.
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>

#include "ew_internal.h"
#include "ew_tb2d_dev.cuh"

namespace ew {

__device__ int g_rb2d_timeout = 0;  // set when a staging wait gave up

template <int R, int NTY, int KY, int B>
struct Rb2dShape {
    static constexpr int CW = 128;        // compute-region width: 32 lanes x 4 columns
    static constexpr int CH = NTY * KY;   // compute-region height
    static constexpr int NT = 32 * NTY;   // threads
    static constexpr int PITCH = 136;     // staged row pitch in floats (a 16-byte multiple, >= 128 + 6)
    static constexpr int H = R * B;       // rim that is wrong after B steps
    static constexpr int TX = CW - 2 * H; // owned tile
    static constexpr int TY = CH - 2 * H;
    static constexpr size_t STAGE_BYTES = sizeof(float) * 2 * (size_t)CH * PITCH;
    static constexpr size_t XBUF_BYTES = 2 * (size_t)NTY * 2 * R * 32 * sizeof(float4);
    static constexpr size_t SMEM = STAGE_BYTES + XBUF_BYTES + 16;  // + the mbarrier
    static_assert(TX > 0 && TY > 0, "rim larger than the tile");
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: gives up after about two seconds of SM clock
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64();
    for (int it = 0; it < (1 << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > 4000000000ll) break;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

// position of staged row r: element (r, c) of a field lives at row(r)[c + o(r)],
// o(r) = (global index of staged column 0 of that row) mod 4, so that every
// 16-byte block of the global row lands on a 16-byte block of shared memory
__device__ __forceinline__ int stage_off(int gy, int nx, int x0) {
    return (int)(((int64_t)gy * nx + x0) & 3);
}

// tile number -> (vector, origin of the staged region)
__device__ __forceinline__ void rb_tile(int t, int tiles_x, int tiles_per_vec, int TX, int TY, int H, int& v, int& x0,
                                        int& y0) {
    v = t / tiles_per_vec;
    const int r = t - v * tiles_per_vec;
    const int ty = r / tiles_x;
    x0 = (r - ty * tiles_x) * TX - H;
    y0 = ty * TY - H;
}

struct RbCoef {
    float2 c0, c1x, c1y, c2x, c2y;
};

// One time step of a thread's KY x 4 points in the summed form: W (W^n) and
// D (D^n = W^n - W^{n-1}) become W^{n+1} and D^{n+1}; ac accumulates
// cs W^{n+1}.  up / dn hold the R rows of W^n above / below the band (rows
// -R..-1 and KY..KY+R-1).  Every D row is updated first, from W^n alone,
// then W and the sums pointwise, so W^n is intact while it is read.  The
// per-point operations and their order are those of tb2d_tile: for the column
// pair (x, x+1) with L = (x-2, x-1) and Q = (x+2, x+3),
//   lap = c0 w + c1x (left + right) + c1y (up + down) [+ c2x (L + Q) + c2y (up2 + down2)]
//   D += lap,  W += D,  acc += cs W.
template <int R, int KY>
__device__ __forceinline__ void rb_rows(float4 (&W)[KY], float4 (&D)[KY], float4 (&ac)[KY], const float4 (&up)[2],
                                        const float4 (&dn)[2], float cs, const RbCoef& k) {
    const float2 CS{cs, cs};
#pragma unroll
    for (int r = 0; r < KY; ++r) {
        const float4 c = W[r];
        const float4 m1 = r >= 1 ? W[r - 1] : up[1];
        const float4 p1 = r + 1 < KY ? W[r + 1] : dn[0];
        // x-neighbours from the adjacent lanes (lane 0 / 31 get their own
        // values: wrong, but finite, and inside the rim)
        const float Lw = __shfl_up_sync(0xffffffffu, c.w, 1);
        const float Ra = __shfl_down_sync(0xffffffffu, c.x, 1);
        float Lz = 0.f, Rb = 0.f;
        if (R == 2) {
            Lz = __shfl_up_sync(0xffffffffu, c.z, 1);
            Rb = __shfl_down_sync(0xffffffffu, c.y, 1);
        }
        // pair (a, b) = columns x, x+1
        float2 w2{c.x, c.y};
        float2 sx1{s_add(Lw, c.y), s_add(c.x, c.z)};
        float2 lap = p_mul(k.c0, w2);
        lap = p_fma(k.c1x, sx1, lap);
        lap = p_fma(k.c1y, p_add(float2{m1.x, m1.y}, float2{p1.x, p1.y}), lap);
        if (R == 2) {
            const float4 m2 = r >= 2 ? W[r - 2] : up[r];
            const float4 p2 = r + 2 < KY ? W[r + 2] : dn[r + 2 - KY];
            lap = p_fma(k.c2x, p_add(float2{Lz, Lw}, float2{c.z, c.w}), lap);
            lap = p_fma(k.c2y, p_add(float2{m2.x, m2.y}, float2{p2.x, p2.y}), lap);
        }
        const float2 da = p_add(float2{D[r].x, D[r].y}, lap);
        // pair (c, d) = columns x+2, x+3: L = (a, b), Q = (Ra, Rb)
        w2 = float2{c.z, c.w};
        sx1 = float2{s_add(c.y, c.w), s_add(c.z, Ra)};
        lap = p_mul(k.c0, w2);
        lap = p_fma(k.c1x, sx1, lap);
        lap = p_fma(k.c1y, p_add(float2{m1.z, m1.w}, float2{p1.z, p1.w}), lap);
        if (R == 2) {
            const float4 m2 = r >= 2 ? W[r - 2] : up[r];
            const float4 p2 = r + 2 < KY ? W[r + 2] : dn[r + 2 - KY];
            lap = p_fma(k.c2x, p_add(float2{c.x, c.y}, float2{Ra, Rb}), lap);
            lap = p_fma(k.c2y, p_add(float2{m2.z, m2.w}, float2{p2.z, p2.w}), lap);
        }
        const float2 db = p_add(float2{D[r].z, D[r].w}, lap);
        D[r] = make_float4(da.x, da.y, db.x, db.y);
    }
#pragma unroll
    for (int r = 0; r < KY; ++r) {
        const float2 na = p_add(float2{W[r].x, W[r].y}, float2{D[r].x, D[r].y});
        const float2 nb = p_add(float2{W[r].z, W[r].w}, float2{D[r].z, D[r].w});
        const float2 aa = p_fma(CS, na, float2{ac[r].x, ac[r].y});
        const float2 ab = p_fma(CS, nb, float2{ac[r].z, ac[r].w});
        W[r] = make_float4(na.x, na.y, nb.x, nb.y);
        ac[r] = make_float4(aa.x, aa.y, ab.x, ab.y);
    }
}

__device__ __forceinline__ float f4get(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ void f4set(float4& v, int i, float x) {
    if (i == 0) v.x = x;
    else if (i == 1) v.y = x;
    else if (i == 2) v.z = x;
    else v.w = x;
}

// Stage D^n (field 0) and W^n (field 1) of tile (v, x0, y0): one bulk copy
// per in-box row and field, 16-byte aligned at both ends (the copy may take a
// few columns beyond the tile, never beyond the field); the tail of the very
// last row of the field, which the rounding would overrun, is copied by plain
// loads.  Each issuing thread adds its bytes to the mbarrier's expected count
// before its copy; the caller arrives once after a CTA barrier.
template <int CH, int CW, int PITCH, int NT>
__device__ __forceinline__ void rb_issue(const float* __restrict__ Ain, const float* __restrict__ Bin, int nx, int ny,
                                         int64_t N, int v, int64_t fstride, int x0, int y0, float* stage, uint64_t* bar,
                                         int tid) {
    const int xa = max(x0, 0), xb = min(x0 + CW, nx);
    if (xa >= xb) return;
    fence_proxy_async();  // earlier generic accesses to the staging buffer come first
    for (int q = tid; q < 2 * CH; q += NT) {
        const int f = q >= CH ? 1 : 0;
        const int r = q - f * CH;
        const int gy = y0 + r;
        if (gy < 0 || gy >= ny) continue;
        const float* base = (f ? Bin : Ain) + (int64_t)v * fstride;
        const int64_t rowg = (int64_t)gy * nx;
        const int64_t e0 = rowg + xa, e1 = rowg + xb;
        const int64_t col0 = rowg + x0 - stage_off(gy, nx, x0);  // global index held at row[0] (a multiple of 4)
        const int64_t f0 = e0 & ~(int64_t)3;
        int64_t f1 = (e1 + 3) & ~(int64_t)3;
        if (f1 > N) f1 = N & ~(int64_t)3;
        float* row = stage + ((size_t)f * CH + r) * PITCH;
        if (f1 > f0) {
            const unsigned bytes = (unsigned)(f1 - f0) * 4u;
            mbar_expect_tx(bar, bytes);
            bulk_g2s(row + (f0 - col0), base + f0, bytes, bar);
        }
        for (int64_t e = max(f1, e0); e < e1; ++e) row[e - col0] = base[e];
    }
}

// Points of the staged region outside the box: the box closure's extension
// (ew_bc_dev.cuh), read from the staged mirror point (0 when the mirror is not
// staged: such a point is farther than H from the owned tile and cannot reach
// it within B steps).
template <int CH, int CW, int PITCH, int NT, bool GEN>
__device__ __forceinline__ void rb_fixup(int nx, int ny, int bc, int x0, int y0, float* stage, int tid) {
    if (x0 >= 0 && y0 >= 0 && x0 + CW <= nx && y0 + CH <= ny) return;
    for (int q = tid; q < 2 * CH * CW; q += NT) {
        const int f = q / (CH * CW);
        const int e = q - f * CH * CW;
        const int r = e / CW, c = e - r * CW;
        const int gx = x0 + c, gy = y0 + r;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
        int sx = 1, sy = 1;
        const int ix = ext2<GEN>(gx, nx, axis_bc(bc, 0), sx), iy = ext2<GEN>(gy, ny, axis_bc(bc, 1), sy);
        float val = 0.f;
        if (ix >= 0 && iy >= 0) {
            const int mc = ix - x0, mr = iy - y0;
            if (mc >= 0 && mc < CW && mr >= 0 && mr < CH) {
                val = stage[((size_t)f * CH + mr) * PITCH + mc + stage_off(iy, nx, x0)];
                if (sx * sy < 0) val = -val;
            }
        }
        stage[((size_t)f * CH + r) * PITCH + c + stage_off(gy, nx, x0)] = val;
    }
}

// the exchange and the rows of one step (Wn, Dn: W^n, D^n -> W^{n+1}, D^{n+1})
template <int R, int NTY, int KY>
__device__ __forceinline__ void rb_step(float4 (&Wn)[KY], float4 (&Dn)[KY], float4 (&ac)[KY], float4 (&up)[2],
                                        float4 (&dn)[2], float4* xbuf, int s, int wy, int lane, float cs,
                                        const RbCoef& k) {
    float4* xb = xbuf + (size_t)(s & 1) * NTY * 2 * R * 32;
    const int wu = wy > 0 ? wy - 1 : 0, wd = wy + 1 < NTY ? wy + 1 : NTY - 1;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        xb[(wy * 2 * R + j) * 32 + lane] = Wn[j];               // top rows of the band
        xb[(wy * 2 * R + R + j) * 32 + lane] = Wn[KY - R + j];  // bottom rows
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < R; ++j) {
        up[2 - R + j] = xb[(wu * 2 * R + R + j) * 32 + lane];  // rows -R..-1: bottom rows of the band above
        dn[j] = xb[(wd * 2 * R + j) * 32 + lane];              // rows KY..KY+R-1: top rows of the band below
    }
    rb_rows<R, KY>(Wn, Dn, ac, up, dn, cs, k);
}

// MINB is 1: the register file holds one CTA of 32 NTY threads per SM.
// GEN: any faces (false: Dirichlet faces only, see ext2 in ew_tb2d_dev.cuh).
template <int R, int NTY, int KY, int B, bool GEN>
__global__ void __launch_bounds__(32 * NTY, 1)
    k_step_rb2d(int nx, int ny, const float* __restrict__ Ain, const float* __restrict__ Bin, float* __restrict__ Aout,
                float* __restrict__ Bout, float* __restrict__ acc, const float* __restrict__ cw, int b, Stencil<float> st,
                int64_t fstride, int tiles_x, int tiles_per_vec, int ntiles, unsigned stall_tx) {
    using S = Rb2dShape<R, NTY, KY, B>;
    constexpr int CW = S::CW, CH = S::CH, NT = S::NT, PITCH = S::PITCH, H = S::H, TX = S::TX, TY = S::TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);  // [2][CH][PITCH]: D^n, W^n of the next tile
    float4* xbuf = reinterpret_cast<float4*>(smem_raw + S::STAGE_BYTES);  // [2][NTY][2R][32]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + S::STAGE_BYTES + S::XBUF_BYTES);
    const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
    const int64_t N = (int64_t)nx * ny;
    int t = blockIdx.x;
    if (t >= ntiles) return;
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    {
        int v, x0, y0;
        rb_tile(t, tiles_x, tiles_per_vec, TX, TY, H, v, x0, y0);
        rb_issue<CH, CW, PITCH, NT>(Ain, Bin, nx, ny, N, v, fstride, x0, y0, stage, bar, tid);
    }
    // stall_tx > 0 (a test of the bounded wait): expect bytes that never arrive, so
    // the first wait runs out and the CTA reports it and returns
    if (tid == 0 && stall_tx) mbar_expect_tx(bar, stall_tx);
    __syncthreads();
    if (tid == 0) mbar_arrive(bar);

    RbCoef K;
    K.c0 = float2{st.c0, st.c0};
    K.c1x = float2{st.c1[0], st.c1[0]};
    K.c1y = float2{st.c1[1], st.c1[1]};
    K.c2x = float2{st.c2[0], st.c2[0]};
    K.c2y = float2{st.c2[1], st.c2[1]};
    float4 A[KY], P[KY], AC[KY];  // W^n, D^n, filter sums
    float4 up[2] = {float4{0.f, 0.f, 0.f, 0.f}, float4{0.f, 0.f, 0.f, 0.f}};
    float4 dn[2] = {float4{0.f, 0.f, 0.f, 0.f}, float4{0.f, 0.f, 0.f, 0.f}};
    unsigned phase = 0;
    for (; t < ntiles; t += gridDim.x) {
        int v, x0, y0;
        rb_tile(t, tiles_x, tiles_per_vec, TX, TY, H, v, x0, y0);
        // ---- staged D^n, W^n of this tile -> registers -----------------------
        const bool ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&g_rb2d_timeout, 1);
            return;
        }
        rb_fixup<CH, CW, PITCH, NT, GEN>(nx, ny, st.bc, x0, y0, stage, tid);
        __syncthreads();
        const int64_t vo = (int64_t)v * fstride, va = (int64_t)v * N;
#pragma unroll
        for (int k = 0; k < KY; ++k) {
            const int r = wy * KY + k;
            const int o = stage_off(y0 + r, nx, x0);
            const float* s0 = stage + (size_t)r * PITCH + 4 * lane + o;
            const float* s1 = s0 + (size_t)CH * PITCH;
            if (o == 0) {
                P[k] = *reinterpret_cast<const float4*>(s0);
                A[k] = *reinterpret_cast<const float4*>(s1);
            } else {
                P[k] = make_float4(s0[0], s0[1], s0[2], s0[3]);
                A[k] = make_float4(s1[0], s1[1], s1[2], s1[3]);
            }
            const int gy = y0 + r;
            const bool orow = r >= H && r < H + TY && gy < ny;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = 4 * lane + i, gx = x0 + c;
                const bool own = orow && c >= H && c < H + TX && gx < nx;
                f4set(AC[k], i, own ? acc[va + (int64_t)gy * nx + gx] : 0.f);
            }
        }
        __syncthreads();  // the staging buffer is free
        const int tn = t + gridDim.x;
        if (tn < ntiles) {
            int vn, xn, yn;
            rb_tile(tn, tiles_x, tiles_per_vec, TX, TY, H, vn, xn, yn);
            rb_issue<CH, CW, PITCH, NT>(Ain, Bin, nx, ny, N, vn, fstride, xn, yn, stage, bar, tid);
            // the next tile's filter sums: warm L2 (one prefetch per 128-byte line of each owned row)
            constexpr int LPR = (TX + 31) / 32 + 1;
            for (int q = tid; q < TY * LPR; q += NT) {
                const int r = q / LPR, l = q - r * LPR;
                const int gy = yn + H + r, gx = min(xn + H + 32 * l, xn + H + TX - 1);
                if (gy < ny && gx < nx) prefetch_l2(acc + (int64_t)vn * N + (int64_t)gy * nx + gx);
            }
        }
        __syncthreads();
        if (tid == 0 && tn < ntiles) mbar_arrive(bar);
        // ---- b time steps in registers ---------------------------------------
        for (int s = 0; s < b; ++s) rb_step<R, NTY, KY>(A, P, AC, up, dn, xbuf, s, wy, lane, cw[s], K);
        // ---- owned points out: D^{n+b} -> Aout, W^{n+b} -> Bout, sums -> acc
#pragma unroll
        for (int k = 0; k < KY; ++k) {
            const int r = wy * KY + k, gy = y0 + r;
            if (r < H || r >= H + TY || gy >= ny) continue;
            const float4 cur = A[k], prv = P[k];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = 4 * lane + i, gx = x0 + c;
                if (c < H || c >= H + TX || gx >= nx) continue;
                const int64_t gi = (int64_t)gy * nx + gx;
                Bout[vo + gi] = f4get(cur, i);
                Aout[vo + gi] = f4get(prv, i);
                acc[va + gi] = f4get(AC[k], i);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#define EW_RB2D(R, NTY, KY, B)                                                                              \
    Rb2dDesc {                                                                                              \
        (void*)k_step_rb2d<R, NTY, KY, B, false>, (void*)k_step_rb2d<R, NTY, KY, B, true>, NTY, KY, B,       \
            Rb2dShape<R, NTY, KY, B>::TX,                                                                   \
            Rb2dShape<R, NTY, KY, B>::TY, Rb2dShape<R, NTY, KY, B>::NT, Rb2dShape<R, NTY, KY, B>::SMEM        \
    }

const std::vector<Rb2dDesc>& rb2d_variants(int R) {
    static const std::vector<Rb2dDesc> r1 = {EW_RB2D(1, 16, 8, 8), EW_RB2D(1, 16, 8, 12), EW_RB2D(1, 16, 8, 16)};
    static const std::vector<Rb2dDesc> r2 = {EW_RB2D(2, 16, 8, 6), EW_RB2D(2, 16, 8, 7), EW_RB2D(2, 16, 8, 8)};
    return R == 1 ? r1 : r2;
}

static std::mutex g_rb_mu;

ew_status rb2d_launch(const Rb2dDesc& d, const GridGeom& g, const float* Ain, const float* Bin, float* Aout,
                      float* Bout, float* acc, const float* cw, int b, const Stencil<float>& s, int nvec,
                      int64_t fstride, cudaStream_t st) {
    // bulk copies read whole 16-byte blocks: every vector of both inputs must start on one
    if (((uintptr_t)Ain | (uintptr_t)Bin) & 15 || (fstride & 3) || g.dim != 2)
        return set_error(EW_EUNSUPPORTED, "register-blocked step needs 16-byte aligned 2D fields");
    if (b < 1 || b > d.B) return set_error(EW_EINVAL, "register-blocked step: depth out of range");
    int dev = 0, nsm = 0;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    void* fn = g.bc ? d.fn_gen : d.fn;
    {
        static std::map<std::pair<void*, int>, int> sms;
        std::lock_guard<std::mutex> lk(g_rb_mu);
        auto key = std::make_pair(fn, dev);
        auto it = sms.find(key);
        if (it == sms.end()) {
            EW_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.smem));
            EW_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            sms[key] = nsm;
        } else {
            nsm = it->second;
        }
    }
    int nx = (int)g.n[0], ny = (int)g.n[1];
    int tiles_x = (nx + d.TX - 1) / d.TX, tiles_y = (ny + d.TY - 1) / d.TY;
    int tiles_per_vec = tiles_x * tiles_y;
    int64_t nt64 = (int64_t)tiles_per_vec * nvec;
    if (nt64 > INT32_MAX) return set_error(EW_EUNSUPPORTED, "register-blocked step: too many tiles");
    int ntiles = (int)nt64;
    int grid = std::min(ntiles, nsm);
    // EW_TEST_RB2D_STALL: test hook that makes every CTA's first staging wait run out
    unsigned stall_tx = getenv("EW_TEST_RB2D_STALL") ? 16u : 0u;
    void* args[] = {(void*)&nx,   (void*)&ny, (void*)&Ain, (void*)&Bin,     (void*)&Aout,          (void*)&Bout,
                    (void*)&acc,  (void*)&cw, (void*)&b,   (void*)&s,       (void*)&fstride,       (void*)&tiles_x,
                    (void*)&tiles_per_vec, (void*)&ntiles, (void*)&stall_tx};
    cudaEvent_t ev = fused_begin(st);
    EW_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(d.threads), args, d.smem, st));
    fused_end(ev, st, g.N * nvec, g.N * nvec * b);
    return EW_OK;
}

ew_status rb2d_check_timeout() {
    int flag = 0, zero = 0;
    EW_CUDA_TRY(cudaMemcpyFromSymbol(&flag, g_rb2d_timeout, sizeof(int)));
    if (!flag) return EW_OK;
    EW_CUDA_TRY(cudaMemcpyToSymbol(g_rb2d_timeout, &zero, sizeof(int)));
    return set_error(EW_ETIMEOUT, "a staging copy of the register-blocked step did not complete");
}

}  // namespace ew
