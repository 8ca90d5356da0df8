// ew_tma2d.cu -- persistent, warp-specialised, TMA-staged form of the
// temporally blocked 2D fused step (eqs. explicitScheme, filterQuadrature),
// FP32.
//
// The per-tile arithmetic is that of the shared-memory form (ew_tb2d_dev.cuh:
// W^n in shared memory, D^n = W^n - W^{n-1} and the filter sums of a thread's
// column pair in registers, one barrier per step), so both forms give
// bit-identical results.  What differs is how tiles are fed and drained:
//
//  * One CTA per SM walks a static list of tiles with two staging slots, each
//    holding D^n and W^n of one tile (the staged region plus a few alignment
//    columns).  A producer warp moves all field data: the tensor-memory
//    accelerator fills a slot (one cp.async.bulk.tensor.3d per field,
//    completing on the slot's "full" mbarrier), and once the compute warps
//    have finished a tile (its "done" mbarrier) the producer writes the owned
//    box of D^{n+b} and of W^{n+b} back with one tensor store each
//    (cp.async.bulk.tensor shared -> global, clipped to the box), waits until
//    they have read the slot, and refills the slot with the tile after next.
//    It also warms L2 with the filter sums of that tile.  The compute warps
//    never wait for a load of D or W, never issue their stores, and stay in
//    step with each other by a named barrier that the producer does not join.
//    (One bulk copy per owned row instead took the producer longer than the
//    compute warps' whole tile: every copy request has a fixed cost.)
//  * Measured on the element-wise staging of the shared-memory form: about a
//    quarter of each tile's time went to issuing the staging copies and a
//    fifth to the gap between consecutive CTAs on an SM; with the copies
//    issued by one of the compute threads, the wait for its stores to drain
//    stalled the whole CTA.  The producer warp takes both off the critical
//    path.
//  * After the copy, the slot's D^n buffer is read into registers and then
//    serves as the second W buffer of the step loop (W^n / W^{n+1}
//    ping-pong).  The last step writes W^{n+b} of the owned points packed
//    (the TX x TY box the tensor store reads), and after its barrier the
//    compute warps put D^{n+b} packed into the other buffer.
//  * Tensor maps and bulk copies need 16-byte aligned rows, so the time-level
//    fields of this form use a padded row pitch (nx rounded up to 4 points,
//    pitch2d()); the filter sum stays in the caller's dense layout and is read
//    and written by the compute warps with plain loads and stores.  The map's
//    x extent is nx, so the pad columns, like every other point outside the
//    box, arrive as zeros; boundary tiles then overwrite their points outside
//    the box with the box closure's extension read from the staged mirror
//    point (ew_bc_dev.cuh).
//  * A load's x coordinate must be a multiple of 4 points: the slot holds the
//    staged region from x0 rounded down to one, and the column offset o =
//    x0 mod 4 is applied when indexing.  Column pairs stay 8-byte aligned
//    because x0 + R is even for every tile (TX even, H - R even); a store's x
//    coordinate (tile_x TX) is a multiple of 4 because TX is.
//  * Every wait is bounded (about two seconds of SM clock).  Compute warps that
//    give up agree through the named barrier and leave together; the producer
//    gives up on its own wait.  Either records the failure in a device flag
//    (EW_ETIMEOUT at the next synchronising call) after letting its copies in
//    flight finish.
#include <cuda.h>  // CUtensorMap and its enums (the encoder comes from the runtime's driver entry point)
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <tuple>

#include "ew_internal.h"
#include "ew_tb2d_dev.cuh"

namespace ew {

__device__ int g_tma2d_timeout = 0;

template <int R, int NWX, int NTY, int KY, int B>
struct Tma2dShape {
    static constexpr int CWX = 64 * NWX;                 // compute-region width (two columns per lane)
    static constexpr int CWY = NTY * KY;                 // compute-region height
    static constexpr int RX = CWX + 2 * R;               // staged width
    static constexpr int RY = CWY + 2 * R;               // staged height
    static constexpr int BOXW = ((RX + 3) + 3) & ~3;     // copied width: room for the offset o <= 3
    static constexpr int H = R * B;                      // halo
    static constexpr int TX = RX - 2 * H;                // owned tile
    static constexpr int TY = RY - 2 * H;
    static constexpr int NTC = 32 * NWX * NTY;           // compute threads
    static constexpr int NT = NTC + 32;                  // + the producer warp
    static constexpr int BUF = BOXW * RY;                // floats of one copied box
    static constexpr int BUFP = (BUF + 31) & ~31;        // buffer stride: copy destinations 128-byte aligned
    static constexpr size_t SMEM = sizeof(float) * 4 * (size_t)BUFP + 128;  // two slots x (D, W), four mbarriers,
                                                                             // the launch's B filter weights
    static_assert(B <= 16, "the weights of one launch live in the shared-memory tail");
    static_assert(TX > 0 && TY > 0, "halo larger than the tile");
    static_assert(TX % 4 == 0 && (H - R) % 2 == 0, "owned rows 16-byte aligned, column pairs 8-byte aligned");
    static_assert(BOXW <= 256 && RY <= 256, "tensor-map box dimensions are at most 256");
};

__device__ __forceinline__ unsigned tma_smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tma_smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tma_mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(tma_smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(tma_smem_u32(bar)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ bool tma_mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tma_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: gives up after about two seconds of SM clock (or 2^26 polls)
__device__ __forceinline__ bool tma_mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64();
    for (int it = 0; it < (1 << 26); ++it) {
        if (tma_mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > 4000000000ll) break;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(tma_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tma_smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const float* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(tma_smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// named barrier 1 among the NTC compute threads (the producer warp does not join)
template <int NTC>
__device__ __forceinline__ void cbar_sync() {
    asm volatile("bar.sync 1, %0;\n" ::"n"(NTC) : "memory");
}
template <int NTC>
__device__ __forceinline__ bool cbar_or(bool v) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)v), "n"(NTC)
        : "memory");
    return r != 0;
}

// tile number -> (vector, origin of the staged region)
__device__ __forceinline__ void tma_tile(int t, int tiles_x, int tiles_per_vec, int TX, int TY, int H, int& v, int& x0,
                                         int& y0) {
    v = t / tiles_per_vec;
    const int r = t - v * tiles_per_vec;
    const int ty = r / tiles_x;
    x0 = (r - ty * tiles_x) * TX - H;
    y0 = ty * TY - H;
}

// Points of the staged region outside the box: the box closure's extension,
// read from the staged mirror point; 0 when the mirror is not staged (such a
// point lies farther than H from every owned point, so it cannot reach the
// owned tile within B steps).  Mirrors are active points, so no cell is both
// read and written here.
template <int RX, int RY, int BOXW, int NTC, bool GEN>
__device__ __forceinline__ void tma_fixup(float* buf, int nx, int ny, int bc, int x0, int y0, int o, int tid) {
    const int xl = min(max(-x0, 0), RX), xr = max(min(nx - x0, RX), xl);  // active columns [xl, xr)
    const int yl = min(max(-y0, 0), RY), yr = max(min(ny - y0, RY), yl);  // active rows [yl, yr)
    const int ncol = RX - (xr - xl);                                      // outside columns, every row
    const int nrow = RY - (yr - yl);                                      // outside rows, active columns
    const int n1 = ncol * RY, n2 = nrow * (xr - xl);
    for (int q = tid; q < n1 + n2; q += NTC) {
        int sx, sy;
        if (q < n1) {
            const int c = q % ncol;
            sy = q / ncol;
            sx = c < xl ? c : xr + (c - xl);
        } else {
            const int e = q - n1, w = xr - xl;
            const int r = e / w;
            sx = xl + (e - r * w);
            sy = r < yl ? r : yr + (r - yl);
        }
        const int gx = x0 + sx, gy = y0 + sy;
        int sgx = 1, sgy = 1;
        const int ix = ext2<GEN>(gx, nx, axis_bc(bc, 0), sgx), iy = ext2<GEN>(gy, ny, axis_bc(bc, 1), sgy);
        float val = 0.f;
        if (ix >= 0 && iy >= 0) {
            const int mc = ix - x0, mr = iy - y0;
            if (mc >= 0 && mc < RX && mr >= 0 && mr < RY) {
                val = buf[mr * BOXW + o + mc];
                if (sgx * sgy < 0) val = -val;
            }
        }
        buf[sy * BOXW + o + sx] = val;
    }
}

template <int R, int NWX, int NTY, int KY, int B, bool GEN>
__global__ void __launch_bounds__(32 * NWX * NTY + 32, 1)
    k_step_tma2d(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const __grid_constant__ CUtensorMap mapAo, const __grid_constant__ CUtensorMap mapBo, int nx, int ny,
                 float* __restrict__ acc,
                 const float* __restrict__ cw, int b, Stencil<float> st, int tiles_x, int tiles_per_vec, int ntiles,
                 unsigned stall_tx) {
    using S = Tma2dShape<R, NWX, NTY, KY, B>;
    constexpr int RX = S::RX, RY = S::RY, BOXW = S::BOXW, H = S::H, TX = S::TX, TY = S::TY, NTC = S::NTC,
                  BUF = S::BUF, BUFP = S::BUFP;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* slots = reinterpret_cast<float*>(smem_raw);  // [2 slots][D, W][BUFP]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + sizeof(float) * 4 * (size_t)BUFP);
    uint64_t* done = full + 2;
    float* cws = reinterpret_cast<float*>(done + 2);  // c_{n+1} .. c_{n+b}: one shared copy for every tile
    const int tid = threadIdx.x;
    const int64_t N = (int64_t)nx * ny;
    if ((int)blockIdx.x >= ntiles) return;
    if (tid == 0) {
        tma_mbar_init(&full[0], 1);
        tma_mbar_init(&full[1], 1);
        tma_mbar_init(&done[0], NTC / 32);
        tma_mbar_init(&done[1], NTC / 32);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (tid < b) cws[tid] = cw[tid];
    __syncthreads();  // the only CTA-wide barrier: from here on the two roles synchronise by mbarriers

    if (tid >= NTC) {
        // ---------------- producer warp ----------------
        const int lane = tid - NTC;
        const unsigned bytes = 2u * (unsigned)BUF * 4u;
        auto issue = [&](int t, int s, unsigned extra) {  // lane 0: both loads of tile t into slot s
            int v, x0, y0;
            tma_tile(t, tiles_x, tiles_per_vec, TX, TY, H, v, x0, y0);
            const int xa = x0 - (((x0 % 4) + 4) % 4);
            float* bD = slots + (size_t)s * 2 * BUFP;
            tma_mbar_arrive_expect(&full[s], bytes + extra);
            tma_load_3d(bD, &mapA, xa, y0, v, &full[s]);
            tma_load_3d(bD + BUFP, &mapB, xa, y0, v, &full[s]);
        };
        auto warm_acc = [&](int t) {  // L2 prefetch of tile t's filter sums (owned rows, dense layout)
            int v, x0, y0;
            tma_tile(t, tiles_x, tiles_per_vec, TX, TY, H, v, x0, y0);
            constexpr int LPR = (TX + 31) / 32 + 1;  // 128-byte lines per owned row, at most
            for (int q = lane; q < TY * LPR; q += 32) {
                const int r = q / LPR, l = q - r * LPR;
                const int gy = y0 + H + r, gx = min(x0 + H + 32 * l, x0 + H + TX - 1);
                if (gy < ny && gx < nx)
                    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(acc + (int64_t)v * N + (int64_t)gy * nx + gx));
            }
        };
        if (lane == 0) {
            // stall_tx > 0 (a test of the bounded wait): the first copy of slot 0 is
            // expected to bring bytes that never arrive, so the waits run out
            issue(blockIdx.x, 0, stall_tx);
            if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1, 0u);
        }
        warm_acc(blockIdx.x);
        if ((int)(blockIdx.x + gridDim.x) < ntiles) warm_acc(blockIdx.x + gridDim.x);
        unsigned ph = 0u;  // bit s: the parity to wait for on slot s (a register, not an indexed array)
        int k = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
            const int s = k & 1;
            const bool ok = tma_mbar_wait_bounded(&done[s], (ph >> s) & 1u);
            ph ^= 1u << s;
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    bulk_wait_all();
                    atomicExch(&g_tma2d_timeout, 1);
                }
                return;  // the compute warps give up on their next wait
            }
            // write back the owned boxes of W^{n+b} (packed by the last step into the
            // buffer it wrote) and of D^{n+b} (packed into the other one)
            if (lane == 0) {
                int v, x0, y0;
                tma_tile(t, tiles_x, tiles_per_vec, TX, TY, H, v, x0, y0);
                const float* bD = slots + (size_t)s * 2 * BUFP;
                const float* wbuf = ((b - 1) & 1) ? bD + BUFP : bD;
                const float* dbuf = ((b - 1) & 1) ? bD : bD + BUFP;
                tma_store_3d(&mapBo, x0 + H, y0 + H, v, wbuf);
                tma_store_3d(&mapAo, x0 + H, y0 + H, v, dbuf);
                bulk_commit();
            }
            const int tn = t + 2 * gridDim.x;
            if (tn < ntiles) {
                if (lane == 0) {
                    bulk_wait_read();  // the stores have read the slot
                    issue(tn, s, 0u);
                }
                warm_acc(tn);
            }
        }
        if (lane == 0) bulk_wait_all();  // every write-back complete before the CTA ends
        return;
    }

    // ---------------- compute warps ----------------
    const int lane = tid & 31;
    const int wx = (tid >> 5) % NWX;
    const int ty = (tid >> 5) / NWX;
    const int sx = R + 2 * (32 * wx + lane);  // first of the thread's two staged columns
    const int sy0 = R + ty * KY;              // first staged row of its segment
    const float2 C0{st.c0, st.c0}, C1X{st.c1[0], st.c1[0]}, C1Y{st.c1[1], st.c1[1]};
    const float2 C2X{st.c2[0], st.c2[0]}, C2Y{st.c2[1], st.c2[1]};
    unsigned ph = 0u;  // bit s: the parity to wait for on slot s
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k & 1;
        int v, x0, y0;
        tma_tile(t, tiles_x, tiles_per_vec, TX, TY, H, v, x0, y0);
        const int o = ((x0 % 4) + 4) % 4;
        float* bD = slots + (size_t)s * 2 * BUFP;
        float* bW = bD + BUFP;
        const int cx = sx + o;  // shared-memory column of the pair (even)
        const int gx = x0 + sx;
        const int gy0 = y0 + sy0;
        const bool own_a = sx >= H && sx < H + TX && gx < nx;
        const bool own_b = sx + 1 >= H && sx + 1 < H + TX && gx + 1 < nx;
        const int klo = max(0, H - sy0);
        const int khi = min(min(KY, H + TY - sy0), ny - gy0);
        // the filter sums (warmed in L2 by the producer) load while the slot fills
        float2 accp[KY];
        {
            int64_t base = (int64_t)v * N + (int64_t)gy0 * nx + gx;
            asm volatile("" : "+l"(base));
#pragma unroll
            for (int kk = 0; kk < KY; ++kk) {
                const bool oy = kk >= klo && kk < khi;
                accp[kk].x = (own_a && oy) ? acc[base + (int64_t)kk * nx] : 0.f;
                accp[kk].y = (own_b && oy) ? acc[base + (int64_t)kk * nx + 1] : 0.f;
            }
        }
        const bool ok = tma_mbar_wait_bounded(&full[s], (ph >> s) & 1u);
        ph ^= 1u << s;
        if (cbar_or<NTC>(!ok)) {
            if (tid == 0) atomicExch(&g_tma2d_timeout, 1);
            return;  // the producer gives up on its wait for this tile
        }
        if (x0 < 0 || y0 < 0 || x0 + RX > nx || y0 + RY > ny) {
            tma_fixup<RX, RY, BOXW, NTC, GEN>(bD, nx, ny, st.bc, x0, y0, o, tid);
            tma_fixup<RX, RY, BOXW, NTC, GEN>(bW, nx, ny, st.bc, x0, y0, o, tid);
            cbar_sync<NTC>();
        }
        float2 dd[KY];
#pragma unroll
        for (int kk = 0; kk < KY; ++kk) dd[kk] = *reinterpret_cast<const float2*>(bD + (sy0 + kk) * BOXW + cx);
        // bD now serves as the W^{n+1} buffer: each of its entries is read above
        // only by the thread that writes it below
        float* cur = bW;
        float* nxt = bD;
        // the owned box, packed: point (sx, sy) of the staged region at (sy - H) TX + sx - H;
        // a column pair is wholly inside or wholly outside it (sx - H and TX even)
        const bool pair_owned = sx >= H && sx < H + TX;
        const int pk0 = (sy0 - H) * TX + (sx - H);
        for (int step = 0; step < b; ++step) {
            const bool last = step == b - 1;
            const float* col = cur + cx;
            float2 w0 = R == 2 ? *reinterpret_cast<const float2*>(col + (sy0 - 2) * BOXW) : float2{0.f, 0.f};
            float2 w1 = *reinterpret_cast<const float2*>(col + (sy0 - 1) * BOXW);
            float2 w2 = *reinterpret_cast<const float2*>(col + sy0 * BOXW);
            float2 w3 = *reinterpret_cast<const float2*>(col + (sy0 + 1) * BOXW);
            const float cs = cws[step];
            const float2 CS{cs, cs};
#pragma unroll
            for (int kk = 0; kk < KY; ++kk) {
                const int row = (sy0 + kk) * BOXW + cx;
                const float2 w4 = (R == 2 || kk + 1 < KY)
                                      ? *reinterpret_cast<const float2*>(col + (sy0 + kk + 2) * BOXW)
                                      : float2{0.f, 0.f};
                const float2 L = *reinterpret_cast<const float2*>(cur + row - 2);  // columns x-2, x-1
                const float2 Q = *reinterpret_cast<const float2*>(cur + row + 2);  // columns x+2, x+3
                float2 sx1;
                sx1.x = s_add(L.y, w2.y);
                sx1.y = s_add(w2.x, Q.x);
                float2 lap = p_mul(C0, w2);
                lap = p_fma(C1X, sx1, lap);
                lap = p_fma(C1Y, p_add(w1, w3), lap);
                if (R == 2) {
                    lap = p_fma(C2X, p_add(L, Q), lap);
                    lap = p_fma(C2Y, p_add(w0, w4), lap);
                }
                const float2 d = p_add(dd[kk], lap);  // D^{n+1} = D^n + dt^2 L W^n
                const float2 nv = p_add(w2, d);       // W^{n+1} = W^n + D^{n+1}
                if (!last) {
                    *reinterpret_cast<float2*>(nxt + row) = nv;
                } else if (pair_owned && sy0 + kk >= H && sy0 + kk < H + TY) {
                    *reinterpret_cast<float2*>(nxt + pk0 + kk * TX) = nv;
                }
                dd[kk] = d;
                accp[kk] = p_fma(CS, nv, accp[kk]);
                w0 = w1;
                w1 = w2;
                w2 = w3;
                w3 = w4;
            }
            cbar_sync<NTC>();
            float* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        // D^{n+b} packed into the buffer that does not hold W^{n+b} (the last step's
        // barrier ordered every read of it), then hand the slot to the producer
        if (pair_owned) {
#pragma unroll
            for (int kk = 0; kk < KY; ++kk)
                if (sy0 + kk >= H && sy0 + kk < H + TY) *reinterpret_cast<float2*>(nxt + pk0 + kk * TX) = dd[kk];
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) tma_mbar_arrive(&done[s]);
        // the filter sums of the owned points
        {
            const int64_t ab = (int64_t)v * N + (int64_t)gy0 * nx + gx;
#pragma unroll
            for (int kk = 0; kk < KY; ++kk) {
                if (kk >= klo && kk < khi) {
                    const int64_t a = ab + (int64_t)kk * nx;
                    if (own_a) acc[a] = accp[kk].x;
                    if (own_b) acc[a + 1] = accp[kk].y;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#define EW_TMA2D(R, NWX, NTY, KY, B)                                                                         \
    Tma2dDesc {                                                                                              \
        (void*)k_step_tma2d<R, NWX, NTY, KY, B, false>, (void*)k_step_tma2d<R, NWX, NTY, KY, B, true>, NWX, NTY, \
            KY, B, Tma2dShape<R, NWX, NTY, KY, B>::TX, Tma2dShape<R, NWX, NTY, KY, B>::TY,                   \
            Tma2dShape<R, NWX, NTY, KY, B>::NT, Tma2dShape<R, NWX, NTY, KY, B>::SMEM,                        \
            Tma2dShape<R, NWX, NTY, KY, B>::BOXW, Tma2dShape<R, NWX, NTY, KY, B>::RY                         \
    }

const std::vector<Tma2dDesc>& tma2d_variants(int R) {
    // Register budget: a CTA's warps are allocated registers in groups of four, so
    // 20 compute warps + the producer count as 24 warps (80 registers a thread)
    // and 24 + 1 as 28 (72, which spills the step loop of some variants).
    // Order 4: any depth keeps column pairs aligned; order 2: odd depths.
    static const std::vector<Tma2dDesc> r2 = {EW_TMA2D(2, 2, 10, 10, 4), EW_TMA2D(2, 2, 10, 10, 3),
                                              EW_TMA2D(2, 2, 10, 10, 5), EW_TMA2D(2, 2, 10, 10, 6),
                                              EW_TMA2D(2, 2, 12, 8, 4),  EW_TMA2D(2, 2, 12, 8, 6)};
    static const std::vector<Tma2dDesc> r1 = {EW_TMA2D(1, 2, 10, 10, 5), EW_TMA2D(1, 2, 10, 10, 3),
                                              EW_TMA2D(1, 2, 10, 10, 7), EW_TMA2D(1, 2, 10, 10, 9),
                                              EW_TMA2D(1, 2, 12, 8, 5),  EW_TMA2D(1, 2, 12, 8, 7)};
    return R == 1 ? r1 : r2;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link-time
// dependency on the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static std::mutex g_tma_mu;

static ew_status encoder(EncodeTiledFn* out) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return set_error(EW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        fn = (EncodeTiledFn)p;
    }
    *out = fn;
    return EW_OK;
}

// the map of one time-level field slot: x extent nx, y extent ny, one plane
// per vector; boxes of boxw x boxh x 1
using MapKey = std::tuple<uintptr_t, int64_t, int64_t, int64_t, int, int64_t, int, int>;
static std::map<MapKey, CUtensorMap> g_maps;

static ew_status field_map(const float* base, int64_t nx, int64_t ny, int64_t pitch, int nvec, int64_t fstride,
                           int boxw, int boxh, CUtensorMap* out) {
    MapKey key{(uintptr_t)base, nx, ny, pitch, nvec, fstride, boxw, boxh};
    std::lock_guard<std::mutex> lk(g_tma_mu);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) {
        *out = it->second;
        return EW_OK;
    }
    EncodeTiledFn enc = nullptr;
    EW_TRY(encoder(&enc));
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nvec};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)fstride * 4};
    const cuuint32_t box[3] = {(cuuint32_t)boxw, (cuuint32_t)boxh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(EW_ECUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    if (g_maps.size() > 4096) g_maps.clear();  // grids come and go: keep the cache bounded
    g_maps[key] = m;
    *out = m;
    return EW_OK;
}

ew_status tma2d_launch(const Tma2dDesc& d, const GridGeom& g, const float* Ain, const float* Bin, float* Aout,
                       float* Bout, float* acc, const float* cw, int b, const Stencil<float>& s, int nvec,
                       int64_t fstride, cudaStream_t st) {
    const int64_t pitch = pitch2d(g.n[0]);
    if (g.dim != 2 || (((uintptr_t)Ain | (uintptr_t)Bin | (uintptr_t)Aout | (uintptr_t)Bout) & 15) || (fstride & 3) ||
        fstride < pitch * g.n[1])
        return set_error(EW_EUNSUPPORTED, "TMA-staged step needs 16-byte aligned 2D fields of padded pitch");
    if (b < 1 || b > d.B) return set_error(EW_EINVAL, "TMA-staged step: depth out of range");
    int dev = 0, nsm = 0;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    void* fn = g.bc ? d.fn_gen : d.fn;
    {
        static std::map<std::pair<void*, int>, int> sms;
        std::lock_guard<std::mutex> lk(g_tma_mu);
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
    CUtensorMap mA, mB, mAo, mBo;  // loads: the staged box; stores: the owned tile
    EW_TRY(field_map(Ain, g.n[0], g.n[1], pitch, nvec, fstride, d.boxw, d.boxh, &mA));
    EW_TRY(field_map(Bin, g.n[0], g.n[1], pitch, nvec, fstride, d.boxw, d.boxh, &mB));
    EW_TRY(field_map(Aout, g.n[0], g.n[1], pitch, nvec, fstride, d.TX, d.TY, &mAo));
    EW_TRY(field_map(Bout, g.n[0], g.n[1], pitch, nvec, fstride, d.TX, d.TY, &mBo));
    int nx = (int)g.n[0], ny = (int)g.n[1];
    int tiles_x = (nx + d.TX - 1) / d.TX, tiles_y = (ny + d.TY - 1) / d.TY;
    int64_t nt64 = (int64_t)tiles_x * tiles_y * nvec;
    if (nt64 > INT32_MAX) return set_error(EW_EUNSUPPORTED, "TMA-staged step: too many tiles");
    int tiles_per_vec = tiles_x * tiles_y, ntiles = (int)nt64;
    int grid = std::min(ntiles, nsm);
    // EW_TEST_RB2D_STALL: test hook that makes every CTA's first staging wait run out
    unsigned stall_tx = getenv("EW_TEST_RB2D_STALL") ? 16u : 0u;
    void* args[] = {(void*)&mA,  (void*)&mB,      (void*)&mAo,           (void*)&mBo,     (void*)&nx,
                    (void*)&ny,  (void*)&acc,     (void*)&cw,            (void*)&b,       (void*)&s,
                    (void*)&tiles_x, (void*)&tiles_per_vec, (void*)&ntiles, (void*)&stall_tx};
    cudaEvent_t ev = fused_begin(st);
    EW_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(d.threads), args, d.smem, st));
    fused_end(ev, st, g.N * nvec, g.N * nvec * b);
    return EW_OK;
}

ew_status tma2d_check_timeout() {
    int flag = 0, zero = 0;
    EW_CUDA_TRY(cudaMemcpyFromSymbol(&flag, g_tma2d_timeout, sizeof(int)));
    if (!flag) return EW_OK;
    EW_CUDA_TRY(cudaMemcpyToSymbol(g_tma2d_timeout, &zero, sizeof(int)));
    return set_error(EW_ETIMEOUT, "a staging copy of the TMA-staged step did not complete");
}

}  // namespace ew
