// ew_smoother.cu -- learned multigrid smoother: forward, backward, training.
//
// The correction N(r) of a residual r (3D, zero outside the active box):
//   h_c(x) = sum_{o in {-1,0,1}^3} W1[c][o] r(x + o),      c = 0..7
//   N(r)(x) = sum_c sum_o W2[c][o] h_c(x + o)
// no bias, no activation, so the smoothing step x <- x + N(b - M x) is linear
// and the multigrid solve (hence the filter operator) stays linear.  Weights,
// the input residual and the hidden activations are rounded to BF16; every
// product is accumulated in FP32 (tensor-core numerics).  Tap order of W[c][o]:
// o = (dz, dy, dx), dz slowest.
//
// Training loss on a residual sample r (with e = M^{-1} r the error it stems
// from, the loss is the M-weighted error left after the correction):
//   loss = 1/2 ||M (e - N(r))||^2 = 1/2 ||r - M N(r)||^2
//   dloss/dN = -M (r - M N(r))     (M symmetric)
// The gradient of the weights is reduced over the grid in a fixed order.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ew_internal.h"
#include "ew_stencil_dev.cuh"

namespace ew {

constexpr int kC = 8;       // hidden channels
constexpr int kW = kC * 27; // weights per layer
constexpr int kTile = 8;    // output tile edge
constexpr int kThreads = 256;
constexpr int kRE = kTile + 4;  // staged residual edge (halo 2)
constexpr int kHE = kTile + 2;  // hidden edge (halo 1)

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

template <typename T>
__device__ __forceinline__ float ld_r(const T* __restrict__ r, int x, int y, int z, int nx, int ny, int nz) {
    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return 0.f;
    return bf16r((float)r[((int64_t)z * ny + y) * nx + x]);
}

// stage r (halo 2) and compute the hidden layer (halo 1, zero outside the box)
template <typename T>
__device__ void stage_hidden(const T* __restrict__ r, const float* sW1, float* sR, float* sH, int x0, int y0, int z0,
                             int nx, int ny, int nz) {
    for (int q = threadIdx.x; q < kRE * kRE * kRE; q += kThreads) {
        int lx = q % kRE, t = q / kRE, ly = t % kRE, lz = t / kRE;
        sR[q] = ld_r(r, x0 - 2 + lx, y0 - 2 + ly, z0 - 2 + lz, nx, ny, nz);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kHE * kHE * kHE; q += kThreads) {
        int lx = q % kHE, t = q / kHE, ly = t % kHE, lz = t / kHE;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
        float acc[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) acc[c] = 0.f;
        if (gx >= 0 && gy >= 0 && gz >= 0 && gx < nx && gy < ny && gz < nz) {
            int tap = 0;
            for (int dz = 0; dz < 3; ++dz)
                for (int dy = 0; dy < 3; ++dy)
                    for (int dx = 0; dx < 3; ++dx, ++tap) {
                        float rv = sR[((lz + dz) * kRE + (ly + dy)) * kRE + (lx + dx)];
#pragma unroll
                        for (int c = 0; c < kC; ++c) acc[c] = fmaf(sW1[c * 27 + tap], rv, acc[c]);
                    }
        }
#pragma unroll
        for (int c = 0; c < kC; ++c) sH[q * kC + c] = bf16r(acc[c]);
    }
    __syncthreads();
}

// x += N(r) (add = true) or y = N(r) (add = false)
template <typename T, bool ADD>
__global__ void __launch_bounds__(kThreads)
    k_smoother_fwd(int nx, int ny, int nz, const float* __restrict__ w, const T* __restrict__ r, T* __restrict__ out) {
    __shared__ float sW[2 * kW];
    __shared__ float sR[kRE * kRE * kRE];
    __shared__ float sH[kHE * kHE * kHE * kC];
    for (int q = threadIdx.x; q < 2 * kW; q += kThreads) sW[q] = bf16r(w[q]);
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile, z0 = blockIdx.z * kTile;
    __syncthreads();
    stage_hidden<T>(r, sW, sR, sH, x0, y0, z0, nx, ny, nz);
    const float* sW2 = sW + kW;
    for (int q = threadIdx.x; q < kTile * kTile * kTile; q += kThreads) {
        int lx = q % kTile, t = q / kTile, ly = t % kTile, lz = t / kTile;
        int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        if (gx >= nx || gy >= ny || gz >= nz) continue;
        float s = 0.f;
        int tap = 0;
        for (int dz = 0; dz < 3; ++dz)
            for (int dy = 0; dy < 3; ++dy)
                for (int dx = 0; dx < 3; ++dx, ++tap) {
                    const float* hp = sH + (((lz + dz) * kHE + (ly + dy)) * kHE + (lx + dx)) * kC;
#pragma unroll
                    for (int c = 0; c < kC; ++c) s = fmaf(sW2[c * 27 + tap], hp[c], s);
                }
        int64_t g = ((int64_t)gz * ny + gy) * nx + gx;
        if (ADD)
            out[g] += (T)s;
        else
            out[g] = (T)s;
    }
}

// per-block partial gradients: part[block][432]
//   dW2[c][o] = sum_x gy(x) h_c(x + o)
//   dh_c(x)   = sum_o W2[c][o] gy(x - o)
//   dW1[c][o] = sum_x dh_c(x) r(x + o)
// (the hidden activations and the residual enter with their BF16 rounding)
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_smoother_bwd(int nx, int ny, int nz, const float* __restrict__ w, const T* __restrict__ r,
                   const T* __restrict__ gy, double* __restrict__ part) {
    __shared__ float sW[2 * kW];
    __shared__ float sR[kRE * kRE * kRE];
    __shared__ float sH[kHE * kHE * kHE * kC];
    __shared__ float sG[kHE * kHE * kHE];      // gy on tile + halo 1
    __shared__ float sD[kTile * kTile * kTile * kC];  // dh on the tile
    for (int q = threadIdx.x; q < 2 * kW; q += kThreads) sW[q] = bf16r(w[q]);
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile, z0 = blockIdx.z * kTile;
    __syncthreads();
    stage_hidden<T>(r, sW, sR, sH, x0, y0, z0, nx, ny, nz);
    for (int q = threadIdx.x; q < kHE * kHE * kHE; q += kThreads) {
        int lx = q % kHE, t = q / kHE, ly = t % kHE, lz = t / kHE;
        int gx = x0 - 1 + lx, gyy = y0 - 1 + ly, gz = z0 - 1 + lz;
        bool in = gx >= 0 && gyy >= 0 && gz >= 0 && gx < nx && gyy < ny && gz < nz;
        sG[q] = in ? (float)gy[((int64_t)gz * ny + gyy) * nx + gx] : 0.f;
    }
    __syncthreads();
    const float* sW2 = sW + kW;
    // dh on the owned tile (zero outside the box)
    for (int q = threadIdx.x; q < kTile * kTile * kTile; q += kThreads) {
        int lx = q % kTile, t = q / kTile, ly = t % kTile, lz = t / kTile;
        int gx = x0 + lx, gyy = y0 + ly, gz = z0 + lz;
        float acc[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) acc[c] = 0.f;
        if (gx < nx && gyy < ny && gz < nz) {
            int tap = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx, ++tap) {
                        float g = sG[((lz + 1 - dz) * kHE + (ly + 1 - dy)) * kHE + (lx + 1 - dx)];
#pragma unroll
                        for (int c = 0; c < kC; ++c) acc[c] = fmaf(sW2[c * 27 + tap], g, acc[c]);
                    }
        }
#pragma unroll
        for (int c = 0; c < kC; ++c) sD[q * kC + c] = acc[c];
    }
    __syncthreads();
    // each thread accumulates a few of the 432 gradient entries over the tile;
    // entry e < 216: dW1[c][tap], else dW2[c][tap]
    for (int e = threadIdx.x; e < 2 * kW; e += kThreads) {
        const int c = (e % kW) / 27, tap = (e % kW) % 27;
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        double s = 0.0;
        for (int q = 0; q < kTile * kTile * kTile; ++q) {
            int lx = q % kTile, t = q / kTile, ly = t % kTile, lz = t / kTile;
            float term;
            if (e < kW)
                term = sD[q * kC + c] * sR[((lz + 2 + dz) * kRE + (ly + 2 + dy)) * kRE + (lx + 2 + dx)];
            else
                term = sG[((lz + 1) * kHE + (ly + 1)) * kHE + (lx + 1)] *
                       sH[(((lz + 1 + dz) * kHE + (ly + 1 + dy)) * kHE + (lx + 1 + dx)) * kC + c];
            s += (double)term;
        }
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[b * (2 * kW) + e] = s;
    }
}

__global__ void k_grad_finish(const double* __restrict__ part, int64_t nblocks, float* __restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * kW) return;
    double s = 0.0;
    for (int64_t b = 0; b < nblocks; ++b) s += part[b * (2 * kW) + e];
    grad[e] = (float)s;
}

// Adam step on the 432 weights (device-resident moments)
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       float lr, float b1, float b2, float eps, int step, float gscale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * kW) return;
    float gg = g[e] * gscale;
    m[e] = b1 * m[e] + (1.f - b1) * gg;
    v[e] = b2 * v[e] + (1.f - b2) * gg * gg;
    float mh = m[e] / (1.f - powf(b1, (float)step));
    float vh = v[e] / (1.f - powf(b2, (float)step));
    w[e] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// Tensor-core forward (FP32 fields): both layers on BF16 mma.sync.m16n8k16
// with FP32 accumulation, streamed along z.
//
//   layer 1  H[q][c]  = sum_k A[q][k] B1[k][c]   A = im2col of r (k = tap,
//            27 padded to 32), B1[k][c] = W1[c][k]; 16 hidden points of one
//            plane per MMA row block, N = 8 channels
//   layer 2  Z[q][o]  = sum_c H[q][c] B2[c][o]  B2[c][o] = W2[c][o] (K = 8
//            channels padded to 16, N = 27 taps padded to 32): the accumulator
//            fragment of layer 1, rounded to BF16, is exactly the A fragment of
//            layer 2 (row q, k = c), so H never leaves registers
//   output   N(r)(x) = sum_o Z[x + o][o]
//
// A CTA owns a 16 x 16 column of outputs and kZC planes of it.  Step s
// computes hidden plane hz = z0 - 1 + s (18 x 18 points) from a three-plane
// ring of residual planes, stores its Z (27 taps) in shared memory, and each
// thread adds the taps of that plane to the three output planes it touches
// (hz + 1, hz, hz - 1 for dz = -1, 0, +1), kept in registers; output plane
// hz - 1 is then complete.  Hidden points outside the box are zero (the
// second convolution's zero padding).
// ---------------------------------------------------------------------------
constexpr int kOX = 16, kOY = 16, kZC = 32;          // output column and planes per CTA
constexpr int kHX = kOX + 2, kHY = kOY + 2;          // hidden plane (halo 1)
constexpr int kRX = kOX + 4, kRY = kOY + 4;          // residual plane (halo 2)
constexpr int kHP = kHX * kHY;                       // 324 hidden points per plane
constexpr int kHG = (kHP + 15) / 16;                 // 21 row blocks of 16
constexpr int kZS = kHG * 16 + 4;                    // Z row stride (340: conflict-free stores)
constexpr int kRP = kRX * kRY;                       // 400 residual points per plane
constexpr int kRS = (kRP + 31) / 32 * 32;            // plane slot stride (416: bank-aligned slots)
__device__ constexpr int kTapOrder[32] = {10, 24, 25, 14, 23, 7,  13, 2,  -1, 0, 16, 12, 15, -1, 9,  4,
                                          21, 6,  -1, 18, 22, 8, 19, -1, 17, 1, 3,  -1, 26, 5,  20, 11};
constexpr int kTcThreads = kOX * kOY;                // 256: one output column each

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <bool ADD>
__global__ void __launch_bounds__(kTcThreads, 4)
    k_smoother_fwd_tc(int nx, int ny, int nz, const float* __restrict__ w, const float* __restrict__ r,
                      float* __restrict__ out) {
    extern __shared__ __align__(16) float smem_tc[];
    float* sR = smem_tc;               // [3][kRS]: residual planes, ring indexed by plane mod 3
    float* sZ = smem_tc + 3 * kRS;     // [27][kZS]: Z of the current hidden plane
    int* sHB = reinterpret_cast<int*>(sZ + 27 * kZS);  // [kHG * 16]: residual offset of each hidden point, -1 outside
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const int x0 = blockIdx.x * kOX, y0 = blockIdx.y * kOY, z0 = blockIdx.z * kZC;
    const int z1 = min(nz, z0 + kZC);
    // hidden points of a plane: offset of tap (-1,-1) in a residual plane, -1 if outside the box in x/y
    for (int q = tid; q < kHG * 16; q += kTcThreads) {
        const int hx = q % kHX, hy = q / kHX;
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
        sHB[q] = (q < kHP && gx >= 0 && gy >= 0 && gx < nx && gy < ny) ? hy * kRX + hx : -1;
    }
    auto load_plane = [&](int zr) {  // residual plane zr (BF16-rounded, zero outside) into its ring slot
        float* dst = sR + ((zr + 3) % 3) * kRS;
        for (int q = tid; q < kRP; q += kTcThreads) {
            const int lx = q % kRX, ly = q / kRX;
            dst[q] = ld_r(r, x0 - 2 + lx, y0 - 2 + ly, zr, nx, ny, nz);
        }
    };
    // B fragments (fixed per thread).  Layer 1, k-step s: b0 = B1[16s + 2tig (+1)][g],
    // b1 = B1[16s + 2tig + 8 (+1)][g] with B1[k][c] = W1[c][k] (0 for k >= 27).
    // K order of layer 1.  Slot e (0..7) of lane group tig holds tap kTapOrder[4e + tig]
    // (k = 16 (e >> 2) + 2 tig + (e & 1) + 8 ((e >> 1) & 1) in the MMA); any order works as
    // long as A and B use the same one.  This one keeps the four lanes of one load on
    // different shared-memory banks as far as the 27 offsets allow (searched offline for
    // the row pitch kRX = 20 and 32-float-aligned plane slots); -1 marks a padding slot,
    // which reads the address of another lane of its load (a broadcast) times a zero weight.
    const int tapo[8] = {kTapOrder[tig], kTapOrder[4 + tig], kTapOrder[8 + tig], kTapOrder[12 + tig],
                         kTapOrder[16 + tig], kTapOrder[20 + tig], kTapOrder[24 + tig], kTapOrder[28 + tig]};
    auto w1 = [&](int tap, int c) { return tap >= 0 ? w[c * 27 + tap] : 0.f; };
    uint32_t b1f[2][2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        b1f[s][0] = pack_bf16(w1(tapo[4 * s], g), w1(tapo[4 * s + 1], g));
        b1f[s][1] = pack_bf16(w1(tapo[4 * s + 2], g), w1(tapo[4 * s + 3], g));
    }
    // layer 2, n-tile j: b0 = B2[2tig (+1)][8j + g] = W2[2tig (+1)][8j + g], b1 = 0 (k >= 8)
    uint32_t b2f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int o = 8 * j + g;
        b2f[j] = o < 27 ? pack_bf16(w[kW + (2 * tig) * 27 + o], w[kW + (2 * tig + 1) * 27 + o]) : 0u;
    }
    // this thread's im2col taps; tap t = (dz+1) 9 + (dy+1) 3 + (dx+1): residual plane dz
    // (relative), offset dy * kRX + dx
    int tdz[8], toff[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        int t = tapo[e];
        if (t < 0)  // padding: the address of the first real tap of this load
            for (int u = 3; u >= 0; --u)
                if (kTapOrder[4 * e + u] >= 0) t = kTapOrder[4 * e + u];
        tdz[e] = t / 9;
        toff[e] = ((t / 3) % 3) * kRX + t % 3;
    }
    load_plane(z0 - 2);
    load_plane(z0 - 1);
    // the next residual plane is loaded into registers one step ahead (raw; the
    // BF16 rounding is applied when it is stored, a step later)
    float pr[2];
    auto prefetch = [&](int zr) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = tid + u * kTcThreads;
            const int lx = q % kRX, ly = q / kRX;
            const int xx = x0 - 2 + lx, yy = y0 - 2 + ly;
            pr[u] = 0.f;
            if (q < kRP && xx >= 0 && yy >= 0 && zr >= 0 && xx < nx && yy < ny && zr < nz)
                pr[u] = r[((int64_t)zr * ny + yy) * nx + xx];
        }
    };
    auto commit = [&](int zr) {
        float* dst = sR + ((zr + 3) % 3) * kRS;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = tid + u * kTcThreads;
            if (q < kRP) dst[q] = bf16r(pr[u]);
        }
    };
    prefetch(z0);
    const int ox = tid % kOX, oy = tid / kOX;  // this thread's output column
    const int gx = x0 + ox, gy = y0 + oy;
    const bool own = gx < nx && gy < ny;
    float oa = 0.f, ob = 0.f, oc = 0.f;        // output planes hz - 1, hz, hz + 1
    for (int hz = z0 - 1; hz <= z1; ++hz) {
        commit(hz + 1);
        prefetch(hz + 2);
        __syncthreads();  // residual planes hz-1..hz+1 in place; the previous Z has been read
        const bool zin = hz >= 0 && hz < nz;
        if (zin) {
            // ring slots of residual planes hz - 1, hz, hz + 1 -> each tap's offset in sR
            const int s0 = ((hz + 2) % 3) * kRS, s1 = ((hz + 3) % 3) * kRS, s2 = ((hz + 4) % 3) * kRS;
            int tap[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) tap[e] = (tdz[e] == 0 ? s0 : tdz[e] == 1 ? s1 : s2) + toff[e];
            for (int G = warp; G < kHG; G += kTcThreads / 32) {
                const int q0 = 16 * G + g, q1 = q0 + 8;
                const int hb0 = sHB[q0], hb1 = sHB[q1];
                const int bb0 = hb0 < 0 ? 0 : hb0, bb1 = hb1 < 0 ? 0 : hb1;
                float h[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    uint32_t a[4];
                    const int e = 4 * s2;
                    a[0] = pack_bf16(sR[bb0 + tap[e]], sR[bb0 + tap[e + 1]]);
                    a[1] = pack_bf16(sR[bb1 + tap[e]], sR[bb1 + tap[e + 1]]);
                    a[2] = pack_bf16(sR[bb0 + tap[e + 2]], sR[bb0 + tap[e + 3]]);
                    a[3] = pack_bf16(sR[bb1 + tap[e + 2]], sR[bb1 + tap[e + 3]]);
                    mma_bf16(h, a, b1f[s2][0], b1f[s2][1]);
                }
                // h: (row g, channels 2tig, 2tig+1), (row g+8, same): zero outside the box,
                // round to BF16 -> the A fragment of layer 2 (k = channel; k >= 8 zero)
                uint32_t a2[4];
                a2[0] = hb0 >= 0 ? pack_bf16(h[0], h[1]) : 0u;
                a2[1] = hb1 >= 0 ? pack_bf16(h[2], h[3]) : 0u;
                a2[2] = 0u;
                a2[3] = 0u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float zf[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_bf16(zf, a2, b2f[j], 0u);
                    const int o = 8 * j + 2 * tig;
                    if (o < 27) {
                        sZ[o * kZS + q0] = zf[0];
                        sZ[o * kZS + q1] = zf[2];
                    }
                    if (o + 1 < 27) {
                        sZ[(o + 1) * kZS + q0] = zf[1];
                        sZ[(o + 1) * kZS + q1] = zf[3];
                    }
                }
            }
        }
        __syncthreads();  // Z of plane hz complete
        if (zin) {
            // taps of plane hz: dz = +1 feeds output plane hz - 1, dz = 0 plane hz, dz = -1 plane hz + 1
            float t[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
                        t[dz] += sZ[(dz * 9 + dy * 3 + dx) * kZS + (oy + dy) * kHX + (ox + dx)];
            oa += t[2];
            ob += t[1];
            oc += t[0];
        }
        // output plane hz - 1 is complete
        const int zo = hz - 1;
        if (own && zo >= z0 && zo < z1) {
            const int64_t gi = ((int64_t)zo * ny + gy) * nx + gx;
            if (ADD)
                out[gi] += oa;
            else
                out[gi] = oa;
        }
        oa = ob;
        ob = oc;
        oc = 0.f;
    }
}

static dim3 tc_tiles(const GridGeom& g) {
    return dim3((unsigned)((g.n[0] + kOX - 1) / kOX), (unsigned)((g.n[1] + kOY - 1) / kOY),
                (unsigned)((g.n[2] + kZC - 1) / kZC));
}

constexpr size_t kTcSmem = sizeof(float) * (3 * (size_t)kRS + 27 * (size_t)kZS) + sizeof(int) * kHG * 16;

template <bool ADD>
static ew_status launch_fwd_tc(const GridGeom& g, const float* w, const float* r, float* out, cudaStream_t st);


template <bool ADD>
static ew_status launch_fwd_tc(const GridGeom& g, const float* w, const float* r, float* out, cudaStream_t st) {
    static bool attr = false;  // raised once per process (same value on every device)
    if (!attr) {
        EW_CUDA_TRY(cudaFuncSetAttribute(k_smoother_fwd_tc<ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmem));
        attr = true;
    }
    k_smoother_fwd_tc<ADD><<<tc_tiles(g), kTcThreads, kTcSmem, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], w, r, out);
    EW_CUDA_TRY(cudaGetLastError());
    return EW_OK;
}

static dim3 tiles(const GridGeom& g) {
    return dim3((unsigned)((g.n[0] + kTile - 1) / kTile), (unsigned)((g.n[1] + kTile - 1) / kTile),
                (unsigned)((g.n[2] + kTile - 1) / kTile));
}

// x += N(r): tensor cores for FP32 fields, the CUDA-core kernel for FP64 ones
template <typename T>
ew_status smoother_apply(const GridGeom& g, const float* weights, const T* r, T* x, cudaStream_t st) {
    if constexpr (sizeof(T) == 4)
        EW_TRY(launch_fwd_tc<true>(g, weights, r, x, st));
    else
        k_smoother_fwd<T, true><<<tiles(g), kThreads, 0, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], weights, r, x);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}
template ew_status smoother_apply<float>(const GridGeom&, const float*, const float*, float*, cudaStream_t);
template ew_status smoother_apply<double>(const GridGeom&, const float*, const double*, double*, cudaStream_t);

template <typename T>
static ew_status smoother_forward_t(const GridGeom& g, const float* w, const T* r, T* y, cudaStream_t st) {
    if constexpr (sizeof(T) == 4)
        EW_TRY(launch_fwd_tc<false>(g, w, r, y, st));
    else
        k_smoother_fwd<T, false><<<tiles(g), kThreads, 0, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], w, r, y);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}

template <typename T>
static ew_status smoother_backward_t(ew_grid* gr, const float* w, const T* r, const T* gy, float* grad, cudaStream_t st) {
    const GridGeom& g = gr->geom;
    dim3 tl = tiles(g);
    int64_t nb = (int64_t)tl.x * tl.y * tl.z;
    EW_TRY(gr->reduce.reserve(sizeof(double) * (size_t)nb * 2 * kW));
    double* part = (double*)gr->reduce.ptr;
    k_smoother_bwd<T><<<tl, kThreads, 0, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], w, r, gy, part);
    k_grad_finish<<<(2 * kW + 127) / 128, 128, 0, st>>>(part, nb, grad);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch(2);
    return EW_OK;
}

static ew_status check_smoother_grid(const ew_grid* g) {
    if (!g) return set_error(EW_EINVAL, "grid is NULL");
    if (g->geom.dim != 3) return set_error(EW_EUNSUPPORTED, "the learned smoother is three-dimensional");
    if (g->geom.n[0] > INT32_MAX / 2 || g->geom.n[1] > INT32_MAX / 2 || g->geom.n[2] > INT32_MAX / 2)
        return set_error(EW_EINVAL, "axis too long");
    return EW_OK;
}

// multigrid pieces used by the trainer (ew_mg.cu)
ew_status mg_collect_residuals(ew_grid* g, double a, const ew_mg_params* mp, int nsamples, uint64_t seed, float* out,
                               cudaStream_t st);
ew_status mg_convergence(ew_grid* g, double a, const ew_mg_params* mp, int ncycles, uint64_t seed, double* rho,
                         cudaStream_t st);

}  // namespace ew

using namespace ew;

extern "C" {

ew_status ew_smoother_forward(const ew_grid* grid, const float* w, const void* r, void* y, cudaStream_t st) try {
    clear_error();
    EW_TRY(check_smoother_grid(grid));
    if (!w || !r || !y) return set_error(EW_EINVAL, "null pointer");
    if (grid->prec == EW_FP32) return smoother_forward_t<float>(grid->geom, w, (const float*)r, (float*)y, st);
    return smoother_forward_t<double>(grid->geom, w, (const double*)r, (double*)y, st);
} catch (...) {
    return abi_exception();
}

ew_status ew_smoother_backward(const ew_grid* grid, const float* w, const void* r, const void* gy, float* grad,
                               cudaStream_t st) try {
    clear_error();
    EW_TRY(check_smoother_grid(grid));
    if (!w || !r || !gy || !grad) return set_error(EW_EINVAL, "null pointer");
    ew_grid* g = const_cast<ew_grid*>(grid);
    if (grid->prec == EW_FP32) return smoother_backward_t<float>(g, w, (const float*)r, (const float*)gy, grad, st);
    return smoother_backward_t<double>(g, w, (const double*)r, (const double*)gy, grad, st);
} catch (...) {
    return abi_exception();
}

ew_status ew_smoother_train(const ew_grid* grid, double half_dt2, const ew_train_params* tp, float* weights,
                            ew_train_report* rep, cudaStream_t st) try {
    clear_error();
    EW_TRY(check_smoother_grid(grid));
    if (!tp || !weights) return set_error(EW_EINVAL, "null pointer");
    if (grid->prec != EW_FP32) return set_error(EW_EUNSUPPORTED, "training runs on FP32 grids");
    if (tp->steps < 1 || tp->samples < 1 || !(tp->lr > 0)) return set_error(EW_EINVAL, "bad training parameters");
    ew_grid* g = const_cast<ew_grid*>(grid);
    const int64_t N = g->geom.N;
    const double a = half_dt2;
    ew_mg_params plain{tp->pre, tp->post, 1, 0.0, tp->jacobi_weight > 0 ? tp->jacobi_weight : 0.8, 0, nullptr, 0};
    // device buffers: samples, N(r), M N(r), e = r - M N(r), gy, weight state
    struct DeviceBuffers {  // freed on every return path
        std::vector<void*> p;
        ~DeviceBuffers() {
            for (void* q : p) cudaFree(q);
        }
    } allocs;
    auto alloc = [&](void** p, size_t bytes) -> ew_status {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(EW_ENOMEM, "training workspace allocation failed");
        }
        allocs.p.push_back(*p);
        return EW_OK;
    };
    float *samples = nullptr, *y = nullptr, *My = nullptr, *res = nullptr, *gy = nullptr, *state = nullptr;
    ew_status s = EW_OK;
    if (s == EW_OK) s = alloc((void**)&samples, sizeof(float) * (size_t)N * tp->samples);
    if (s == EW_OK) s = alloc((void**)&y, sizeof(float) * (size_t)N);
    if (s == EW_OK) s = alloc((void**)&My, sizeof(float) * (size_t)N);
    if (s == EW_OK) s = alloc((void**)&res, sizeof(float) * (size_t)N);
    if (s == EW_OK) s = alloc((void**)&gy, sizeof(float) * (size_t)N);
    if (s == EW_OK) s = alloc((void**)&state, sizeof(float) * 4 * 2 * kW);  // grad, m, v, best
    if (s != EW_OK) return s;
    float* grad = state;
    float* m = state + 2 * kW;
    float* v = state + 4 * kW;
    float* best = state + 6 * kW;
    cudaMemsetAsync(m, 0, sizeof(float) * 4 * kW, st);
    cudaMemcpyAsync(best, weights, sizeof(float) * 2 * kW, cudaMemcpyDeviceToDevice, st);
    // (1) residual samples from plain multigrid solves of this system
    s = mg_collect_residuals(g, a, &plain, tp->samples, tp->seed, samples, st);
    // (2) gradient steps: loss 1/2 ||r - M N(r)||^2 / ||r||^2 (every sample
    //     weighs the same whatever its size), gradient -M (r - M N(r)) / ||r||^2
    double loss_first = 0.0, loss_last = 0.0;
    EW_TRY(g->misc.reserve(sizeof(double) * (kReduceBlocks + 8)));
    double* dpart = (double*)g->misc.ptr;
    double* dloss = dpart + kReduceBlocks;
    std::vector<double> rn2(tp->samples, 1.0);
    for (int k = 0; k < tp->samples && s == EW_OK; ++k) {
        s = launch_dots<float>(samples + (size_t)k * N, samples + (size_t)k * N, N, 1, dpart, dloss, st);
        if (s == EW_OK) {
            cudaMemcpyAsync(&rn2[k], dloss, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            if (!(rn2[k] > 0.0)) rn2[k] = 1.0;
        }
    }
    auto applyM = [&](const float* in, float* out) -> ew_status {
        // out = M in = in - a L in
        EW_TRY(launch_apply_L<float>(g->geom, in, out, 1, -a, st));
        return EW_OK;
    };
    for (int step = 0; step < tp->steps && s == EW_OK; ++step) {
        const int ks = step % tp->samples;
        const float* r = samples + (size_t)ks * N;
        s = smoother_forward_t<float>(g->geom, weights, r, y, st);
        if (s == EW_OK) s = applyM(y, My);                           // My = -a L y (partial)
        if (s == EW_OK) s = axpy_f(N, 1.f, y, My, st);               // My = y - a L y = M y
        if (s == EW_OK) {                                            // res = r - M y
            cudaMemcpyAsync(res, r, sizeof(float) * N, cudaMemcpyDeviceToDevice, st);
            s = axpy_f(N, -1.f, My, res, st);
        }
        if (s == EW_OK) s = applyM(res, gy);                         // gy = -a L res
        if (s == EW_OK) s = axpy_f(N, 1.f, res, gy, st);             // gy = M res
        if (s == EW_OK) s = launch_dots<float>(res, res, N, 1, dpart, dloss, st);
        // dloss/dN = -M res: the backward takes gy and the sign goes into the step
        if (s == EW_OK) s = smoother_backward_t<float>(g, weights, r, gy, grad, st);
        double l2 = 0.0;
        if (s == EW_OK) {
            cudaMemcpyAsync(&l2, dloss, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            // the backward took +M res; the true gradient is -M res / ||r||^2
            k_adam<<<(2 * kW + 127) / 128, 128, 0, st>>>(weights, grad, m, v, (float)tp->lr, 0.9f, 0.999f, 1e-20f,
                                                         step + 1, (float)(-1.0 / rn2[ks]));
            count_launch();
        }
        if (step < tp->samples) loss_first += 0.5 * l2 / rn2[ks] / std::min(tp->samples, tp->steps);
        if (step >= tp->steps - tp->samples) loss_last += 0.5 * l2 / rn2[ks] / std::min(tp->samples, tp->steps);
    }
    // (3) acceptance: convergence factor of plain and learned V-cycles on the same
    //     system.  The correction is linear in W2, so scaling W2 by s scales
    //     N by s; a few scalings are compared and the best one is kept.
    const int jc = tp->accept_cycles > 0 ? tp->accept_cycles : 6;
    double rho_plain = 0.0, rho_learned = INFINITY;
    if (s == EW_OK) s = mg_convergence(g, a, &plain, jc, tp->seed + 99, &rho_plain, st);
    std::vector<float> hw(2 * kW), hbest(2 * kW);
    if (s == EW_OK) {
        cudaMemcpyAsync(hw.data(), weights, sizeof(float) * 2 * kW, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
    }
    float* trial = grad;  // reuse the gradient buffer for the scaled weights
    ew_mg_params learned = plain;
    learned.learned_levels = 1;
    learned.weights_dev = trial;
    const double scales[4] = {1.0, 0.85, 0.7, 0.5};
    for (int q = 0; q < 4 && s == EW_OK; ++q) {
        std::vector<float> ht(hw);
        for (int e = kW; e < 2 * kW; ++e) ht[e] = (float)(ht[e] * scales[q]);
        cudaMemcpyAsync(trial, ht.data(), sizeof(float) * 2 * kW, cudaMemcpyHostToDevice, st);
        double rho = INFINITY;
        s = mg_convergence(g, a, &learned, jc, tp->seed + 99, &rho, st);
        if (s == EW_OK && std::isfinite(rho) && rho < rho_learned) {
            rho_learned = rho;
            hbest = ht;
        }
    }
    int accepted = s == EW_OK && std::isfinite(rho_learned) && rho_learned < rho_plain;
    if (accepted) cudaMemcpyAsync(weights, hbest.data(), sizeof(float) * 2 * kW, cudaMemcpyHostToDevice, st);
    if (s == EW_OK && !accepted)  // plain multigrid stays: hand back the initial weights
        cudaMemcpyAsync(weights, best, sizeof(float) * 2 * kW, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    if (rep) {
        rep->loss_first = loss_first;
        rep->loss_last = loss_last;
        rep->conv_plain = rho_plain;
        rep->conv_learned = rho_learned;
        rep->accepted = accepted;
    }
    return s;
} catch (...) {
    return abi_exception();
}

}  // extern "C"
