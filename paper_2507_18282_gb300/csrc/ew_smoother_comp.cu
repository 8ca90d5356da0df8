// ew_smoother_comp.cu -- the learned smoother inside the V-cycle, applied as
// its composed stencil.
//
// The network has no activation (the smoothing step must stay linear), so
// its two 3x3x3 convolutions compose into one 5x5x5 stencil:
//   N(r)(x) = sum_c sum_{o2} W2[c][o2] h_c(x + o2),  h_c(y) = sum_{o1} W1[c][o1] r(y + o1)
//           = sum_d K(d) r(x + d),   K(d) = sum_c sum_{o1 + o2 = d} W2[c][o2] W1[c][o1],
// with one exception at the walls: the hidden activations are zero outside
// the active box, so for an output point on the first or last plane of an
// axis the hidden points beyond the wall drop out of its sum.  Per axis an
// output is "low" (index 0), "high" (index n - 1), "both" (n = 1) or
// interior; each of the 4^3 classes has its own composed stencil.  The
// weights are rounded to BF16 as in the tensor-core kernels and composed in
// FP64; the stencil runs in FP32 without the BF16 rounding of the hidden
// activations (the same operator, with rounding below the two-layer form's).
//
// Why: the two-layer tensor-core forward (ew_smoother.cu) is bound by its
// im2col gather (about 420 us per application on 255^3), while the composed
// stencil is 125 multiply-adds per point with the interior weights as
// constant operands, on data staged plane by plane in shared memory.
// Training and the ABI forward/backward keep the two-layer form (the
// gradient needs the layers).
//
// Kernels: the interior stencil is applied at every output, on the residual
// zero-padded outside the box; a second launch then adds, at each output on
// a wall plane, the difference between its class's stencil and the interior
// one (one thread per wall output, about 2.3 % of the points on 255^3).  In
// the first, a CTA owns 128 x 8 output columns and kZ planes of them; a thread
// owns four consecutive x outputs of one row and streams along z, keeping the
// partial sums of the five output planes an input plane feeds in registers.
// Input planes (with a halo of 2) are staged in a double-buffered shared tile,
// one barrier per plane; the global loads of plane z + 2 are issued into
// registers before plane z + 1 is computed, so their latency is hidden.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ew_internal.h"

namespace ew {

constexpr int kCompTX = 128;  // outputs per CTA row (32 threads x 4)
constexpr int kCompTY = 8;    // rows per CTA
constexpr int kCompZMin = 16;  // fewest planes per CTA (the grid's z chunks are chosen at launch)
constexpr int kCompSX = kCompTX + 4;  // staged width (halo 2), a multiple of 4
constexpr int kCompSY = kCompTY + 4;
constexpr int kCompPlane = kCompSX * kCompSY;

struct K125 {
    float k[125];  // index (dz + 2) 25 + (dy + 2) 5 + (dx + 2)
};

// class of an output coordinate on an axis: 0 low wall, 1 interior, 2 high wall, 3 both (n = 1)
__host__ __device__ __forceinline__ int comp_class(int i, int n) {
    return n == 1 ? 3 : (i == 0 ? 0 : (i == n - 1 ? 2 : 1));
}

// x += K_int * r at every output (FP32 fields, r zero outside the box); a
// CTA owns planes [z0, z0 + zc) of its 128 x 8 columns
__global__ void __launch_bounds__(256, 4)
    k_smoother_comp(int nx, int ny, int nz, int zc, const float* __restrict__ r, float* __restrict__ x, const K125 K) {
    constexpr int kPer = (kCompPlane + 255) / 256;  // staged elements per thread and plane
    __shared__ __align__(16) float sp[2][kCompPlane];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int x0 = blockIdx.x * kCompTX, y0 = blockIdx.y * kCompTY, z0 = blockIdx.z * zc;
    const int z1 = min(nz, z0 + zc);
    const int ox = x0 + 4 * lx, oy = y0 + ly;  // first output of the thread
    const int64_t plane = (int64_t)nx * ny;
    const bool orow = oy < ny;
    // the staged elements of this thread: offset within a plane, or -1 outside the box
    int off[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int q = threadIdx.x + 256 * u;
        const int c = q % kCompSX, rr = q / kCompSX;
        const int gx = x0 - 2 + c, gy = y0 - 2 + rr;
        off[u] = (q < kCompPlane && gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? gy * nx + gx : -1;
    }
    float pre[kPer];
    auto fetch = [&](int zr) {  // global loads of input plane zr into registers
        const bool zin = zr >= 0 && zr < nz;
        const float* rp = r + (int64_t)zr * plane;
#pragma unroll
        for (int u = 0; u < kPer; ++u) pre[u] = (zin && off[u] >= 0) ? rp[off[u]] : 0.f;
    };
    auto put = [&](float* dst) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int q = threadIdx.x + 256 * u;
            if (q < kCompPlane) dst[q] = pre[u];
        }
    };
    // acc[j][i]: output plane (input plane - 2 + j), x output ox + i
    float acc[5][4];
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
    fetch(z0 - 2);
    put(sp[0]);
    fetch(z0 - 1);
    __syncthreads();
    int buf = 0;
    for (int zi = z0 - 2; zi <= z1 + 1; ++zi) {
        // x of the output plane completed in this iteration, loaded now so that
        // the plane's multiply-adds hide the latency
        const int zo = zi - 2;
        const bool ostore = zo >= z0 && zo < z1 && orow;
        float xo[4];
        float* px = x + (int64_t)zo * plane + (int64_t)oy * nx + ox;
#pragma unroll
        for (int i = 0; i < 4; ++i) xo[i] = (ostore && ox + i < nx) ? px[i] : 0.f;
        // input plane zi feeds output planes zi - 2 .. zi + 2 (acc[0] .. acc[4]) with dz = 2 - j;
        // output planes outside [z0, z1) are skipped (the same for the whole CTA)
        bool need[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) need[j] = zi - 2 + j >= z0 && zi - 2 + j < z1;
        const float* p = sp[buf] + ly * kCompSX + 4 * lx;
#pragma unroll
        for (int dy = 0; dy < 5; ++dy) {
            const float4 a = *reinterpret_cast<const float4*>(p + dy * kCompSX);
            const float4 bq = *reinterpret_cast<const float4*>(p + dy * kCompSX + 4);
            const float w[8] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w};
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                if (!need[j]) continue;
                const int dz = 2 - j;
#pragma unroll
                for (int dx = 0; dx < 5; ++dx) {
                    const float kv = K.k[(dz + 2) * 25 + dy * 5 + dx];
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[j][i] = fmaf(kv, w[i + dx], acc[j][i]);
                }
            }
        }
        // output plane zi - 2 is complete
        if (ostore) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (ox + i < nx) px[i] = xo[i] + acc[0][i];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[j][i] = acc[j + 1][i];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[4][i] = 0.f;
        // plane zi + 1 (in registers) into the other buffer: its last readers
        // (plane zi - 1) passed the previous barrier
        if (zi + 1 <= z1 + 1) put(sp[buf ^ 1]);
        __syncthreads();
        if (zi + 2 <= z1 + 1) fetch(zi + 2);
        buf ^= 1;
    }
}

// Wall outputs, in three disjoint parts: the z-wall planes (all x, y), then
// the y-wall rows of the other planes (all x), then the x-wall points of the
// remaining rows.  Each adds sum_d (K_class - K_int)(d) r(p + d).  On a wall
// axis a the difference is made of hidden offsets beyond the wall, whose taps
// reach r at offsets d_a in {-2, -1, 0} (low wall) or {0, 1, 2} (high wall),
// all outside the box but d_a = 0 (and only d_a = 0 for n = 1): so only the
// taps with d_a = 0 on some wall axis a are summed (25 on a face, 45 on an
// edge, 61 at a corner), each once.
__global__ void __launch_bounds__(256)
    k_smoother_comp_walls(int nx, int ny, int nz, const float* __restrict__ r, float* __restrict__ x,
                          const float* __restrict__ kdiff, int64_t nz_part, int64_t ny_part, int64_t nwall) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nwall) return;
    const int cyn = ny == 1 ? 1 : 2, cxn = nx == 1 ? 1 : 2;
    int gx, gy, gz;
    if (idx < nz_part) {
        const int64_t pl = (int64_t)nx * ny;
        gz = (idx / pl) ? nz - 1 : 0;
        const int64_t rem = idx % pl;
        gy = (int)(rem / nx);
        gx = (int)(rem % nx);
    } else if ((idx -= nz_part) < ny_part) {
        const int64_t per = (int64_t)cyn * nx;
        gz = 1 + (int)(idx / per);
        const int64_t rem = idx % per;
        gy = (rem / nx) ? ny - 1 : 0;
        gx = (int)(rem % nx);
    } else {
        idx -= ny_part;
        const int64_t per = (int64_t)(ny - 2) * cxn;
        gz = 1 + (int)(idx / per);
        const int64_t rem = idx % per;
        gy = 1 + (int)(rem / cxn);
        gx = (rem % cxn) ? nx - 1 : 0;
    }
    const int cz = comp_class(gz, nz), cy = comp_class(gy, ny), cx = comp_class(gx, nx);
    const bool wz = cz != 1, wy = cy != 1, wx = cx != 1;
    const float* kd = kdiff + (size_t)((cz * 4 + cy) * 4 + cx) * 125;
    const int64_t q = ((int64_t)gz * ny + gy) * nx + gx;
    float s = 0.f;
    // taps with dz = 0 (z wall)
    if (wz) {
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx)
                if (gy + dy >= 0 && gy + dy < ny && gx + dx >= 0 && gx + dx < nx)
                    s = fmaf(__ldg(kd + 50 + (dy + 2) * 5 + (dx + 2)), r[q + (int64_t)dy * nx + dx], s);
    }
    // taps with dy = 0 (y wall), dz = 0 already summed on a z wall
    if (wy) {
#pragma unroll
        for (int dz = -2; dz <= 2; ++dz)
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx)
                if (!(wz && dz == 0) && gz + dz >= 0 && gz + dz < nz && gx + dx >= 0 && gx + dx < nx)
                    s = fmaf(__ldg(kd + (dz + 2) * 25 + 10 + (dx + 2)), r[q + (int64_t)dz * ny * nx + dx], s);
    }
    // taps with dx = 0 (x wall), dz = 0 or dy = 0 already summed on those walls
    if (wx) {
#pragma unroll
        for (int dz = -2; dz <= 2; ++dz)
#pragma unroll
            for (int dy = -2; dy <= 2; ++dy)
                if (!(wz && dz == 0) && !(wy && dy == 0) && gz + dz >= 0 && gz + dz < nz && gy + dy >= 0 &&
                    gy + dy < ny)
                    s = fmaf(__ldg(kd + (dz + 2) * 25 + (dy + 2) * 5 + 2), r[q + ((int64_t)dz * ny + dy) * nx], s);
    }
    x[q] += s;
}

// round to the nearest BF16 (ties to even), as the tensor-core kernels do
static float bf16_host(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    float o;
    std::memcpy(&o, &u, 4);
    return o;
}

// the 64 class stencils of weights w (432 values [W1 8x27 | W2 8x27], taps dz slowest)
static void compose_classes(const float* w, std::vector<float>& kall) {
    double W1[8][27], W2[8][27];
    for (int c = 0; c < 8; ++c)
        for (int t = 0; t < 27; ++t) {
            W1[c][t] = bf16_host(w[c * 27 + t]);
            W2[c][t] = bf16_host(w[216 + c * 27 + t]);
        }
    kall.assign(64 * 125, 0.f);
    auto allowed = [](int cls, int o) {  // hidden offset o of an output of this class stays in the box
        if (cls == 3) return o == 0;
        if (cls == 0) return o >= 0;
        if (cls == 2) return o <= 0;
        return true;
    };
    for (int cz = 0; cz < 4; ++cz)
        for (int cy = 0; cy < 4; ++cy)
            for (int cx = 0; cx < 4; ++cx) {
                double K[125] = {0};
                for (int c = 0; c < 8; ++c)
                    for (int z2 = -1; z2 <= 1; ++z2)
                        for (int y2 = -1; y2 <= 1; ++y2)
                            for (int x2 = -1; x2 <= 1; ++x2) {
                                if (!allowed(cz, z2) || !allowed(cy, y2) || !allowed(cx, x2)) continue;
                                const double w2 = W2[c][(z2 + 1) * 9 + (y2 + 1) * 3 + (x2 + 1)];
                                for (int z1 = -1; z1 <= 1; ++z1)
                                    for (int y1 = -1; y1 <= 1; ++y1)
                                        for (int x1 = -1; x1 <= 1; ++x1) {
                                            const double w1 = W1[c][(z1 + 1) * 9 + (y1 + 1) * 3 + (x1 + 1)];
                                            K[(z1 + z2 + 2) * 25 + (y1 + y2 + 2) * 5 + (x1 + x2 + 2)] += w2 * w1;
                                        }
                            }
                float* dst = kall.data() + (size_t)((cz * 4 + cy) * 4 + cx) * 125;
                for (int q = 0; q < 125; ++q) dst[q] = (float)K[q];
            }
}

ew_status ComposedSmoother::build(const float* weights_dev, cudaStream_t st) {
    float w[432];
    EW_CUDA_TRY(cudaMemcpyAsync(w, weights_dev, sizeof(w), cudaMemcpyDeviceToHost, st));
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<float> kall;
    compose_classes(w, kall);
    const size_t ci = (size_t)((1 * 4 + 1) * 4 + 1) * 125;  // the interior class
    interior.assign(kall.begin() + ci, kall.begin() + ci + 125);
    std::vector<float> kint(interior);
    for (size_t c = 0; c < 64; ++c)  // difference stencils, K_class - K_int (rounded once from FP32 values)
        for (int q = 0; q < 125; ++q) kall[c * 125 + q] -= kint[q];
    EW_TRY(dev.alloc(sizeof(float) * kall.size()));
    EW_CUDA_TRY(cudaMemcpyAsync(dev.p, kall.data(), sizeof(float) * kall.size(), cudaMemcpyHostToDevice, st));
    // the host vector must outlive the copy
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    return EW_OK;
}

ew_status ComposedSmoother::apply(const GridGeom& g, const float* r, float* x, cudaStream_t st) const {
    if (g.dim != 3 || interior.size() != 125) return set_error(EW_EINVAL, "composed smoother: not built for a 3D grid");
    K125 K;
    std::memcpy(K.k, interior.data(), sizeof(K.k));
    const int nx = (int)g.n[0], ny = (int)g.n[1], nz = (int)g.n[2];
    // z chunks: as many as fill the resident CTA slots once (four a SM), at
    // least kCompZMin planes each (each chunk restages two planes on each side)
    int cdev = 0, nsm = 0;
    EW_CUDA_TRY(cudaGetDevice(&cdev));
    EW_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, cdev));
    const int bx = (nx + kCompTX - 1) / kCompTX, by = (ny + kCompTY - 1) / kCompTY;
    const int nzc = std::max(1, (4 * nsm) / std::max(1, bx * by));
    const int zc = std::max(std::min(kCompZMin, nz), (nz + nzc - 1) / nzc);
    dim3 grid((unsigned)bx, (unsigned)by, (unsigned)((nz + zc - 1) / zc));
    k_smoother_comp<<<grid, 256, 0, st>>>(nx, ny, nz, zc, r, x, K);
    EW_CUDA_TRY(cudaGetLastError());
    const int64_t nz_part = (int64_t)(nz == 1 ? 1 : 2) * nx * ny;
    const int64_t ny_part = (int64_t)std::max(nz - 2, 0) * (ny == 1 ? 1 : 2) * nx;
    const int64_t nx_part = (int64_t)std::max(nz - 2, 0) * std::max(ny - 2, 0) * (nx == 1 ? 1 : 2);
    const int64_t nwall = nz_part + ny_part + nx_part;
    k_smoother_comp_walls<<<(unsigned)((nwall + 255) / 256), 256, 0, st>>>(nx, ny, nz, r, x, dev.as<float>(), nz_part,
                                                                          ny_part, nwall);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch(2);
    return EW_OK;
}

}  // namespace ew
