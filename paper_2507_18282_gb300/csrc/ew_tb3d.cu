// ew_tb3d.cu -- temporally blocked fused leapfrog + filter steps on 3D grids,
// second-order stencil (eqs. explicitScheme, filterQuadrature), in the summed
// form of the recurrence (see ew_stencil.cu):
//
//   D^{k} = D^{k-1} + dt^2 L_h W^{k-1},  W^{k} = W^{k-1} + D^{k},  acc += c_k W^{k}
//
// 2.5D blocking.  A CTA owns a TXo x TYo column of the box and streams it
// along z.  Its 32 x 32 threads cover the tile plus a rim of H = B points in x
// and y (one thread per (x, y)); one launch advances b <= B time levels.
// Level k works one plane behind level k-1: at step z of the march, level 0
// loads plane z of W^n and D^n, and level k (1..b) computes plane z - k from
// level k-1's planes z-k-1 .. z-k+1.  Each thread keeps, per level, the
// z-neighbours of its own column in a three-entry register queue, the D value
// it hands to the next level, and the filter sums of the last B planes; only
// the x/y neighbours go through shared memory, one double-buffered plane per
// level, and one barrier per plane serves all levels.  Level b writes
// D^{n+b}, W^{n+b} and the finished filter sum of plane z - b for the owned
// points.  Wrong x/y neighbours at the region's edge spread one point per
// level and stay inside the rim.
//
// Points outside the box (x, y or z) are loaded with the box closure's
// extension of the field (ew_bc_dev.cuh: 0 on a Dirichlet wall, -u(mirror)
// beyond it, +u(mirror) beyond a Neumann face); the update keeps it exact, as
// in the 2D kernel, so planes beyond the box are simply computed.
// Global traffic per point and launch: W^n, D^n, acc in, W^{n+b}, D^{n+b}, acc
// out (24 B in FP32), i.e. 24/b B per cell-step.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "ew_bc_dev.cuh"
#include "ew_internal.h"
#include "ew_tb2d_dev.cuh"  // p_add, p_mul, p_fma, s_add

namespace ew {

constexpr int kT3 = 32;  // compute region edge (threads per axis)

// FULL: b == B (every launch but the last of a wave-solve)
template <typename T, int B, bool FULL>
__global__ void __launch_bounds__(kT3* kT3, 1)
    k_step_tb3d(int nx, int ny, int nz, const T* __restrict__ Din, const T* __restrict__ Win, T* __restrict__ Dout,
                T* __restrict__ Wout, T* __restrict__ acc, const T* __restrict__ cw, int b, Stencil<T> st,
                int64_t fstride) {
    constexpr int H = B, TO = kT3 - 2 * H;  // rim, owned tile edge
    extern __shared__ __align__(16) unsigned char smem_tb3d[];
    // sP[k][buf]: level k's output plane (k = 0: the loaded W^n), double-buffered
    T(*sP)[2][kT3 * kT3] = reinterpret_cast<T(*)[2][kT3 * kT3]>(smem_tb3d);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = blockIdx.x * TO - H + tx, gy = blockIdx.y * TO - H + ty;
    const int64_t v = blockIdx.z;
    const int64_t N = (int64_t)nx * ny * nz, plane = (int64_t)nx * ny;
    Din += v * fstride;
    Win += v * fstride;
    Dout += v * fstride;
    Wout += v * fstride;
    acc += v * N;
    // x/y extension of this column: source column and sign (0: a Dirichlet wall)
    int sx = 1, sy = 1;
    const int ix = ext_axis<int>(gx, nx, axis_bc(st.bc, 0), sx), iy = ext_axis<int>(gy, ny, axis_bc(st.bc, 1), sy);
    const int sxy = (ix < 0 || iy < 0) ? 0 : sx * sy;
    const int64_t col = sxy ? (int64_t)iy * nx + ix : 0;
    const bool own = tx >= H && tx < H + TO && ty >= H && ty < H + TO && gx < nx && gy < ny;
    const int64_t ocol = (int64_t)gy * nx + gx;
    // neighbours inside the region (clamped at its edge: those values are wrong but stay in the rim)
    const int ixm = max(tx - 1, 0), ixp = min(tx + 1, kT3 - 1), iym = max(ty - 1, 0), iyp = min(ty + 1, kT3 - 1);
    const int me = ty * kT3 + tx;
    const int nxm = ty * kT3 + ixm, nxp = ty * kT3 + ixp, nym = iym * kT3 + tx, nyp = iyp * kT3 + tx;

    // plane z's inputs are loaded kPF steps ahead into slot z mod kPF, raw, with
    // the extension's sign kept beside them (applying it at load time would
    // make the warp wait for the load right away); the march is unrolled by kPF
    // so every slot is a fixed register
    constexpr int kPF = 4;
    T pw[kPF], pd[kPF], pa[kPF], sg[kPF];
    auto issue = [&](int z, T& w, T& d, T& a, T& sgn) {
        int szz = 1, iz = z;
        if (z < 0 || z >= nz) iz = ext_axis<int>(z, nz, axis_bc(st.bc, 2), szz);
        const bool live = sxy != 0 && iz >= 0 && z < nz + B;
        const int64_t gi = (int64_t)(live ? iz : 0) * plane + col;
        w = T(0);
        d = T(0);
        a = T(0);
        if (live) {
            w = Win[gi];
            d = Din[gi];
        }
        if (own && z >= 0 && z < nz) a = acc[(int64_t)z * plane + ocol];
        sgn = live ? T(sxy * szz) : T(0);
    };
#pragma unroll
    for (int q = 0; q < kPF; ++q) issue(-B + q, pw[q], pd[q], pa[q], sg[q]);

    T Wq[B + 1][3];  // Wq[k]: W of level k-1 at planes p_k - 1, p_k, p_k + 1 (k = 1..B)
    T Dq[B + 1];     // Dq[k]: D of level k-1 at plane p_k
    T accq[B];       // accq[j]: filter sum of plane z - 1 - j
    T cwr[B];        // filter weights of the b levels
#pragma unroll
    for (int k = 0; k <= B; ++k) {
        Wq[k][0] = Wq[k][1] = Wq[k][2] = T(0);
        Dq[k] = T(0);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
        accq[j] = T(0);
        cwr[j] = (FULL || j < b) ? cw[j] : T(0);
    }
    const T c0 = st.c0, c1x = st.c1[0], c1y = st.c1[1], c1z = st.c1[2];
    const int nb = FULL ? B : b;

    for (int zb = -B; zb < nz + B; zb += kPF) {
#pragma unroll
        for (int j = 0; j < kPF; ++j) {
            const int z = zb + j;
            if (z >= nz + B) break;
            const int buf = z & 1, obuf = buf ^ 1;
            // ---- level 0: plane z of W^n, D^n and its filter sum (loaded kPF steps ago) -
            const T w0 = sg[j] * pw[j], d0 = sg[j] * pd[j], a0 = pa[j];
            issue(z + kPF, pw[j], pd[j], pa[j], sg[j]);
            sP[0][buf][me] = w0;
            T dnext = d0;  // D handed from level k-1 to level k (this step's plane p_{k-1})
            T wnext = w0;  // W of level k-1 at plane p_{k-1} = p_k + 1
            // ---- levels 1..b -----------------------------------------------------------
#pragma unroll
            for (int k = 1; k <= B; ++k) {
                if (!FULL && k > nb) break;
                // z-queue of level k-1 around plane p_k = z - k
                Wq[k][0] = Wq[k][1];
                Wq[k][1] = Wq[k][2];
                Wq[k][2] = wnext;
                const T* sq = sP[k - 1][obuf];  // level k-1's plane p_k, written one step ago
                const T u = Wq[k][1];
                T lap = c0 * u;
                lap += c1x * (sq[nxm] + sq[nxp]);
                lap += c1y * (sq[nym] + sq[nyp]);
                lap += c1z * (Wq[k][0] + Wq[k][2]);
                const T d = Dq[k] + lap;
                const T wn = u + d;
                Dq[k] = dnext;  // level k-1's D of plane p_k + 1, used by level k next step
                accq[k - 1] += cwr[k - 1] * wn;
                if (k < nb) {
                    sP[k][buf][me] = wn;
                    dnext = d;
                    wnext = wn;
                } else {
                    const int p = z - k;
                    if (own && p >= 0 && p < nz) {
                        const int64_t gi = (int64_t)p * plane + ocol;
                        Wout[gi] = wn;
                        Dout[gi] = d;
                    }
                }
            }
            // ---- plane z - b is complete: store its filter sum, shift the queue ---------
            {
                const int p = z - nb;
                if (own && p >= 0 && p < nz) acc[(int64_t)p * plane + ocol] = accq[nb - 1];
#pragma unroll
                for (int q = B - 1; q > 0; --q) accq[q] = accq[q - 1];
                accq[0] = a0;
            }
            __syncthreads();
        }
    }
}

// FP32 form of the same march: 16 x 32 threads, each with two adjacent columns
// of the 32 x 32 region, so every level's update runs in paired FP32
// instructions (f32x2 multiply-add and add) and the shared-memory neighbours
// come in 8-byte pairs: (x-2, x-1) and (x+2, x+3) beside the thread's own pair,
// the rows above and below as pairs.  The operations of a level and their
// order are those of the scalar kernel above, so both give the same values.
// Measured reason: the scalar kernel issues an instruction on 80 % of the
// cycles (ncu, 511^3), so it is bound by its instruction count, which pairing
// roughly halves.
template <int B, bool FULL>
__global__ void __launch_bounds__(kT3* kT3 / 2, 1)
    k_step_tb3d_f2(int nx, int ny, int nz, const float* __restrict__ Din, const float* __restrict__ Win,
                   float* __restrict__ Dout, float* __restrict__ Wout, float* __restrict__ acc,
                   const float* __restrict__ cw, int b, Stencil<float> st, int64_t fstride) {
    constexpr int H = B, TO = kT3 - 2 * H;
    extern __shared__ __align__(16) unsigned char smem_tb3d[];
    float(*sP)[2][kT3 * kT3] = reinterpret_cast<float(*)[2][kT3 * kT3]>(smem_tb3d);
    const int c = 2 * threadIdx.x, ty = threadIdx.y;  // columns c, c + 1 of the region, row ty
    const int gxa = blockIdx.x * TO - H + c, gy = blockIdx.y * TO - H + ty;
    const int64_t v = blockIdx.z;
    const int64_t N = (int64_t)nx * ny * nz, plane = (int64_t)nx * ny;
    Din += v * fstride;
    Win += v * fstride;
    Dout += v * fstride;
    Wout += v * fstride;
    acc += v * N;
    // x/y extension of each column: source column and sign (0: a Dirichlet wall)
    int sxa = 1, sxb = 1, sy = 1;
    const int iy = ext_axis<int>(gy, ny, axis_bc(st.bc, 1), sy);
    const int ixa = ext_axis<int>(gxa, nx, axis_bc(st.bc, 0), sxa);
    const int ixb = ext_axis<int>(gxa + 1, nx, axis_bc(st.bc, 0), sxb);
    const int sga = (ixa < 0 || iy < 0) ? 0 : sxa * sy, sgb = (ixb < 0 || iy < 0) ? 0 : sxb * sy;
    const int64_t cola = sga ? (int64_t)iy * nx + ixa : 0, colb = sgb ? (int64_t)iy * nx + ixb : 0;
    const bool rowown = ty >= H && ty < H + TO && gy < ny;
    const bool owna = rowown && c >= H && c < H + TO && gxa < nx;
    const bool ownb = rowown && c + 1 >= H && c + 1 < H + TO && gxa + 1 < nx;
    const int64_t ocol = (int64_t)gy * nx + gxa;  // column a's point of a plane (b: + 1)
    // neighbour pairs inside the region (clamped at its edge: those values are wrong but stay in the rim)
    const int me = ty * kT3 + c;
    const int nxm = ty * kT3 + max(c - 2, 0), nxp = ty * kT3 + min(c + 2, kT3 - 2);
    const int nym = max(ty - 1, 0) * kT3 + c, nyp = min(ty + 1, kT3 - 1) * kT3 + c;

    constexpr int kPF = 4;
    float2 pw[kPF], pd[kPF], pa[kPF], sg[kPF];
    auto issue = [&](int z, float2& w, float2& d, float2& a, float2& sgn) {
        int szz = 1, iz = z;
        if (z < 0 || z >= nz) iz = ext_axis<int>(z, nz, axis_bc(st.bc, 2), szz);
        const bool zl = iz >= 0 && z < nz + B;
        const int64_t zb = (int64_t)(zl ? iz : 0) * plane;
        const bool la = zl && sga != 0, lb = zl && sgb != 0;
        w = make_float2(0.f, 0.f);
        d = make_float2(0.f, 0.f);
        a = make_float2(0.f, 0.f);
        if (la) {
            w.x = Win[zb + cola];
            d.x = Din[zb + cola];
        }
        if (lb) {
            w.y = Win[zb + colb];
            d.y = Din[zb + colb];
        }
        if (z >= 0 && z < nz) {
            const int64_t q = (int64_t)z * plane + ocol;
            if (owna) a.x = acc[q];
            if (ownb) a.y = acc[q + 1];
        }
        sgn = make_float2(la ? (float)(sga * szz) : 0.f, lb ? (float)(sgb * szz) : 0.f);
    };
#pragma unroll
    for (int q = 0; q < kPF; ++q) issue(-B + q, pw[q], pd[q], pa[q], sg[q]);

    float2 Wq[B + 1][3];
    float2 Dq[B + 1];
    float2 accq[B];
    float2 cwr[B];
#pragma unroll
    for (int k = 0; k <= B; ++k) {
        Wq[k][0] = Wq[k][1] = Wq[k][2] = make_float2(0.f, 0.f);
        Dq[k] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
        accq[j] = make_float2(0.f, 0.f);
        const float w = (FULL || j < b) ? cw[j] : 0.f;
        cwr[j] = make_float2(w, w);
    }
    const float2 C0 = make_float2(st.c0, st.c0), C1X = make_float2(st.c1[0], st.c1[0]);
    const float2 C1Y = make_float2(st.c1[1], st.c1[1]), C1Z = make_float2(st.c1[2], st.c1[2]);
    const int nb = FULL ? B : b;

    for (int zb = -B; zb < nz + B; zb += kPF) {
#pragma unroll
        for (int j = 0; j < kPF; ++j) {
            const int z = zb + j;
            if (z >= nz + B) break;
            const int buf = z & 1, obuf = buf ^ 1;
            const float2 w0 = p_mul(sg[j], pw[j]), d0 = p_mul(sg[j], pd[j]), a0 = pa[j];
            issue(z + kPF, pw[j], pd[j], pa[j], sg[j]);
            *reinterpret_cast<float2*>(&sP[0][buf][me]) = w0;
            float2 dnext = d0;
            float2 wnext = w0;
#pragma unroll
            for (int k = 1; k <= B; ++k) {
                if (!FULL && k > nb) break;
                Wq[k][0] = Wq[k][1];
                Wq[k][1] = Wq[k][2];
                Wq[k][2] = wnext;
                const float* sq = sP[k - 1][obuf];
                const float2 u = Wq[k][1];
                const float2 L = *reinterpret_cast<const float2*>(sq + nxm);  // columns c - 2, c - 1
                const float2 Q = *reinterpret_cast<const float2*>(sq + nxp);  // columns c + 2, c + 3
                const float2 YM = *reinterpret_cast<const float2*>(sq + nym);
                const float2 YP = *reinterpret_cast<const float2*>(sq + nyp);
                float2 sx1;
                sx1.x = s_add(L.y, u.y);  // column c: (c - 1) + (c + 1)
                sx1.y = s_add(u.x, Q.x);  // column c + 1: c + (c + 2)
                float2 lap = p_mul(C0, u);
                lap = p_fma(C1X, sx1, lap);
                lap = p_fma(C1Y, p_add(YM, YP), lap);
                lap = p_fma(C1Z, p_add(Wq[k][0], Wq[k][2]), lap);
                const float2 d = p_add(Dq[k], lap);
                const float2 wn = p_add(u, d);
                Dq[k] = dnext;
                accq[k - 1] = p_fma(cwr[k - 1], wn, accq[k - 1]);
                if (k < nb) {
                    *reinterpret_cast<float2*>(&sP[k][buf][me]) = wn;
                    dnext = d;
                    wnext = wn;
                } else {
                    const int p = z - k;
                    if (p >= 0 && p < nz) {
                        const int64_t gi = (int64_t)p * plane + ocol;
                        if (owna) {
                            Wout[gi] = wn.x;
                            Dout[gi] = d.x;
                        }
                        if (ownb) {
                            Wout[gi + 1] = wn.y;
                            Dout[gi + 1] = d.y;
                        }
                    }
                }
            }
            {
                const int p = z - nb;
                if (p >= 0 && p < nz) {
                    const int64_t q = (int64_t)p * plane + ocol;
                    if (owna) acc[q] = accq[nb - 1].x;
                    if (ownb) acc[q + 1] = accq[nb - 1].y;
                }
#pragma unroll
                for (int q = B - 1; q > 0; --q) accq[q] = accq[q - 1];
                accq[0] = a0;
            }
            __syncthreads();
        }
    }
}

template <typename T, int B>
static ew_status launch_tb3d(const GridGeom& g, const T* Din, const T* Win, T* Dout, T* Wout, T* acc, const T* cw,
                             int b, const Stencil<T>& s, int nvec, int64_t fstride, cudaStream_t st) {
    constexpr int TO = kT3 - 2 * B;
    constexpr size_t smem = sizeof(T) * (size_t)B * 2 * kT3 * kT3;
    static bool attr = false;  // per instantiation (same value on every device)
    if (!attr) {
        const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if constexpr (sizeof(T) == 4) {
            EW_CUDA_TRY(cudaFuncSetAttribute(k_step_tb3d_f2<B, true>, A, (int)smem));
            EW_CUDA_TRY(cudaFuncSetAttribute(k_step_tb3d_f2<B, false>, A, (int)smem));
        } else {
            EW_CUDA_TRY(cudaFuncSetAttribute(k_step_tb3d<T, B, true>, A, (int)smem));
            EW_CUDA_TRY(cudaFuncSetAttribute(k_step_tb3d<T, B, false>, A, (int)smem));
        }
        attr = true;
    }
    dim3 grid((unsigned)((g.n[0] + TO - 1) / TO), (unsigned)((g.n[1] + TO - 1) / TO), (unsigned)nvec);
    cudaEvent_t ev = fused_begin(st);
    if constexpr (sizeof(T) == 4) {
        auto kern = b == B ? k_step_tb3d_f2<B, true> : k_step_tb3d_f2<B, false>;
        kern<<<grid, dim3(kT3 / 2, kT3), smem, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], Din, Win, Dout, Wout,
                                                     acc, cw, b, s, fstride);
    } else {
        auto kern = b == B ? k_step_tb3d<T, B, true> : k_step_tb3d<T, B, false>;
        kern<<<grid, dim3(kT3, kT3), smem, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], Din, Win, Dout, Wout,
                                                 acc, cw, b, s, fstride);
    }
    EW_CUDA_TRY(cudaGetLastError());
    fused_end(ev, st, g.N * nvec, g.N * nvec * b);
    return EW_OK;
}

template <typename T>
static ew_status launch_depth(int B, const GridGeom& g, const T* Din, const T* Win, T* Dout, T* Wout, T* acc,
                              const T* cw, int b, const Stencil<T>& s, int nvec, int64_t fstride, cudaStream_t st) {
    if (B == 4) return launch_tb3d<T, 4>(g, Din, Win, Dout, Wout, acc, cw, b, s, nvec, fstride, st);
    if (B == 3) return launch_tb3d<T, 3>(g, Din, Win, Dout, Wout, acc, cw, b, s, nvec, fstride, st);
    return launch_tb3d<T, 2>(g, Din, Win, Dout, Wout, acc, cw, b, s, nvec, fstride, st);
}

// depth autotuner: times depths 2..4 on the caller's buffers (before the real
// wave-solve overwrites them) and caches the fastest per grid shape
using Tb3dKey = std::tuple<int64_t, int64_t, int64_t, int, int, int>;  // nx, ny, nz, elem, nvec, device
static std::map<Tb3dKey, int> g_tb3d_cache;
static std::mutex g_tb3d_mu;

template <typename T>
ew_status tb3d_tune(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, T* acc, int nvec,
                    int64_t fstride, cudaStream_t st) {
    if (g.dim != 3 || g.order != 2) return EW_OK;
    int dev = 0;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    Tb3dKey key{g.n[0], g.n[1], g.n[2], (int)sizeof(T), nvec, dev};
    {
        std::lock_guard<std::mutex> lk(g_tb3d_mu);
        if (g_tb3d_cache.count(key)) return EW_OK;
    }
    Stencil<T> s = make_stencil<T>(g, plan.dt * plan.dt);
    ProfilePause pause;  // tuning launches are not counted
    EventPair ev;
    EW_TRY(ev.create());
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    int best = 4;
    double best_rate = -1.0;
    ew_status status = EW_OK;
    for (int B = 2; B <= 4 && status == EW_OK; ++B) {
        for (int rep = 0; rep < 3 && status == EW_OK; ++rep) {  // one warm launch, two timed
            if (rep == 1) cudaEventRecord(e0, st);
            status = launch_depth<T>(B, g, F[0], F[1], F[2], F[3], acc, cdev, B, s, nvec, fstride, st);
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = 2.0 * B / std::max(ms, 1e-6f);  // time steps per ms
        if (getenv("EW_TUNE_LOG"))
            fprintf(stderr, "[ew tune] %lldx%lldx%lld 3D order 2 %s: depth %d: %.4f ms/step\n", (long long)g.n[0],
                    (long long)g.n[1], (long long)g.n[2], sizeof(T) == 4 ? "fp32" : "fp64", B, 1.0 / rate);
        if (rate > best_rate) {
            best_rate = rate;
            best = B;
        }
    }
    EW_TRY(status);
    std::lock_guard<std::mutex> lk(g_tb3d_mu);
    g_tb3d_cache[key] = best;
    return EW_OK;
}
template ew_status tb3d_tune<float>(const GridGeom&, const FilterPlan&, const float*, float* const*, float*, int,
                                    int64_t, cudaStream_t);
template ew_status tb3d_tune<double>(const GridGeom&, const FilterPlan&, const double*, double* const*, double*, int,
                                     int64_t, cudaStream_t);

// Advance from level L (W = F[cur], D = F[prv]) to level Nt in launches of up
// to B levels (the tuned depth, 4 before tuning, or `tb` when 1 < tb <= 4).
// Second-order 3D grids only.
template <typename T>
ew_status tb3d_advance(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, int* prv, int* cur,
                       int64_t L, T* acc, int nvec, int64_t fstride, int tb, cudaStream_t st) {
    if (g.dim != 3 || g.order != 2) return set_error(EW_EUNSUPPORTED, "3D temporal blocking is second order only");
    if (nvec > 65535) return set_error(EW_EUNSUPPORTED, "too many vectors in one call");
    Stencil<T> s = make_stencil<T>(g, plan.dt * plan.dt);
    int B = 4;
    if (tb > 1) {
        B = std::min(tb, 4);
    } else {
        int dev = 0;
        EW_CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(g_tb3d_mu);
        auto it = g_tb3d_cache.find(Tb3dKey{g.n[0], g.n[1], g.n[2], (int)sizeof(T), nvec, dev});
        if (it != g_tb3d_cache.end()) B = it->second;
    }
    int p = *prv, c = *cur, a = -1, d = -1;
    for (int q = 0; q < 4; ++q)
        if (q != p && q != c) (a < 0 ? a : d) = q;
    while (L < plan.Nt) {
        const int b = (int)std::min<int64_t>(B, plan.Nt - L);
        EW_TRY(launch_depth<T>(B, g, F[p], F[c], F[a], F[d], acc, cdev + L + 1, b, s, nvec, fstride, st));
        L += b;
        std::swap(p, a);
        std::swap(c, d);
    }
    *prv = p;
    *cur = c;
    return EW_OK;
}
template ew_status tb3d_advance<float>(const GridGeom&, const FilterPlan&, const float*, float* const*, int*, int*,
                                       int64_t, float*, int, int64_t, int, cudaStream_t);
template ew_status tb3d_advance<double>(const GridGeom&, const FilterPlan&, const double*, double* const*, int*, int*,
                                        int64_t, double*, int, int64_t, int, cudaStream_t);

}  // namespace ew
