// ew_tb2d.cu -- temporally blocked fused leapfrog + filter step for 2D grids.
//
// One launch advances every active point by b <= B time steps
// (eq. explicitScheme) and adds c_{n+1} W^{n+1} + ... + c_{n+b} W^{n+b} to the
// filter sum (eq. filterQuadrature) without leaving shared memory.
//
// Tiling.  A CTA owns a TX x TY tile.  It stages D^n = W^n - W^{n-1} (the
// summed form of the recurrence, see ew_stencil.cu) and W^n over the tile
// plus a halo of H = R B points (R = stencil radius: 1 for order 2, 2 for
// order 4) in two shared-memory buffers, and updates the fixed "compute
// region" (the staged region minus an R-wide rim) B times.  Each step the
// valid part of the region shrinks by R, so after b steps the owned tile is
// exact; halo points are recomputed by several CTAs but only owned points are
// accumulated and stored.  D^{n+b}, W^{n+b} go to a second pair of global
// buffers because neighbouring CTAs still read the first pair.
//
// Threads.  A warp covers 32 consecutive columns of the compute region and
// each thread a column segment of KY rows, held as a sliding register window
// along y, so a point costs five shared-memory loads (centre column entry,
// x +- 1, x +- 2) and one store per step (D^n stays in registers), and the step needs
// one barrier.
//
// Boundary conditions without branches.  Points of the staged region outside
// the box are loaded with the box closure's extension of the grid function
// (ew_bc_dev.cuh: beyond a Dirichlet face zero on the wall and -u(mirror)
// further out, beyond a Neumann face +u(mirror); applied per axis and
// periodically for tiny boxes).  The update is linear, uses the same
// instruction sequence at every point and forms every neighbour sum as a
// (left + right) pair, which a mirror only swaps; IEEE addition is commutative
// and negation exact, so the updated values stay the exact extension: the
// Dirichlet walls stay 0 and the ghosts stay -u(mirror) or u(mirror), with no
// fix-up pass.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "ew_internal.h"
#include "ew_tb2d_dev.cuh"

namespace ew {

// ---------------------------------------------------------------------------
// variant table
// ---------------------------------------------------------------------------
struct Tb2dVariant {
    int nwx, nty, ky, B;
    int TX, TY, threads;
    size_t smem;
    void* fn;  // kernel pointer, boxes with Dirichlet faces only
    void* fn_gen;  // the same kernel for any faces (see ext2 in ew_tb2d_dev.cuh)
    int minb, fence;
    int kind = 0;  // 0: shared-memory form (k_step_tb2d), 1: register-blocked persistent form (k_step_rb2d),
                   // 2: TMA-staged persistent form (k_step_tma2d, padded field pitch)
    int rb = -1;   // index into rb2d_variants(R) for kind 1, into tma2d_variants(R) for kind 2
};

// FP32 lists also carry the register-blocked forms; the autotuner picks among all
static std::vector<Tb2dVariant> with_rb2d(std::vector<Tb2dVariant> v, int R) {
    const auto& rb = rb2d_variants(R);
    for (size_t i = 0; i < rb.size(); ++i) {
        Tb2dVariant x{1, rb[i].nty, rb[i].ky, rb[i].B, rb[i].TX, rb[i].TY, rb[i].threads, rb[i].smem, rb[i].fn,
                      rb[i].fn_gen, 1, 0};
        x.kind = 1;
        x.rb = (int)i;
        v.push_back(x);
    }
    return v;
}

// FP32 lists also carry the TMA-staged forms
static std::vector<Tb2dVariant> with_tma2d(std::vector<Tb2dVariant> v, int R) {
    const auto& tm = tma2d_variants(R);
    for (size_t i = 0; i < tm.size(); ++i) {
        Tb2dVariant x{tm[i].nwx, tm[i].nty, tm[i].ky, tm[i].B, tm[i].TX, tm[i].TY, tm[i].threads, tm[i].smem, tm[i].fn,
                      tm[i].fn_gen, 1, 0};
        x.kind = 2;
        x.rb = (int)i;
        v.push_back(x);
    }
    return v;
}

#define EW_TB2D_VARIANT(T, R, NWX, NTY, KY, B, MINB)                                                  \
    Tb2dVariant {                                                                                     \
        NWX, NTY, KY, B, Tb2dShape<T, R, NWX, NTY, KY, B>::TX, Tb2dShape<T, R, NWX, NTY, KY, B>::TY,  \
            Tb2dShape<T, R, NWX, NTY, KY, B>::NT, Tb2dShape<T, R, NWX, NTY, KY, B>::SMEM,              \
            (void*)k_step_tb2d<T, R, NWX, NTY, KY, B, MINB, false>,                                   \
            (void*)k_step_tb2d<T, R, NWX, NTY, KY, B, MINB, true>, MINB, 0                             \
    }

template <typename T, int R>
static const std::vector<Tb2dVariant>& tb2d_variants();

// Index 0 of each list is the default used when the caller fixes the depth.
template <>
const std::vector<Tb2dVariant>& tb2d_variants<float, 2>() {
    static const std::vector<Tb2dVariant> v = with_tma2d(with_rb2d({
        EW_TB2D_VARIANT(float, 2, 2, 8, 8, 4, 2),  EW_TB2D_VARIANT(float, 2, 2, 8, 8, 2, 2),
        EW_TB2D_VARIANT(float, 2, 2, 8, 8, 3, 2),  EW_TB2D_VARIANT(float, 2, 2, 16, 8, 4, 1),
        EW_TB2D_VARIANT(float, 2, 2, 16, 8, 6, 1), EW_TB2D_VARIANT(float, 2, 2, 4, 16, 4, 2),
        EW_TB2D_VARIANT(float, 2, 4, 4, 8, 4, 2),  EW_TB2D_VARIANT(float, 2, 2, 8, 12, 4, 1),
        EW_TB2D_VARIANT(float, 2, 2, 16, 8, 8, 1), EW_TB2D_VARIANT(float, 2, 1, 16, 8, 4, 2),
        // depths whose tile count fills whole waves of 152 SMs on common grids
        EW_TB2D_VARIANT(float, 2, 2, 16, 8, 7, 1), EW_TB2D_VARIANT(float, 2, 2, 16, 8, 5, 1),
    }, 2), 2);
    return v;
}
template <>
const std::vector<Tb2dVariant>& tb2d_variants<float, 1>() {
    static const std::vector<Tb2dVariant> v = with_tma2d(with_rb2d({
        EW_TB2D_VARIANT(float, 1, 2, 8, 8, 4, 2),  EW_TB2D_VARIANT(float, 1, 2, 8, 8, 8, 2),
        EW_TB2D_VARIANT(float, 1, 2, 8, 8, 2, 2),  EW_TB2D_VARIANT(float, 1, 2, 16, 8, 8, 1),
        EW_TB2D_VARIANT(float, 1, 2, 16, 8, 12, 1), EW_TB2D_VARIANT(float, 1, 2, 4, 16, 8, 2),
        EW_TB2D_VARIANT(float, 1, 4, 4, 8, 8, 2),
    }, 1), 1);
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

// double-FP32 pairs: ALU-bound, yet on 2047 x 3071 depths 2-3 beat depth 1 (which moves 48 B per
// point and step); the tuner picks among depths 1-5
template <>
const std::vector<Tb2dVariant>& tb2d_variants<dd, 2>() {
    static const std::vector<Tb2dVariant> v = {
        EW_TB2D_VARIANT(dd, 2, 2, 8, 8, 1, 1), EW_TB2D_VARIANT(dd, 2, 2, 8, 8, 2, 1),
        EW_TB2D_VARIANT(dd, 2, 2, 8, 8, 3, 1), EW_TB2D_VARIANT(dd, 2, 2, 4, 8, 1, 2),
        EW_TB2D_VARIANT(dd, 2, 2, 4, 8, 2, 2), EW_TB2D_VARIANT(dd, 2, 2, 8, 8, 4, 1),
        EW_TB2D_VARIANT(dd, 2, 2, 8, 8, 5, 1), EW_TB2D_VARIANT(dd, 2, 2, 4, 8, 3, 2),
        EW_TB2D_VARIANT(dd, 2, 2, 4, 8, 4, 2),
    };
    return v;
}
template <>
const std::vector<Tb2dVariant>& tb2d_variants<dd, 1>() {
    static const std::vector<Tb2dVariant> v = {
        EW_TB2D_VARIANT(dd, 1, 2, 8, 8, 1, 1), EW_TB2D_VARIANT(dd, 1, 2, 8, 8, 2, 1),
        EW_TB2D_VARIANT(dd, 1, 2, 8, 8, 4, 1), EW_TB2D_VARIANT(dd, 1, 2, 4, 8, 1, 2),
        EW_TB2D_VARIANT(dd, 1, 2, 4, 8, 2, 2),
    };
    return v;
}

template <typename T>
static const char* type_name() {
    return sizeof(T) == 4 ? "fp32" : std::is_same<T, dd>::value ? "fp32x2" : "fp64";
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
    if (var.kind == 1) {
        if constexpr (sizeof(T) == 4)
            return rb2d_launch(rb2d_variants(g.order == 2 ? 1 : 2)[(size_t)var.rb], g, Ain, Bin, Aout, Bout, acc, cw, b,
                               s, nvec, fstride, st);
        return set_error(EW_EUNSUPPORTED, "register-blocked step is FP32 only");
    }
    if (var.kind == 2) {
        if constexpr (sizeof(T) == 4)
            return tma2d_launch(tma2d_variants(g.order == 2 ? 1 : 2)[(size_t)var.rb], g, Ain, Bin, Aout, Bout, acc, cw,
                                b, s, nvec, fstride, st);
        return set_error(EW_EUNSUPPORTED, "TMA-staged step is FP32 only");
    }
    void* fn = g.bc ? var.fn_gen : var.fn;
    {
        // raise the dynamic shared-memory limit once per kernel and device
        static std::map<std::pair<void*, int>, bool> done;
        int dev = 0;
        EW_CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(g_attr_mu);
        auto key = std::make_pair(fn, dev);
        if (!done.count(key)) {
            EW_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)var.smem));
            done[key] = true;
        }
    }
    int nx = (int)g.n[0], ny = (int)g.n[1];
    dim3 grid((unsigned)((nx + var.TX - 1) / var.TX), (unsigned)((ny + var.TY - 1) / var.TY), (unsigned)nvec);
    void* args[] = {(void*)&nx, (void*)&ny, (void*)&Ain, (void*)&Bin, (void*)&Aout, (void*)&Bout,
                    (void*)&acc, (void*)&cw, (void*)&b, (void*)&s, (void*)&fstride};
    cudaEvent_t ev = fused_begin(st);
    EW_CUDA_TRY(cudaLaunchKernel(fn, grid, dim3(var.threads), args, var.smem, st));
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
    const auto& vars = variants_for<T>(g.order);
    // the register-blocked forms stage rows with 16-byte bulk copies; the
    // TMA-staged forms also need room for the padded row pitch
    const bool rb_ok = sizeof(T) == 4 && fstride % 4 == 0 &&
                       (((uintptr_t)F[0] | (uintptr_t)F[1] | (uintptr_t)F[2] | (uintptr_t)F[3]) & 15) == 0;
    const bool tma_ok = rb_ok && g.dim == 2 && fstride >= pitch2d(g.n[0]) * g.n[1];
    auto usable = [&](const Tb2dVariant& v) { return v.kind == 0 || (v.kind == 1 && rb_ok) || (v.kind == 2 && tma_ok); };
    // EW_TB2D_VARIANT=i fixes the variant (index into this precision's and
    // order's list) instead of timing them, "rb:i" / "tma:i" the i-th
    // register-blocked / TMA-staged one: a tuning and testing override
    if (const char* fv = getenv("EW_TB2D_VARIANT")) {
        int kind = 0;
        const char* num = fv;
        if (!strncmp(fv, "rb:", 3)) kind = 1, num = fv + 3;
        if (!strncmp(fv, "tma:", 4)) kind = 2, num = fv + 4;
        int i = atoi(num);
        if (kind) {  // the i-th entry of that kind
            int k = -1;
            for (size_t j = 0; j < vars.size() && k < 0; ++j)
                if (vars[j].kind == kind && i-- == 0) k = (int)j;
            i = k;
        }
        if (i < 0 || i >= (int)vars.size() || !usable(vars[(size_t)i]))
            return set_error(EW_EINVAL, "EW_TB2D_VARIANT: no such variant for this grid");
        *out = i;
        return EW_OK;
    }
    int dev = 0;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    TuneKey key{g.n[0], g.n[1], g.order, MantBits<T>::value, nvec, dev};
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
    ProfilePause pause;  // tuning launches are not counted
    EventPair ev;
    EW_TRY(ev.create());
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    int best = 0;
    double best_rate = -1.0;
    ew_status status = EW_OK;
    for (size_t i = 0; i < vars.size() && status == EW_OK; ++i) {
        const auto& var = vars[i];
        if (!usable(var)) continue;
        int b = var.B;
        // one warm launch, then three timed ones
        for (int rep = 0; rep < 4 && status == EW_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            status = launch_variant<T>(var, g, F[0], F[1], F[2], F[3], acc, cw, b, s, nvec, fstride, st);
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        if (status == EW_OK && var.kind == 1) status = rb2d_check_timeout();
        if (status == EW_OK && var.kind == 2) status = tma2d_check_timeout();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        double rate = (double)b * 3.0 / std::max(ms, 1e-6f);  // time steps per ms
        if (getenv("EW_TUNE_LOG"))
            fprintf(stderr, "[ew tune] %lldx%lld order %d %s: variant %zu (warps %dx%d, rows %d, depth %d, "
                            "minb %d, fence %d, tile %dx%d)%s: %.4f ms/step\n",
                    (long long)g.n[0], (long long)g.n[1], g.order, type_name<T>(), i, var.nwx,
                    var.nty, var.ky, var.B, var.minb, var.fence, var.TX, var.TY, var.kind == 1 ? " register-blocked" : var.kind == 2 ? " TMA-staged" : "",
                    1.0 / rate);
        if (rate > best_rate) {
            best_rate = rate;
            best = (int)i;
        }
    }
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
template ew_status tb2d_tune<dd>(const GridGeom&, const FilterPlan&, const dd*, dd* const*, dd*,
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
template ew_status tb2d_advance<dd>(const GridGeom&, const FilterPlan&, const dd*, dd* const*, int*,
                                        int*, int64_t, dd*, int, int64_t, int, cudaStream_t);

// row pitch of the time-level fields the advance will use: the padded pitch
// when the variant it runs is a TMA-staged one, nx otherwise (call after the
// tuner)
template <typename T>
int64_t tb2d_field_pitch(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, T* acc, int nvec,
                         int64_t fstride, int tb, cudaStream_t st) {
    if (g.dim != 2 || sizeof(T) != 4) return g.n[0];
    int vi = 0;
    if (tb == 0) {
        Stencil<T> s = make_stencil<T>(g, plan.dt * plan.dt);
        if (autotune<T>(g, F, acc, cdev, s, nvec, fstride, st, &vi, true) != EW_OK) return g.n[0];
    }
    return variants_for<T>(g.order)[(size_t)vi].kind == 2 ? pitch2d(g.n[0]) : g.n[0];
}
template int64_t tb2d_field_pitch<float>(const GridGeom&, const FilterPlan&, const float*, float* const*, float*, int,
                                         int64_t, int, cudaStream_t);
template int64_t tb2d_field_pitch<double>(const GridGeom&, const FilterPlan&, const double*, double* const*, double*,
                                          int, int64_t, int, cudaStream_t);
template int64_t tb2d_field_pitch<dd>(const GridGeom&, const FilterPlan&, const dd*, dd* const*, dd*, int, int64_t,
                                      int, cudaStream_t);

// description of the tuned choice (for reports)
template <typename T>
int tb2d_choice(const GridGeom& g, int nvec, int* B, int* TX, int* TY) {
    int dev = 0;
    cudaGetDevice(&dev);
    TuneKey key{g.n[0], g.n[1], g.order, MantBits<T>::value, nvec, dev};
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
template int tb2d_choice<dd>(const GridGeom&, int, int*, int*, int*);

// the tuned variant's kernel with its template shape, e.g. "k_step_tma2d<2, 2, 12, 8, 4, false>"
template <typename T>
static std::string tb2d_choice_name(const GridGeom& g, int vi) {
    const auto& v = variants_for<T>(g.order)[(size_t)vi];
    const int R = g.order == 2 ? 1 : 2;
    const char* gen = g.bc ? "true" : "false";
    char buf[160];
    if (v.kind == 2)
        snprintf(buf, sizeof buf, "k_step_tma2d<%d, %d, %d, %d, %d, %s>", R, v.nwx, v.nty, v.ky, v.B, gen);
    else if (v.kind == 1)
        snprintf(buf, sizeof buf, "k_step_rb2d<%d, %d, %d, %d, %s>", R, v.nty, v.ky, v.B, gen);
    else
        snprintf(buf, sizeof buf, "k_step_tb2d<%s, %d, %d, %d, %d, %d, %d, %s>",
                 sizeof(T) == 4 ? "float" : std::is_same<T, dd>::value ? "dd" : "double", R, v.nwx, v.nty, v.ky,
                 v.B, v.minb, gen);
    return buf;
}

}  // namespace ew

using namespace ew;

extern "C" ew_status ew_tuned_variant(const ew_grid* grid, int nvec, char* name_host, int cap, int* depth,
                                      int* tile_x, int* tile_y) try {
    clear_error();
    if (!grid || !name_host || cap < 1) return set_error(EW_EINVAL, "null argument");
    const GridGeom& g = grid->geom;
    if (g.dim != 2 || g.map) return set_error(EW_EINVAL, "not a 2D box grid");
    int B = 0, TX = 0, TY = 0, vi = -1;
    std::string name;
    if (grid->prec == EW_FP32) {
        vi = tb2d_choice<float>(g, nvec, &B, &TX, &TY);
        if (vi >= 0) name = tb2d_choice_name<float>(g, vi);
    } else if (grid->prec == EW_FP64) {
        vi = tb2d_choice<double>(g, nvec, &B, &TX, &TY);
        if (vi >= 0) name = tb2d_choice_name<double>(g, vi);
    } else {
        vi = tb2d_choice<dd>(g, nvec, &B, &TX, &TY);
        if (vi >= 0) name = tb2d_choice_name<dd>(g, vi);
    }
    if (vi < 0) return set_error(EW_EINVAL, "no wave-solve of this grid shape and nvec has been tuned");
    snprintf(name_host, (size_t)cap, "%s", name.c_str());
    if (depth) *depth = B;
    if (tile_x) *tile_x = TX;
    if (tile_y) *tile_y = TY;
    return EW_OK;
} catch (...) {
    return abi_exception();
}
