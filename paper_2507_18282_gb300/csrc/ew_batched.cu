// ew_batched.cu -- many independent 2D wave-solves (uneven boxes, each with
// its own omega, time step, N_t and filter weights) advanced together.
//
// Work queue.  Time is cut into rounds of up to B steps.  In round r every
// problem that still has steps left contributes all its tiles, each a work
// item (problem descriptor, tile index); one persistent launch per round runs
// the items with a grid-stride loop (one tile = the temporally blocked tile
// step of ew_tb2d_dev.cuh, same arithmetic per point as the single-grid path,
// so results are bit-identical to it).  A problem's descriptor for round r
// holds its ping-pong buffers, its weights c_{L+1..L+b} and its own b.  The
// first steps and every round are captured in one CUDA graph and replayed on
// the caller's stream; the tile shape and depth are chosen by timing one
// round of each candidate (autotuner), cached per batch shape.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ew_internal.h"
#include "ew_tb2d_dev.cuh"

namespace ew {

template <typename T>
ew_status first_step(const GridGeom& g, const T* vin, T* D1, T* W1, T* vout, const FilterPlan& plan, int nvec,
                     int64_t fstride, cudaStream_t st);

template <typename T>
struct BatchDesc {
    const T* Ain;
    const T* Bin;
    T* Aout;
    T* Bout;
    T* acc;
    const T* cw;
    int nx, ny, b, ntx;
    Stencil<T> st;
};

struct BatchItem {
    int desc;
    int tile;
};

template <typename T, int R, int NWX, int NTY, int KY, int B, int MINB, bool GEN>
__global__ void __launch_bounds__(32 * NWX * NTY, MINB)
    k_step_tb2d_batched(const BatchDesc<T>* __restrict__ descs, const BatchItem* __restrict__ items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchDesc<T> d = descs[w.desc];
        tb2d_tile<T, R, NWX, NTY, KY, B, GEN>(d.nx, d.ny, d.Ain, d.Bin, d.Aout, d.Bout, d.acc, d.cw, d.b, d.st,
                                         w.tile % d.ntx, w.tile / d.ntx);
        __syncthreads();  // the next item restages the shared buffers
    }
}

struct BVariant {
    int B, TX, TY, threads;
    size_t smem;
    void* fn;      // boxes with Dirichlet faces only
    void* fn_gen;  // any faces (see ext2 in ew_tb2d_dev.cuh)
};
#define EW_BVAR(T, R, NWX, NTY, KY, B, MINB)                                                               \
    BVariant {                                                                                            \
        B, Tb2dShape<T, R, NWX, NTY, KY, B>::TX, Tb2dShape<T, R, NWX, NTY, KY, B>::TY,                    \
            Tb2dShape<T, R, NWX, NTY, KY, B>::NT, Tb2dShape<T, R, NWX, NTY, KY, B>::SMEM,                 \
            (void*)k_step_tb2d_batched<T, R, NWX, NTY, KY, B, MINB, false>,                              \
            (void*)k_step_tb2d_batched<T, R, NWX, NTY, KY, B, MINB, true>                                \
    }

template <typename T, int R>
static const std::vector<BVariant>& bvariants();
template <>
const std::vector<BVariant>& bvariants<float, 1>() {
    static const std::vector<BVariant> v = {EW_BVAR(float, 1, 2, 8, 8, 4, 2),   EW_BVAR(float, 1, 2, 8, 8, 8, 2),
                                            EW_BVAR(float, 1, 2, 16, 8, 8, 1),  EW_BVAR(float, 1, 2, 4, 16, 8, 2),
                                            EW_BVAR(float, 1, 2, 16, 8, 12, 1), EW_BVAR(float, 1, 2, 16, 8, 16, 1)};
    return v;
}
template <>
const std::vector<BVariant>& bvariants<float, 2>() {
    static const std::vector<BVariant> v = {EW_BVAR(float, 2, 2, 8, 8, 4, 2), EW_BVAR(float, 2, 2, 16, 8, 6, 1),
                                            EW_BVAR(float, 2, 2, 16, 8, 8, 1)};
    return v;
}
template <>
const std::vector<BVariant>& bvariants<double, 1>() {
    static const std::vector<BVariant> v = {EW_BVAR(double, 1, 2, 8, 8, 4, 1), EW_BVAR(double, 1, 2, 4, 8, 1, 2)};
    return v;
}
template <>
const std::vector<BVariant>& bvariants<double, 2>() {
    static const std::vector<BVariant> v = {EW_BVAR(double, 2, 2, 8, 8, 4, 1), EW_BVAR(double, 2, 2, 4, 8, 1, 2)};
    return v;
}

// process-wide batched workspace (device), one per call at a time
struct BatchCache {
    std::mutex mu;
    void* dev = nullptr;
    size_t dev_bytes = 0;
    void* host = nullptr;
    size_t host_bytes = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::map<std::vector<int64_t>, int> tune;
    std::map<void*, int> occ;
};
static BatchCache g_batch;

struct BProblem {
    GridGeom g;
    FilterPlan plan;
    const void* vin;
    void* vout;
    size_t field_off, c_off;  // element offsets in the workspace
};

template <typename T>
static ew_status run_rounds(const std::vector<BProblem>& P, const BVariant& var, T* base, int nsm, cudaStream_t cs,
                            std::vector<BatchDesc<T>>& hd, std::vector<BatchItem>& hi,
                            std::vector<std::pair<size_t, size_t>>& ranges, bool build_only, BatchDesc<T>* ddesc,
                            BatchItem* ditem, bool gen) {
    // ping-pong state per problem: fields 0..3, level L
    const int np = (int)P.size();
    std::vector<int> prv(np, 0), cur(np, 1), spa(np, 2), spb(np, 3);
    std::vector<int64_t> L(np, 1);
    for (;;) {
        size_t d0 = hd.size(), i0 = hi.size();
        for (int p = 0; p < np; ++p) {
            if (L[p] >= P[p].plan.Nt) continue;
            const GridGeom& g = P[p].g;
            T* F = base + P[p].field_off;
            BatchDesc<T> d;
            d.Ain = F + (size_t)prv[p] * g.N;
            d.Bin = F + (size_t)cur[p] * g.N;
            d.Aout = F + (size_t)spa[p] * g.N;
            d.Bout = F + (size_t)spb[p] * g.N;
            d.acc = (T*)P[p].vout;
            d.cw = base + P[p].c_off + L[p] + 1;
            d.b = (int)std::min<int64_t>(var.B, P[p].plan.Nt - L[p]);
            d.nx = (int)g.n[0];
            d.ny = (int)g.n[1];
            d.ntx = (d.nx + var.TX - 1) / var.TX;
            d.st = make_stencil<T>(g, P[p].plan.dt * P[p].plan.dt);
            int nty = (d.ny + var.TY - 1) / var.TY;
            int di = (int)hd.size();
            hd.push_back(d);
            for (int t = 0; t < d.ntx * nty; ++t) hi.push_back(BatchItem{di, t});
            L[p] += d.b;
            int op = prv[p], oc = cur[p];
            prv[p] = spa[p];
            cur[p] = spb[p];
            spa[p] = op;
            spb[p] = oc;
        }
        if (hd.size() == d0) break;
        ranges.emplace_back(d0, i0);
    }
    ranges.emplace_back(hd.size(), hi.size());
    if (build_only) return EW_OK;
    for (size_t r = 0; r + 1 < ranges.size(); ++r) {
        const BatchDesc<T>* dd = ddesc;
        const BatchItem* di = ditem + ranges[r].second;
        int nitems = (int)(ranges[r + 1].second - ranges[r].second);
        int grid = std::min(nitems, nsm);
        void* args[] = {(void*)&dd, (void*)&di, (void*)&nitems};
        EW_CUDA_TRY(cudaLaunchKernel(gen ? var.fn_gen : var.fn, dim3(grid), dim3(var.threads), args, var.smem, cs));
        count_launch();
    }
    return EW_OK;
}

template <typename T>
static ew_status batched_t(std::vector<BProblem>& P, int order, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_batch.mu);
    const auto& vars = order == 2 ? bvariants<T, 1>() : bvariants<T, 2>();
    int dev = 0;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    int nsm = 0;
    EW_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // any problem with a Neumann face: the general instantiation for the whole batch
    bool gen = false;
    for (const auto& p : P) gen = gen || p.g.bc != 0;
    for (const auto& v : vars) {
        if (!g_batch.occ.count(v.fn)) {
            EW_CUDA_TRY(cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
            EW_CUDA_TRY(cudaFuncSetAttribute(v.fn_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
            int occ = 0;
            EW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, v.threads, v.smem));
            g_batch.occ[v.fn] = std::max(occ, 1);
        }
    }
    // workspace: 4 fields per problem + weight tables
    size_t off = 0;
    for (auto& p : P) {
        p.field_off = off;
        off += 4 * (size_t)p.g.N;
    }
    for (auto& p : P) {
        p.c_off = off;
        off += p.plan.c.size();
    }
    size_t field_bytes = ((off * sizeof(T) + 255) / 256) * 256;
    // tables: worst case over the variants (deepest tiles: the most rounds x tiles)
    std::vector<std::vector<BatchDesc<T>>> hds(vars.size());
    std::vector<std::vector<BatchItem>> his(vars.size());
    std::vector<std::vector<std::pair<size_t, size_t>>> rgs(vars.size());
    size_t tbl = 0;
    for (size_t v = 0; v < vars.size(); ++v) {
        EW_TRY(run_rounds<T>(P, vars[v], nullptr, nsm, nullptr, hds[v], his[v], rgs[v], true, nullptr, nullptr, gen));
        tbl = std::max(tbl, hds[v].size() * sizeof(BatchDesc<T>) + 256 + his[v].size() * sizeof(BatchItem));
    }
    size_t need = field_bytes + tbl + 256;
    if (g_batch.dev_bytes < need) {
        if (g_batch.dev) cudaFree(g_batch.dev);
        g_batch.dev = nullptr;
        g_batch.dev_bytes = 0;
        cudaError_t e = cudaMalloc(&g_batch.dev, need);
        if (e != cudaSuccess) {
            g_batch.dev = nullptr;
            cudaGetLastError();
            return set_error(EW_ENOMEM, "batched workspace allocation failed");
        }
        g_batch.dev_bytes = need;
    }
    if (g_batch.host_bytes < need) {
        if (g_batch.host) cudaFreeHost(g_batch.host);
        g_batch.host = nullptr;
        g_batch.host_bytes = 0;
        cudaError_t e = cudaMallocHost(&g_batch.host, need);
        if (e != cudaSuccess) {
            g_batch.host = nullptr;
            cudaGetLastError();
            return set_error(EW_ENOMEM, "batched pinned staging allocation failed");
        }
        g_batch.host_bytes = need;
    }
    if (!g_batch.cap) EW_CUDA_TRY(cudaStreamCreateWithFlags(&g_batch.cap, cudaStreamNonBlocking));
    if (!g_batch.ev_in) EW_CUDA_TRY(cudaEventCreateWithFlags(&g_batch.ev_in, cudaEventDisableTiming));
    if (!g_batch.ev_out) EW_CUDA_TRY(cudaEventCreateWithFlags(&g_batch.ev_out, cudaEventDisableTiming));
    T* base = (T*)g_batch.dev;
    char* tdev = (char*)g_batch.dev + field_bytes;
    // weights (host staging -> device)
    EW_CUDA_TRY(cudaStreamSynchronize(st));  // the pinned staging may still feed a previous copy
    T* hw = (T*)g_batch.host;
    for (auto& p : P)
        for (size_t i = 0; i < p.plan.c.size(); ++i) hw[p.c_off - P[0].c_off + i] = (T)p.plan.c[i];
    size_t cbytes = (off - P[0].c_off) * sizeof(T);
    EW_CUDA_TRY(cudaMemcpyAsync(base + P[0].c_off, hw, cbytes, cudaMemcpyHostToDevice, st));
    EW_CUDA_TRY(cudaStreamSynchronize(st));

    // choose the variant for this batch shape (time one full batched solve per candidate)
    std::vector<int64_t> key = {(int64_t)sizeof(T), order, dev};
    for (auto& p : P) {
        key.push_back(p.g.n[0]);
        key.push_back(p.g.n[1]);
        key.push_back(p.plan.Nt);
    }
    auto upload_and_run = [&](size_t v, cudaStream_t s) -> ew_status {
        // descriptors with their real device addresses, then items
        std::vector<BatchDesc<T>> hd;
        std::vector<BatchItem> hi;
        std::vector<std::pair<size_t, size_t>> rg;
        EW_TRY(run_rounds<T>(P, vars[v], base, nsm, nullptr, hd, hi, rg, true, nullptr, nullptr, gen));
        BatchDesc<T>* ddesc = (BatchDesc<T>*)tdev;
        BatchItem* ditem = (BatchItem*)(tdev + ((hd.size() * sizeof(BatchDesc<T>) + 255) / 256) * 256);
        char* hstage = (char*)g_batch.host + field_bytes;
        std::memcpy(hstage, hd.data(), hd.size() * sizeof(BatchDesc<T>));
        std::memcpy(hstage + ((char*)ditem - tdev), hi.data(), hi.size() * sizeof(BatchItem));
        size_t tb = ((char*)ditem - tdev) + hi.size() * sizeof(BatchItem);
        EW_CUDA_TRY(cudaMemcpyAsync(tdev, hstage, tb, cudaMemcpyHostToDevice, st));
        // the first step of every problem, then the rounds, captured in one graph
        EW_CUDA_TRY(cudaEventRecord(g_batch.ev_in, st));
        EW_CUDA_TRY(cudaStreamWaitEvent(s, g_batch.ev_in, 0));
        EW_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        ew_status rs = EW_OK;
        {
            ProfilePause pause;  // the captured launches are counted once, below
            for (auto& p : P) {
                T* F = base + p.field_off;
                if (rs == EW_OK)
                    rs = first_step<T>(p.g, (const T*)p.vin, F, F + p.g.N, (T*)p.vout, p.plan, 1, p.g.N, s);
            }
            int grid_mult = g_batch.occ[vars[v].fn];
            if (rs == EW_OK) {
                std::vector<BatchDesc<T>> d2;
                std::vector<BatchItem> i2;
                std::vector<std::pair<size_t, size_t>> r2;
                rs = run_rounds<T>(P, vars[v], base, nsm * grid_mult, s, d2, i2, r2, false, ddesc, ditem, gen);
            }
        }
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (rs != EW_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rs;
        }
        if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphInstantiate");
        ce = cudaGraphLaunch(exec, st);
        cudaGraphExecDestroy(exec);
        if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphLaunch");
        count_launch((int64_t)P.size() + (int64_t)rg.size() - 1);  // first steps + rounds in the graph
        return EW_OK;
    };
    int vi = 0;
    auto it = g_batch.tune.find(key);
    if (it != g_batch.tune.end()) {
        vi = it->second;
    } else if (vars.size() > 1) {
        EventPair ev;
        EW_TRY(ev.create());
        cudaEvent_t e0 = ev.a, e1 = ev.b;
        float best = 1e30f;
        for (size_t v = 0; v < vars.size(); ++v) {
            EW_CUDA_TRY(cudaEventRecord(e0, st));
            EW_TRY(upload_and_run(v, g_batch.cap));
            EW_CUDA_TRY(cudaEventRecord(e1, st));
            EW_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (getenv("EW_TUNE_LOG"))
                fprintf(stderr, "[ew tune] batched %zu problems: variant %zu (depth %d, tile %dx%d): %.3f ms\n",
                        P.size(), v, vars[v].B, vars[v].TX, vars[v].TY, ms);
            if (ms < best) {
                best = ms;
                vi = (int)v;
            }
        }
        g_batch.tune[key] = vi;
    }
    return upload_and_run((size_t)vi, g_batch.cap);
}

}  // namespace ew

using namespace ew;

extern "C" ew_status ew_filter_apply_batched(int nprob, const ew_grid* const* grids, const ew_filter_params* params,
                                             const void* const* v_in, void* const* v_out, const int* nvec,
                                             cudaStream_t stream) try {
    clear_error();
    if (nprob < 1 || !grids || !params || !v_in || !v_out) return set_error(EW_EINVAL, "bad arguments");
    int dev = -1;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    const ew_grid* g0 = grids[0];
    if (!g0) return set_error(EW_EINVAL, "null grid");
    std::vector<BProblem> P;
    bool uniform = true;
    for (int q = 0; q < nprob; ++q) {
        const ew_grid* g = grids[q];
        if (!g || !v_in[q] || !v_out[q]) return set_error(EW_EINVAL, "null grid or vector");
        if (g->device >= 0 && g->device != dev) return set_error(EW_EINVAL, "grid was created on another device");
        int nv = nvec ? nvec[q] : 1;
        if (nv < 1) return set_error(EW_EINVAL, "nvec must be >= 1");
        FilterPlan plan;
        EW_TRY(plan_filter(g->geom, &params[q], &plan));
        if (g->geom.dim != 2 || params[q].scheme != EW_EXPLICIT || g->prec != g0->prec ||
            g->geom.order != g0->geom.order || g->geom.map || g->prec == EW_FP32X2)
            uniform = false;
        size_t es = g->prec == EW_FP32 ? 4 : 8;
        const size_t bytes = (size_t)nv * g->geom.N * es;
        const char* a = (const char*)v_in[q];
        const char* b = (const char*)v_out[q];
        if (a < b + bytes && b < a + bytes) return set_error(EW_EINVAL, "v_in and v_out of a problem overlap");
        for (int v = 0; v < nv; ++v) {
            BProblem b;
            b.g = g->geom;
            b.plan = plan;
            b.vin = (const char*)v_in[q] + (size_t)v * g->geom.N * es;
            b.vout = (char*)v_out[q] + (size_t)v * g->geom.N * es;
            P.push_back(b);
        }
    }
    if (!uniform) {
        // mixed batches (3D, implicit, curvilinear, mixed precision or order): one call per problem
        for (int q = 0; q < nprob; ++q)
            EW_TRY(ew_filter_apply(grids[q], &params[q], v_in[q], v_out[q], nvec ? nvec[q] : 1, stream));
        return EW_OK;
    }
    if (g0->prec == EW_FP32) return batched_t<float>(P, g0->geom.order, stream);
    return batched_t<double>(P, g0->geom.order, stream);
} catch (...) {
    return abi_exception();
}
