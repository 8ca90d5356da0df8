// ew_core.cu -- C ABI entry points: grid handles, filter parameters (a1),
// wave-solve dispatch, Rayleigh quotient (a8) and the power iteration
// (Algorithm EigenWave).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <stdexcept>
#include <utility>
#include <vector>
#include <cstring>
#include <string>

#include "ew_dd.cuh"
#include "ew_internal.h"

namespace ew {

static thread_local std::string g_last_error;

// ---- launch accounting -------------------------------------------------------
std::atomic<bool> g_profile_on{false};
static std::mutex g_prof_mu;
static int64_t g_launches = 0, g_fused_launches = 0, g_fused_cells = 0, g_fused_points = 0;
static int64_t g_mg_cycles = 0, g_mg_solves = 0;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_fused_events;
static std::vector<cudaEvent_t> g_event_pool;

void count_launch(int64_t k) {
    if (!g_profile_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += k;
}

void count_mg_solve(int cycles) {
    if (!g_profile_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_mg_cycles += cycles;
    g_mg_solves += 1;
}

static cudaEvent_t pool_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

cudaEvent_t fused_begin(cudaStream_t st) {
    if (!g_profile_on) return nullptr;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = pool_event();
    if (e) cudaEventRecord(e, st);
    return e;
}

void fused_end(cudaEvent_t start, cudaStream_t st, int64_t points, int64_t cell_steps) {
    if (!g_profile_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += 1;
    g_fused_launches += 1;
    g_fused_cells += cell_steps;
    g_fused_points += points;
    if (!start) return;
    cudaEvent_t e = pool_event();
    if (!e) return;
    cudaEventRecord(e, st);
    g_fused_events.emplace_back(start, e);
}

static void profile_reset_locked() {
    for (auto& pr : g_fused_events) {
        g_event_pool.push_back(pr.first);
        g_event_pool.push_back(pr.second);
    }
    g_fused_events.clear();
    g_launches = g_fused_launches = g_fused_cells = g_fused_points = 0;
    g_mg_cycles = g_mg_solves = 0;
}

ew_status set_error(ew_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
ew_status cuda_error(cudaError_t e, const char* what) {
    return set_error(EW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
void clear_error() { g_last_error.clear(); }

ew_status abi_exception() {
    try {
        throw;
    } catch (const std::bad_alloc&) {
        return set_error(EW_ENOMEM, "host allocation failed");
    } catch (const std::length_error& e) {
        return set_error(EW_ENOMEM, std::string("host container too large: ") + e.what());
    } catch (const std::exception& e) {
        return set_error(EW_EINVAL, std::string("host exception: ") + e.what());
    } catch (...) {
        return set_error(EW_EINVAL, "unknown host exception");
    }
}

ew_status Scratch::reserve(size_t want) {
    if (want <= bytes) return EW_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        return set_error(EW_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed: " +
                                        cudaGetErrorString(e));
    }
    bytes = want;
    return EW_OK;
}
void Scratch::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

// Longest wave-solve: N_t (and with it the N_t + 1 filter weights) stays below 2^31 - 1.
static constexpr int64_t kMaxSteps = INT32_MAX - 1;

// Largest eigenvalue of -L_h: the 1D symbols 4 s (order 2) and 4 s + (4/3) s^2
// (order 4) at s = sin^2 = 1, summed over the axes.
static double rho_bound(const GridGeom& g) {
    if (g.map) return g.map->rho;
    double inv = 0.0;
    for (int a = 0; a < g.dim; ++a) inv += 1.0 / (g.h[a] * g.h[a]);
    return (g.order == 2 ? 4.0 : 16.0 / 3.0) * inv;
}

ew_status plan_filter(const GridGeom& g, const ew_filter_params* p, FilterPlan* out, bool with_weights) {
    if (!p) return set_error(EW_EINVAL, "params is NULL");
    if (!(p->omega > 0.0) || !std::isfinite(p->omega)) return set_error(EW_EINVAL, "omega must be > 0");
    if (p->num_periods < 1) return set_error(EW_EINVAL, "num_periods must be >= 1");
    if (p->scheme != EW_EXPLICIT && p->scheme != EW_IMPLICIT) return set_error(EW_EINVAL, "bad scheme");
    int spp = p->steps_per_period;
    if (spp < 0) return set_error(EW_EINVAL, "steps_per_period < 0");
    if (spp == 0) {
        if (p->scheme != EW_EXPLICIT)
            return set_error(EW_EINVAL, "steps_per_period must be given for the implicit scheme");
        double cfl = p->cfl > 0.0 ? p->cfl : 0.8;
        double dtmax = 2.0 / sqrt(rho_bound(g));
        double period = 2.0 * M_PI / p->omega;
        double want = ceil(period / (cfl * dtmax) - 1e-12);
        if (!(want <= (double)kMaxSteps))
            return set_error(EW_EINVAL, "omega too small for this grid: more than 2^31 - 2 steps per period");
        spp = want < 1.0 ? 1 : (int)want;
    }
    if (spp < 2) return set_error(EW_EINVAL, "need at least 2 steps per period");
    if ((int64_t)p->num_periods * spp > kMaxSteps)
        return set_error(EW_EINVAL, "N_t = num_periods * steps_per_period exceeds 2^31 - 2");
    double w = p->omega;
    if (p->adjust_omega) {
        // omega~ = (omega pi / N_its) sqrt((1 - 2 sin^2(pi/N_its)) / sin^2(pi/N_its))  (eq. adjustedOmega)
        if (spp <= 4) return set_error(EW_EINVAL, "adjust_omega needs more than 4 steps per period");
        double s = sin(M_PI / spp);
        w = p->omega * M_PI / spp * sqrt((1.0 - 2.0 * s * s) / (s * s));
    }
    out->omega = w;
    out->spp = spp;
    out->Nt = (int64_t)p->num_periods * spp;
    out->Tf = p->num_periods * 2.0 * M_PI / w;
    out->dt = out->Tf / (double)out->Nt;
    out->alpha_d = tan(0.5 * w * out->dt) / tan(w * out->dt);
    if (p->scheme == EW_EXPLICIT) {
        // leapfrog is stable only for dt^2 rho / 4 <= 1
        if (out->dt * out->dt * rho_bound(g) > 4.0 * (1.0 + 1e-12))
            return set_error(EW_EINVAL, "explicit time step beyond the stability limit (raise steps_per_period)");
    }
    out->c.clear();
    if (with_weights) {
        out->c.resize((size_t)out->Nt + 1);
        for (int64_t n = 0; n <= out->Nt; ++n) out->c[(size_t)n] = out->cn(n);
    }
    return EW_OK;
}

ew_status check_grid(const ew_grid* g) {
    if (!g) return set_error(EW_EINVAL, "grid is NULL");
    int dev = -1;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    // a grid created while no device was visible binds to the first device it runs on
    if (g->device < 0) const_cast<ew_grid*>(g)->device = dev;
    if (dev != g->device) return set_error(EW_EINVAL, "grid was created on another device");
    return EW_OK;
}

size_t elem_size(const ew_grid* g) { return g->prec == EW_FP32 ? 4 : 8; }

static ew_status pinned(ew_grid* g, size_t bytes, void** out) {
    if (g->host_pinned_bytes < bytes) {
        if (g->host_pinned) cudaFreeHost(g->host_pinned);
        g->host_pinned = nullptr;
        g->host_pinned_bytes = 0;
        EW_CUDA_TRY(cudaMallocHost(&g->host_pinned, bytes));
        g->host_pinned_bytes = bytes;
    }
    *out = g->host_pinned;
    return EW_OK;
}

// upload the filter weights (type T) into the grid's misc scratch
template <typename T>
static ew_status upload_weights(ew_grid* g, const FilterPlan& plan, cudaStream_t st, const T** out) {
    size_t n = plan.c.size();
    EW_TRY(g->misc.reserve(n * sizeof(T)));
    void* hp = nullptr;
    EW_TRY(pinned(g, n * sizeof(T), &hp));
    // the pinned buffer may still feed an earlier copy on this stream
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    T* h = (T*)hp;
    for (size_t i = 0; i < n; ++i) h[i] = (T)plan.c[i];
    EW_CUDA_TRY(cudaMemcpyAsync(g->misc.ptr, h, n * sizeof(T), cudaMemcpyHostToDevice, st));
    *out = (const T*)g->misc.ptr;
    return EW_OK;
}

ew_status implicit_wave_solve_any(ew_grid* g, const FilterPlan& plan, const ew_filter_params* p,
                                  const void* vin, void* vout, int nvec, cudaStream_t st);

template <typename T>
static ew_status filter_apply_t(ew_grid* g, const ew_filter_params* p, const FilterPlan& plan, const T* vin,
                                T* vout, int nvec, cudaStream_t st) {
    if (p->scheme == EW_IMPLICIT) return implicit_wave_solve_any(g, plan, p, vin, vout, nvec, st);
    const T* cdev = nullptr;
    EW_TRY(upload_weights<T>(g, plan, st, &cdev));
    EW_TRY(g->fields.reserve((size_t)4 * nvec * wave_field_stride(g->geom) * sizeof(T)));
    return explicit_wave_solve<T>(g->geom, plan, cdev, vin, vout, nvec, (T*)g->fields.ptr, p->temporal_block, st);
}

__global__ void k_to_dd(const double* __restrict__ x, dd* __restrict__ y, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        y[q] = dd(x[q]);
}
__global__ void k_from_dd(const dd* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        y[q] = (double)x[q];
}

// EW_FP32X2 grids: FP64 vectors in and out, the wave-solve in double-FP32 pairs
static ew_status filter_apply_dd(ew_grid* g, const ew_filter_params* p, const FilterPlan& plan, const double* vin,
                                 double* vout, int nvec, cudaStream_t st) {
    if (p->scheme == EW_IMPLICIT)
        return set_error(EW_EUNSUPPORTED, "double-FP32 grids run the explicit scheme only");
    const int64_t n = g->geom.N * (int64_t)nvec;
    const dd* cdev = nullptr;
    EW_TRY(upload_weights<dd>(g, plan, st, &cdev));
    EW_TRY(g->fields.reserve((size_t)4 * nvec * wave_field_stride(g->geom) * sizeof(dd)));
    EW_TRY(g->pairs.reserve((size_t)2 * n * sizeof(dd)));
    dd* din = (dd*)g->pairs.ptr;
    dd* dout = din + n;
    k_to_dd<<<kReduceBlocks * 4, 256, 0, st>>>(vin, din, n);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    EW_TRY(explicit_wave_solve<dd>(g->geom, plan, cdev, din, dout, nvec, (dd*)g->fields.ptr, p->temporal_block, st));
    k_from_dd<<<kReduceBlocks * 4, 256, 0, st>>>(dout, vout, n);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}

ew_status filter_apply_any(ew_grid* g, const ew_filter_params* p, const FilterPlan& plan, const void* vin,
                           void* vout, int nvec, cudaStream_t st) {
    if (g->prec == EW_FP32X2) return filter_apply_dd(g, p, plan, (const double*)vin, (double*)vout, nvec, st);
    if (g->prec == EW_FP32) return filter_apply_t<float>(g, p, plan, (const float*)vin, (float*)vout, nvec, st);
    return filter_apply_t<double>(g, p, plan, (const double*)vin, (double*)vout, nvec, st);
}

}  // namespace ew

using namespace ew;

extern "C" {

const char* ew_last_error(void) { return g_last_error.c_str(); }

ew_status ew_profile_enable(int on) try {
    clear_error();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& pr : g_fused_events) {
        cudaEventSynchronize(pr.second);
    }
    profile_reset_locked();
    g_profile_on = on != 0;
    return EW_OK;
} catch (...) {
    return abi_exception();
}

ew_status ew_profile_read(ew_profile* out) try {
    clear_error();
    if (!out) return set_error(EW_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double ms = 0.0;
    for (auto& pr : g_fused_events) {
        EW_CUDA_TRY(cudaEventSynchronize(pr.second));
        float t = 0.f;
        EW_CUDA_TRY(cudaEventElapsedTime(&t, pr.first, pr.second));
        ms += t;
    }
    out->launches = g_launches;
    out->fused_launches = g_fused_launches;
    out->fused_ms = ms;
    out->fused_cell_steps = g_fused_cells;
    out->fused_points = g_fused_points;
    out->mg_cycles = g_mg_cycles;
    out->mg_solves = g_mg_solves;
    profile_reset_locked();
    return EW_OK;
} catch (...) {
    return abi_exception();
}

ew_status ew_grid_create(int dim, const int64_t n_interior[3], const double length[3], int order,
                         const ew_bc bc[6], ew_prec prec, ew_grid** out) try {
    clear_error();
    if (!out || !n_interior || !length) return set_error(EW_EINVAL, "null argument");
    *out = nullptr;
    if (dim != 2 && dim != 3) return set_error(EW_EINVAL, "dim must be 2 or 3");
    if (order != 2 && order != 4) return set_error(EW_EINVAL, "order must be 2 or 4");
    if (prec != EW_FP32 && prec != EW_FP64 && prec != EW_FP32X2) return set_error(EW_EINVAL, "bad precision");
    if (prec == EW_FP32X2 && dim != 2) return set_error(EW_EUNSUPPORTED, "double-FP32 fields: 2D boxes only");
    GridGeom geom;
    geom.bc = 0;
    if (bc)
        for (int f = 0; f < 2 * dim; ++f) {
            if (bc[f] != EW_BC_DIRICHLET && bc[f] != EW_BC_NEUMANN) return set_error(EW_EINVAL, "bad boundary kind");
            if (bc[f] == EW_BC_NEUMANN) geom.bc |= 1 << f;
        }
    geom.dim = dim;
    geom.order = order;
    geom.N = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < dim) {
            if (n_interior[a] < 1) return set_error(EW_EINVAL, "n_interior must be >= 1");
            if (n_interior[a] > (int64_t)1 << 30) return set_error(EW_EINVAL, "axis too long");
            if (!(length[a] > 0.0)) return set_error(EW_EINVAL, "length must be > 0");
            // a Neumann face's wall point is active (a symmetry plane of the vertex grid)
            geom.n[a] = n_interior[a] + ((geom.bc >> (2 * a)) & 1) + ((geom.bc >> (2 * a + 1)) & 1);
            geom.h[a] = length[a] / (double)(n_interior[a] + 1);
        } else {
            geom.n[a] = 1;
            geom.h[a] = 1.0;
        }
        // 2^40 active points (4 TB of FP32 per field) is far beyond any device;
        // the bound keeps N and every byte count derived from it exact
        if (geom.N > ((int64_t)1 << 40) / geom.n[a])
            return set_error(EW_EINVAL, "grid too large: more than 2^40 active points");
        geom.N *= geom.n[a];
    }
    if (dim == 2 && (geom.n[0] > INT32_MAX / 2 || geom.n[1] > INT32_MAX / 2))
        return set_error(EW_EINVAL, "2D axis too long");
    // creating a grid needs no GPU (parameters and weights are host work);
    // without a visible device the handle binds to the first device it runs on
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        dev = -1;
        cudaGetLastError();
    }
    ew_grid* g = new (std::nothrow) ew_grid();
    if (!g) return set_error(EW_ENOMEM, "host allocation failed");
    g->geom = geom;
    for (int a = 0; a < 3; ++a) g->length[a] = a < dim ? length[a] : 1.0;
    g->prec = prec;
    g->device = dev;
    *out = g;
    return EW_OK;
} catch (...) {
    return abi_exception();
}

void ew_grid_destroy(ew_grid* g) {
    if (!g) return;
    if (g->geom.map) {
        mapped_release(g->geom.map);
        delete g->geom.map;
        g->geom.map = nullptr;
    }
    g->fields.release();
    g->reduce.release();
    g->misc.release();
    g->mg.release();
    g->pairs.release();
    g->mgh.release();
    g->hostio.release();
    if (g->host_pinned) cudaFreeHost(g->host_pinned);
    delete g;
}

ew_status ew_filter_setup(const ew_grid* grid, const ew_filter_params* params, ew_filter_info* info,
                          double* weights, int64_t cap) try {
    clear_error();
    if (!grid) return set_error(EW_EINVAL, "grid is NULL");
    FilterPlan plan;
    EW_TRY(plan_filter(grid->geom, params, &plan));
    if (info) {
        info->omega_used = plan.omega;
        info->final_time = plan.Tf;
        info->dt = plan.dt;
        info->alpha_d = plan.alpha_d;
        info->num_steps = plan.Nt;
        info->steps_per_period = plan.spp;
    }
    if (weights) {
        if (cap < plan.Nt + 1) return set_error(EW_EINVAL, "weights capacity < N_t + 1");
        std::memcpy(weights, plan.c.data(), sizeof(double) * plan.c.size());
    }
    return EW_OK;
} catch (...) {
    return abi_exception();
}

ew_status ew_filter_apply(const ew_grid* grid, const ew_filter_params* params, const void* v_in, void* v_out,
                          int nvec, cudaStream_t stream) try {
    clear_error();
    EW_TRY(check_grid(grid));
    if (!v_in || !v_out) return set_error(EW_EINVAL, "null vector pointer");
    if (nvec < 1 || nvec > 65535) return set_error(EW_EINVAL, "nvec must be in [1, 65535]");
    size_t bytes = (size_t)nvec * grid->geom.N * elem_size(grid);
    const char* a = (const char*)v_in;
    const char* b = (const char*)v_out;
    if (a < b + bytes && b < a + bytes) return set_error(EW_EINVAL, "v_in and v_out overlap");
    FilterPlan plan;
    EW_TRY(plan_filter(grid->geom, params, &plan));
    ew_grid* g = const_cast<ew_grid*>(grid);
    return filter_apply_any(g, params, plan, v_in, v_out, nvec, stream);
} catch (...) {
    return abi_exception();
}

ew_status ew_apply_L(const ew_grid* grid, const void* u, void* Lu, int nvec, cudaStream_t stream) try {
    clear_error();
    EW_TRY(check_grid(grid));
    if (!u || !Lu) return set_error(EW_EINVAL, "null vector pointer");
    if (nvec < 1 || nvec > 65535) return set_error(EW_EINVAL, "nvec must be in [1, 65535]");
    if (grid->prec == EW_FP32X2) return set_error(EW_EUNSUPPORTED, "double-FP32 grids: ew_filter_apply only");
    if (grid->prec == EW_FP32) return launch_apply_L<float>(grid->geom, (const float*)u, (float*)Lu, nvec, 1.0, stream);
    return launch_apply_L<double>(grid->geom, (const double*)u, (double*)Lu, nvec, 1.0, stream);
} catch (...) {
    return abi_exception();
}

}  // extern "C"

namespace ew {

template <typename T>
static ew_status rayleigh_t(ew_grid* g, const T* phi, int nvec, double* lam_host, double* res_host,
                            cudaStream_t st) {
    const int64_t N = g->geom.N;
    // scratch: Lphi (nvec * N of T) in fields; reduction partials and results in reduce
    const bool weighted = weighted_sums(g->geom);
    EW_TRY(g->fields.reserve((weighted ? 3 : 1) * (size_t)nvec * N * sizeof(T)));
    size_t part = (size_t)2 * nvec * kReduceBlocks;
    EW_TRY(g->reduce.reserve((part + 6 * (size_t)nvec) * sizeof(double)));
    double* dpart = (double*)g->reduce.ptr;
    double* dnum = dpart + part;     // phi . L phi
    double* dden = dnum + nvec;      // phi . phi
    double* dlam2 = dden + nvec;     // lambda^2
    double* dres = dlam2 + nvec;     // 2 * nvec: (resid, xinf)
    T* Lphi = (T*)g->fields.ptr;
    EW_TRY(launch_apply_L<T>(g->geom, phi, Lphi, nvec, 1.0, st));
    if (weighted) {
        // Neumann faces: the sums of the quotient carry the trapezoid weights W
        // (the discrete L_2 inner product, in which L_h is symmetric there):
        // (W^{1/2} phi) . (W^{1/2} L phi) and |W^{1/2} phi|^2
        T* wp = Lphi + (size_t)nvec * N;
        T* wl = wp + (size_t)nvec * N;
        EW_TRY(launch_wsqrt<T>(g->geom, phi, wp, nvec, 1, st));
        EW_TRY(launch_wsqrt<T>(g->geom, Lphi, wl, nvec, 1, st));
        EW_TRY(launch_dots<T>(wp, wl, N, nvec, dpart, dnum, st));
        EW_TRY(launch_dots<T>(wp, wp, N, nvec, dpart, dden, st));
    } else {
        EW_TRY(launch_dots<T>(phi, Lphi, N, nvec, dpart, dnum, st));
        EW_TRY(launch_dots<T>(phi, phi, N, nvec, dpart, dden, st));
    }
    void* hp = nullptr;
    EW_TRY(pinned(g, sizeof(double) * 4 * (size_t)nvec, &hp));
    double* h = (double*)hp;
    EW_CUDA_TRY(cudaMemcpyAsync(h, dnum, sizeof(double) * 2 * nvec, cudaMemcpyDeviceToHost, st));
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    EW_TRY(rb2d_check_timeout());  // a register-blocked wave-solve before this point gave up a wait
    EW_TRY(tma2d_check_timeout());  // the same for a TMA-staged one
    std::vector<double> lam2(nvec);
    for (int j = 0; j < nvec; ++j) {
        double den = h[nvec + j];
        lam2[j] = den > 0.0 ? -h[j] / den : 0.0;
        lam_host[j] = sqrt(std::max(lam2[j], 0.0));
    }
    if (res_host) {
        std::memcpy(h, lam2.data(), sizeof(double) * nvec);
        EW_CUDA_TRY(cudaMemcpyAsync(dlam2, h, sizeof(double) * nvec, cudaMemcpyHostToDevice, st));
        EW_TRY(launch_resid_inf<T>(Lphi, phi, N, nvec, dlam2, dpart, dres, nullptr, st));
        EW_CUDA_TRY(cudaMemcpyAsync(h, dres, sizeof(double) * 2 * nvec, cudaMemcpyDeviceToHost, st));
        EW_CUDA_TRY(cudaStreamSynchronize(st));
        for (int j = 0; j < nvec; ++j) {
            double xinf = h[2 * j + 1];
            res_host[j] = (lam2[j] > 0.0 && xinf > 0.0) ? h[2 * j] / (lam2[j] * xinf) : INFINITY;
        }
    }
    return EW_OK;
}

template <typename T>
static ew_status power_t(ew_grid* g, const ew_filter_params* p, T* v, int iters, double tol, double* beta_host,
                         int* done, double* lam_host, cudaStream_t st) {
    const int64_t N = g->geom.N;
    FilterPlan plan;
    EW_TRY(plan_filter(g->geom, p, &plan));
    // the new iterate lives in the `mg` scratch, which explicit wave-solves do not use
    if (p->scheme == EW_IMPLICIT) return set_error(EW_EUNSUPPORTED, "power iteration runs the explicit scheme");
    EW_TRY(g->mg.reserve((size_t)N * sizeof(T)));
    T* w = (T*)g->mg.ptr;
    size_t part = (size_t)kReduceBlocks;
    EW_TRY(g->reduce.reserve((part + 8) * sizeof(double)));
    double* dpart = (double*)g->reduce.ptr;
    double* dsc = dpart + part;  // [0] |w|^2, [1] scale, [2] beta, [3] diff^2
    void* hp = nullptr;
    EW_TRY(pinned(g, sizeof(double) * 8, &hp));
    double* h = (double*)hp;
    EW_TRY(launch_dots<T>(v, v, N, 1, dpart, dsc, st));
    EW_CUDA_TRY(cudaMemcpyAsync(h, dsc, sizeof(double), cudaMemcpyDeviceToHost, st));
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(h[0] > 0.0) || !std::isfinite(h[0])) return set_error(EW_EINVAL, "start vector is zero or not finite");
    h[1] = 1.0 / sqrt(h[0]);
    EW_CUDA_TRY(cudaMemcpyAsync(dsc + 1, h + 1, sizeof(double), cudaMemcpyHostToDevice, st));
    EW_TRY(launch_scale<T>(v, N, 1, dsc + 1, st));
    int k = 0;
    for (k = 0; k < iters;) {
        EW_TRY(filter_apply_t<T>(g, p, plan, v, w, 1, st));      // w = S v
        EW_TRY(launch_dots<T>(w, v, N, 1, dpart, dsc + 2, st));   // beta = (S v, v)
        EW_TRY(launch_dots<T>(w, w, N, 1, dpart, dsc, st));
        EW_CUDA_TRY(cudaMemcpyAsync(h, dsc, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
        EW_CUDA_TRY(cudaStreamSynchronize(st));
        double beta = h[2];
        if (!(h[0] > 0.0) || !std::isfinite(h[0]) || !std::isfinite(beta))
            return set_error(EW_ENOCONV, "power iterate vanished or is not finite");
        if (beta_host) beta_host[k] = beta;
        h[1] = 1.0 / sqrt(h[0]);
        EW_CUDA_TRY(cudaMemcpyAsync(dsc + 1, h + 1, sizeof(double), cudaMemcpyHostToDevice, st));
        EW_TRY(launch_scale<T>(w, N, 1, dsc + 1, st));             // normalise
        EW_TRY(launch_diffnorm_sign<T>(w, v, N, dsc + 2, dpart, dsc + 3, st));
        EW_CUDA_TRY(cudaMemcpyAsync(v, w, (size_t)N * sizeof(T), cudaMemcpyDeviceToDevice, st));
        EW_CUDA_TRY(cudaMemcpyAsync(h + 3, dsc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
        EW_CUDA_TRY(cudaStreamSynchronize(st));
        ++k;
        if (sqrt(h[3]) < tol) break;
    }
    if (done) *done = k;
    if (lam_host) EW_TRY(rayleigh_t<T>(g, v, 1, lam_host, nullptr, st));
    return EW_OK;
}

}  // namespace ew

namespace ew {
ew_status rayleigh_any(ew_grid* g, const void* phi, int nvec, double* lam, double* res, cudaStream_t st) {
    if (g->prec == EW_FP32) return rayleigh_t<float>(g, (const float*)phi, nvec, lam, res, st);
    return rayleigh_t<double>(g, (const double*)phi, nvec, lam, res, st);
}
}  // namespace ew

extern "C" {

ew_status ew_rayleigh(const ew_grid* grid, const void* phi, int nvec, double* lambda_host, double* eig_res_host,
                      cudaStream_t stream) try {
    clear_error();
    EW_TRY(check_grid(grid));
    if (!phi || !lambda_host) return set_error(EW_EINVAL, "null pointer");
    if (nvec < 1 || nvec > 65535) return set_error(EW_EINVAL, "nvec must be in [1, 65535]");
    if (grid->prec == EW_FP32X2) return set_error(EW_EUNSUPPORTED, "double-FP32 grids: ew_filter_apply only");
    ew_grid* g = const_cast<ew_grid*>(grid);
    if (grid->prec == EW_FP32) return rayleigh_t<float>(g, (const float*)phi, nvec, lambda_host, eig_res_host, stream);
    return rayleigh_t<double>(g, (const double*)phi, nvec, lambda_host, eig_res_host, stream);
} catch (...) {
    return abi_exception();
}

ew_status ew_power_iteration(const ew_grid* grid, const ew_filter_params* params, void* v, int iters, double tol,
                             double* beta_host, int* iters_done, double* lambda_host, cudaStream_t stream) try {
    clear_error();
    EW_TRY(check_grid(grid));
    if (!v || !params) return set_error(EW_EINVAL, "null pointer");
    if (iters < 0) return set_error(EW_EINVAL, "iters < 0");
    if (grid->prec == EW_FP32X2) return set_error(EW_EUNSUPPORTED, "double-FP32 grids: ew_filter_apply only");
    ew_grid* g = const_cast<ew_grid*>(grid);
    if (grid->prec == EW_FP32)
        return power_t<float>(g, params, (float*)v, iters, tol, beta_host, iters_done, lambda_host, stream);
    return power_t<double>(g, params, (double*)v, iters, tol, beta_host, iters_done, lambda_host, stream);
} catch (...) {
    return abi_exception();
}

}  // extern "C"
