// ew_internal.h -- shared declarations of the EigenWave CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ew.h"

namespace ew {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
ew_status set_error(ew_status s, const std::string& msg);
ew_status cuda_error(cudaError_t e, const char* what);
void clear_error();
// Called from the handler of an entry point's function-try-block (`catch (...)`):
// turns the active C++ exception (a failed host allocation, a container size
// beyond its limit) into a status and message, so that none crosses the ABI.
ew_status abi_exception();

#define EW_CUDA_TRY(call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ew::cuda_error(e_, #call); \
    } while (0)

#define EW_TRY(call)                          \
    do {                                      \
        ew_status s_ = (call);                \
        if (s_ != EW_OK) return s_;           \
    } while (0)

// a device allocation owned by a scope, freed on every return path
struct DeviceBuffer {
    void* p = nullptr;
    DeviceBuffer() = default;
    DeviceBuffer(const DeviceBuffer&) = delete;
    DeviceBuffer& operator=(const DeviceBuffer&) = delete;
    ~DeviceBuffer() {
        if (p) cudaFree(p);
    }
    ew_status alloc(size_t bytes) {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return set_error(EW_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        }
        return EW_OK;
    }
    template <typename T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

// ---------------------------------------------------------------------------
// launch accounting (ew_profile_*)
// ---------------------------------------------------------------------------
extern std::atomic<bool> g_profile_on;  // read by every launch, set by ew_profile_enable
void count_launch(int64_t k = 1);
// one multigrid solve of an implicit time step that ran `cycles` V-cycles
void count_mg_solve(int cycles);
// brackets a fused-step launch: returns the start event (or null when off)
cudaEvent_t fused_begin(cudaStream_t st);
void fused_end(cudaEvent_t start, cudaStream_t st, int64_t points, int64_t cell_steps);
// pauses the launch accounting for its lifetime (the autotuners' trial launches
// are not counted)
struct ProfilePause {
    bool prev;
    ProfilePause() : prev(g_profile_on.exchange(false)) {}
    ~ProfilePause() { g_profile_on = prev; }
    ProfilePause(const ProfilePause&) = delete;
    ProfilePause& operator=(const ProfilePause&) = delete;
};
// two timing events, destroyed with the object
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() = default;
    EventPair(const EventPair&) = delete;
    EventPair& operator=(const EventPair&) = delete;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    ew_status create() {
        EW_CUDA_TRY(cudaEventCreate(&a));
        EW_CUDA_TRY(cudaEventCreate(&b));
        return EW_OK;
    }
};

// ---------------------------------------------------------------------------
// stencil coefficients, already multiplied by a scale (dt^2, dt^2/2, -a, 1)
//   scale * L_h u = c0 u + sum_axis c1[a] (u[-1] + u[+1]) + c2[a] (u[-2] + u[+2])
// order 2: c1 = scale / h^2, c2 = 0,          c0 = -2 sum c1
// order 4: c1 = scale 16 / (12 h^2), c2 = -scale / (12 h^2), c0 = -scale 30/12 sum 1/h^2
// ---------------------------------------------------------------------------
// bc: the grid's face mask (bit 2a: lower face of axis a is a Neumann face,
// bit 2a+1: its upper face), which decides how points beyond the box are
// extended (ew_bc_dev.cuh)
template <typename T>
struct Stencil {
    T c0;
    T c1[3];
    T c2[3];
    int bc;
};

// a single curvilinear grid (ew_mapped.cu): couplings of J L on the vertex
// lattice (vertex (I, J) to (I+1, J), (I, J+1), (I+1, J+1), (I+1, J-1)), J at
// the active vertices, the vertex coordinates, the Gershgorin bound of
// rho(-L), and device copies made on first use
struct MappedData {
    int64_t n1 = 0, n2 = 0;
    std::vector<double> E, N, NE, SE;
    std::vector<double> J;
    std::vector<double> xy;
    double rho = 0.0;
    void* dev[2] = {nullptr, nullptr};  // per vertex (E, N, NE, SE), then (centre, 1/J): FP32 / FP64
    double* sqrtJ = nullptr;
    std::mutex mu;
};

struct GridGeom {
    int dim;
    int order;
    int64_t n[3];  // active points per axis (n[2] = 1 in 2D): interior points plus Neumann wall points
    double h[3];
    int64_t N;     // active points
    int bc = 0;    // face mask, as in Stencil
    MappedData* map = nullptr;  // a curvilinear grid (2D, order 2, Dirichlet): the couplings replace the stencil
};

// the sums of inner products carry weights (Neumann faces: trapezoid; mapped grids: J)
inline bool weighted_sums(const GridGeom& g) { return g.bc != 0 || g.map != nullptr; }

template <typename T>
Stencil<T> make_stencil(const GridGeom& g, double scale);

// ---------------------------------------------------------------------------
// device scratch owned by a grid handle
// ---------------------------------------------------------------------------
struct Scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
    ew_status reserve(size_t want);
    void release();
};

}  // namespace ew

struct ew_grid {
    ew::GridGeom geom;
    double length[3];
    ew_prec prec;
    int device;
    ew::Scratch fields;    // wave-solve time levels
    ew::Scratch reduce;    // reduction partials
    ew::Scratch misc;      // small device tables (filter weights)
    ew::Scratch mg;        // power-iteration iterate
    ew::Scratch mgh;       // multigrid hierarchy
    ew::Scratch pairs;     // EW_FP32X2 grids: the input and output vectors as double-FP32 pairs
    ew::Scratch hostio;    // ew_filter_apply_host: device buffers of two input and two output chunks
    void* host_pinned = nullptr;  // small pinned staging for reductions
    size_t host_pinned_bytes = 0;
};

namespace ew {

// filter parameters (a1) on the host
struct FilterPlan {
    double omega;
    double Tf;
    double dt;
    double alpha_d;
    int64_t Nt;
    int spp;
    std::vector<double> c;  // N_t + 1 weights (empty when planned without them)
    // weight n: (2/T_f) sigma_n (cos(omega t^n) - alpha_d / 2), trapezoid sigma
    double cn(int64_t n) const {
        double sigma = (n == 0 || n == Nt) ? 0.5 * dt : dt;
        return 2.0 / Tf * sigma * (cos(omega * (double)n * dt) - 0.5 * alpha_d);
    }
};
ew_status plan_filter(const GridGeom& g, const ew_filter_params* p, FilterPlan* out, bool with_weights = true);
// the grid is usable on the current device (binds it on first use); bytes of one vector element
ew_status check_grid(const ew_grid* g);
size_t elem_size(const ew_grid* g);

// --- kernels launchers (ew_stencil.cu) ------------------------------------
template <typename T>
ew_status launch_apply_L(const GridGeom& g, const T* u, T* Lu, int nvec, double scale,
                         cudaStream_t st);

// one explicit wave-solve for nvec vectors; fields = 4 * N * nvec elements
// of scratch; cdev = N_t + 1 weights (device, type T).
// temporally blocked 3D second-order steps (ew_tb3d.cu)
template <typename T>
ew_status tb3d_tune(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, T* acc, int nvec,
                    int64_t fstride, cudaStream_t st);
template <typename T>
ew_status tb3d_advance(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, int* prv, int* cur,
                       int64_t L, T* acc, int nvec, int64_t fstride, int tb, cudaStream_t st);

// register-blocked persistent form of the 2D FP32 blocked step (ew_rb2d.cu)
struct Rb2dDesc {
    void* fn;      // boxes with Dirichlet faces only
    void* fn_gen;  // any faces
    int nty, ky, B, TX, TY, threads;
    size_t smem;
};
const std::vector<Rb2dDesc>& rb2d_variants(int R);
ew_status rb2d_launch(const Rb2dDesc& d, const GridGeom& g, const float* Ain, const float* Bin, float* Aout,
                      float* Bout, float* acc, const float* cw, int b, const Stencil<float>& s, int nvec,
                      int64_t fstride, cudaStream_t st);
// reads (and clears) the flag a staging wait sets when it gives up: EW_ETIMEOUT if set
ew_status rb2d_check_timeout();

// TMA-staged persistent form of the 2D FP32 blocked step (ew_tma2d.cu)
struct Tma2dDesc {
    void* fn;      // boxes with Dirichlet faces only
    void* fn_gen;  // any faces
    int nwx, nty, ky, B, TX, TY, threads;
    size_t smem;
    int boxw, boxh;  // tensor-map box of one staged field
};
const std::vector<Tma2dDesc>& tma2d_variants(int R);
// fields of padded row pitch pitch2d(nx) (Ain, Bin, Aout, Bout), acc dense
ew_status tma2d_launch(const Tma2dDesc& d, const GridGeom& g, const float* Ain, const float* Bin, float* Aout,
                       float* Bout, float* acc, const float* cw, int b, const Stencil<float>& s, int nvec,
                       int64_t fstride, cudaStream_t st);
// reads (and clears) the flag a staging wait of the TMA-staged step sets when it gives up
ew_status tma2d_check_timeout();

// distance between consecutive vectors of a wave-solve's time-level fields:
// N rounded up to 64 points, so every vector starts on a 256-byte boundary
// (bulk copies need 16-byte aligned rows)
inline int64_t field_stride(int64_t N) { return (N + 63) & ~(int64_t)63; }
// row pitch of the 2D time-level fields in the layout of the TMA-staged step:
// nx rounded up to 4 points (tensor maps need 16-byte row strides)
inline int64_t pitch2d(int64_t nx) { return (nx + 3) & ~(int64_t)3; }
// vector stride of a wave-solve's time-level fields: room for either row
// pitch on 2D grids
inline int64_t wave_field_stride(const GridGeom& g) {
    return g.dim == 2 ? field_stride(pitch2d(g.n[0]) * g.n[1]) : field_stride(g.N);
}

template <typename T>
ew_status explicit_wave_solve(const GridGeom& g, const FilterPlan& plan, const T* cdev,
                              const T* vin, T* vout, int nvec, T* fields, int temporal_block,
                              cudaStream_t st);

// --- curvilinear grids (ew_mapped.cu) ----------------------------------------
ew_status mapped_build(int64_t n1, int64_t n2, const double* xy, MappedData* m);
void mapped_release(MappedData* m);
template <typename T>
ew_status mapped_apply_L(const GridGeom& g, const T* u, T* Lu, int nvec, double scale, cudaStream_t st);
template <typename T>
ew_status mapped_wave_solve(const GridGeom& g, const FilterPlan& plan, const T* vin, T* vout, int nvec, T* fields,
                            cudaStream_t st);
template <typename T>
ew_status mapped_wsqrt(const GridGeom& g, const T* in, T* out, int nvec, int e, cudaStream_t st);

// --- temporally blocked 2D steps (ew_tb2d.cu) -----------------------------
// choose (and cache) the tile / depth variant for this grid shape by timing
// each candidate on the given buffers; writes F[2], F[3] and acc.
template <typename T>
ew_status tb2d_tune(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, T* acc, int nvec,
                    int64_t fstride, cudaStream_t st);
// advance from level L (F[*cur], F[*prv] = level L-1) to level N_t; tb > 0
// caps the steps per launch (and uses the default variant), tb == 0 uses the
// tuned variant.
template <typename T>
ew_status tb2d_advance(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, int* prv, int* cur,
                       int64_t L, T* acc, int nvec, int64_t fstride, int tb, cudaStream_t st);
template <typename T>
int tb2d_choice(const GridGeom& g, int nvec, int* B, int* TX, int* TY);
// row pitch of the time-level fields for the variant tb2d_advance will run
// (pitch2d(nx) for a TMA-staged one, else nx); call after tb2d_tune
template <typename T>
int64_t tb2d_field_pitch(const GridGeom& g, const FilterPlan& plan, const T* cdev, T* const* F, T* acc, int nvec,
                         int64_t fstride, int tb, cudaStream_t st);

// --- learned smoother as its composed 5x5x5 stencil (ew_smoother_comp.cu) ----
// built from one level's 432 weights (device); applies x += N(r) on FP32 3D fields
struct ComposedSmoother {
    std::vector<float> interior;  // the interior stencil (125 values)
    DeviceBuffer dev;             // the 64 class stencils (wall classes per axis)
    ew_status build(const float* weights_dev, cudaStream_t st);
    ew_status apply(const GridGeom& g, const float* r, float* x, cudaStream_t st) const;
};

// --- eigen-solver (ew_arnoldi.cu) ------------------------------------------
// S v for nvec vectors, routed by the caller: the batched eigen-solver gathers
// the filter applications of several solvers into one batched call
struct FilterHook {
    virtual ew_status apply(ew_grid* g, const ew_filter_params* p, const FilterPlan& plan, const void* vin, void* vout,
                            int nvec, cudaStream_t st) = 0;

   protected:
    ~FilterHook() = default;
};
ew_status filter_apply_any(ew_grid* g, const ew_filter_params* p, const FilterPlan& plan, const void* vin, void* vout,
                           int nvec, cudaStream_t st);
// ew_arnoldi_eigs without the ABI wrapper; hook (may be NULL) takes every filter application
ew_status arnoldi_eigs_impl(const ew_grid* grid, const ew_filter_params* params, const ew_eigs_params* ep,
                            const double* start_dev, double* lambda_host, double* vecs_dev, ew_eigs_report* rep,
                            cudaStream_t st, FilterHook* hook);
// ew_filter_apply_batched without the ABI wrapper; *variant (may be NULL; < 0: tune
// and store the choice) pins the tile variant across calls of different batch shapes
ew_status filter_apply_batched_impl(int nprob, const ew_grid* const* grids, const ew_filter_params* params,
                                    const void* const* v_in, void* const* v_out, const int* nvec, cudaStream_t stream,
                                    int* variant);

// --- reductions (ew_reduce.cu) ---------------------------------------------
// out[j] = sum_i x_j[i] * y_j[i] for nvec pairs of vectors (FP64 accumulate),
// partial sums in `part` (>= nvec * kReduceBlocks doubles), result on device.
constexpr int kReduceBlocks = 304;
template <typename T>
ew_status launch_dots(const T* x, const T* y, int64_t N, int nvec, double* part, double* out,
                      cudaStream_t st);
// out[j] = max_i |x_j[i] + s_j y_j[i]| (s on device) and max_i |y_j[i]|
template <typename T>
ew_status launch_resid_inf(const T* Lx, const T* x, int64_t N, int nvec, const double* lam2,
                           double* part, double* out_res, double* out_xinf, cudaStream_t st);
template <typename T>
ew_status launch_scale(T* x, int64_t N, int nvec, const double* s, cudaStream_t st);
// out = W^{e/2} in (e = +1 / -1) for nvec vectors: W the trapezoid weights of
// the active points (1/2 per Neumann wall coordinate); in == out allowed
template <typename T>
ew_status launch_wsqrt(const GridGeom& g, const T* in, T* out, int nvec, int e, cudaStream_t st);
// y += alpha x (FP32)
ew_status axpy_f(int64_t n, float alpha, const float* x, float* y, cudaStream_t st);
// y = a * x + y with device scalar: y_j -= s_j * x_j
template <typename T>
ew_status launch_diffnorm_sign(const T* xnew, const T* xold, int64_t N, const double* beta,
                               double* part, double* out, cudaStream_t st);

}  // namespace ew
