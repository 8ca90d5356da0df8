// ew_noalloc.cu -- the explicit wave-solve for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: plugins whose host application owns
// every device allocation (the library may not take memory behind its back),
// or real-time loops that must not enter the allocator, whose latency is
// unbounded.
// ew_filter_apply keeps its time levels in scratch it allocates on first use;
// this variant takes them from one file-scope device array instead, of a
// fixed size, which every GPU that loads the library holds until the process
// exits.  The caller still passes the input and output vectors.
//
// The array: the four time-level fields (up to kFieldBytes) followed by the
// filter weights (up to kWeightBytes).  Every call overwrites what it reads
// before reading it (the first step writes two levels, each later launch
// writes the next two, the weights are recomputed by a kernel), so nothing
// has to start at zero; but all calls share the array, so calls whose GPU
// work overlaps (other streams, other host threads) race on it.
#include <math.h>

#include <mutex>

#include "ew_internal.h"

namespace ew {

constexpr size_t kFieldBytes = (size_t)16 << 20;   // 16 MiB: four FP32 fields of 2^20 points
constexpr size_t kWeightBytes = (size_t)512 << 10; // 512 KiB of filter weights

static __device__ __align__(256) unsigned char g_noalloc_scratch[kFieldBytes + kWeightBytes];

// Host code must not use the array's name as an address (it names a host-side
// stand-in): the device address comes from cudaGetSymbolAddress, once per
// device, with that device current.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[128] = {nullptr};

static ew_status noalloc_scratch(void** out) {
    int dev = 0;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return set_error(EW_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return EW_OK;
}

// c_n = (2/T_f) sigma_n (cos(omega t^n) - alpha_d / 2), computed on the device
template <typename T>
__global__ void k_noalloc_weights(int64_t Nt, double Tf, double dt, double omega, double alpha_d, T* __restrict__ c) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= Nt; n += (int64_t)gridDim.x * blockDim.x) {
        double sigma = (n == 0 || n == Nt) ? 0.5 * dt : dt;
        c[n] = (T)(2.0 / Tf * sigma * (cos(omega * (double)n * dt) - 0.5 * alpha_d));
    }
}

template <typename T>
static ew_status noalloc_t(const ew_grid* g, const ew_filter_params* p, const FilterPlan& plan, const T* vin, T* vout,
                           cudaStream_t st) {
    const int64_t N = g->geom.N;
    if ((size_t)4 * wave_field_stride(g->geom) * sizeof(T) > kFieldBytes)
        return set_error(EW_EINVAL, "grid too large for ew_filter_apply_noalloc: at most " +
                                        std::to_string(kFieldBytes / (4 * sizeof(T))) +
                                        " points per time level in this precision (2D rows padded to 4 points)");
    if ((size_t)(plan.Nt + 1) * sizeof(T) > kWeightBytes)
        return set_error(EW_EINVAL, "too many time steps for ew_filter_apply_noalloc: at most " +
                                        std::to_string(kWeightBytes / sizeof(T) - 1));
    void* base = nullptr;
    EW_TRY(noalloc_scratch(&base));
    T* fields = (T*)base;
    T* cdev = (T*)((char*)base + kFieldBytes);
    int blocks = (int)std::min<int64_t>((plan.Nt + 256) / 256, 1024);
    k_noalloc_weights<T><<<blocks, 256, 0, st>>>(plan.Nt, plan.Tf, plan.dt, plan.omega, plan.alpha_d, cdev);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    // a fixed temporal depth: the autotuner (which times candidates with CUDA
    // events) is not used on this path
    if (p->temporal_block < 0) return set_error(EW_EINVAL, "temporal_block < 0");
    int tb = p->temporal_block > 0 ? p->temporal_block : 4;
    return explicit_wave_solve<T>(g->geom, plan, cdev, vin, vout, 1, fields, tb, st);
}

}  // namespace ew

using namespace ew;

extern "C" ew_status ew_filter_apply_noalloc(const ew_grid* grid, const ew_filter_params* params, const void* v_in,
                                             void* v_out, cudaStream_t stream) try {
    clear_error();
    if (!grid || !params || !v_in || !v_out) return set_error(EW_EINVAL, "null argument");
    int dev = -1;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    if (grid->device >= 0 && grid->device != dev) return set_error(EW_EINVAL, "grid was created on another device");
    if (params->scheme != EW_EXPLICIT)
        return set_error(EW_EUNSUPPORTED, "ew_filter_apply_noalloc runs the explicit scheme only");
    if (grid->geom.map) return set_error(EW_EUNSUPPORTED, "ew_filter_apply_noalloc takes box grids only");
    if (grid->prec == EW_FP32X2) return set_error(EW_EUNSUPPORTED, "ew_filter_apply_noalloc: FP32 or FP64 grids only");
    const size_t bytes = (size_t)grid->geom.N * (grid->prec == EW_FP32 ? 4 : 8);
    const char* a = (const char*)v_in;
    const char* b = (const char*)v_out;
    if (a < b + bytes && b < a + bytes) return set_error(EW_EINVAL, "v_in and v_out overlap");
    FilterPlan plan;
    EW_TRY(plan_filter(grid->geom, params, &plan, /*with_weights=*/false));
    if (grid->prec == EW_FP32) return noalloc_t<float>(grid, params, plan, (const float*)v_in, (float*)v_out, stream);
    return noalloc_t<double>(grid, params, plan, (const double*)v_in, (double*)v_out, stream);
} catch (...) {
    return abi_exception();
}
