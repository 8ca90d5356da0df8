// ew_hostio.cu -- the wave-solve (Algorithm matVec) from and to host memory,
// with the copies overlapped with the filter applications.
//
// The nvec vectors are cut into chunks; chunk k is copied to the device on a
// copy stream, filtered on the caller's stream and copied back on a second
// copy stream, so while chunk k is filtered chunk k + 1 arrives and chunk k - 1
// leaves.  Two device buffers per direction alternate between chunks; a
// buffer is refilled only after the filter application (input) or the copy
// back (output) that used it two chunks earlier, which the events below
// order.  The results are those of ew_filter_apply on the same vectors bit
// for bit: every tile form of the wave-solve performs the same operations on
// each point, whatever the number of vectors in a launch.
#include <algorithm>

#include "ew_internal.h"

namespace ew {

namespace {

// default chunking: chunks of at least four vectors (the wave-solve kernels
// lose efficiency on fewer), at most four chunks
int default_chunk(int nvec) {
    const int nch = std::max(1, std::min(4, nvec / 4));
    return (nvec + nch - 1) / nch;
}

// a CUDA stream or event that is destroyed on every exit path; destroying
// them while work is pending is allowed (the resources go once it completes)
struct StreamH {
    cudaStream_t s = nullptr;
    ~StreamH() {
        if (s) cudaStreamDestroy(s);
    }
};
struct EventH {
    cudaEvent_t e = nullptr;
    ~EventH() {
        if (e) cudaEventDestroy(e);
    }
};

}  // namespace

}  // namespace ew

using namespace ew;

extern "C" ew_status ew_filter_apply_host(const ew_grid* grid, const ew_filter_params* params, const void* v_in_host,
                                          void* v_out_host, int nvec, int chunk, cudaStream_t stream) try {
    clear_error();
    EW_TRY(check_grid(grid));
    if (!params) return set_error(EW_EINVAL, "params is NULL");
    if (!v_in_host || !v_out_host) return set_error(EW_EINVAL, "null vector pointer");
    if (nvec < 1 || nvec > 65535) return set_error(EW_EINVAL, "nvec must be in [1, 65535]");
    if (chunk < 0) return set_error(EW_EINVAL, "chunk must be >= 0");
    const int64_t N = grid->geom.N;
    const size_t es = elem_size(grid);
    const size_t bytes = (size_t)nvec * N * es;
    const char* hin = (const char*)v_in_host;
    char* hout = (char*)v_out_host;
    if (hin < hout + bytes && hout < hin + bytes) return set_error(EW_EINVAL, "v_in and v_out overlap");
    FilterPlan plan;
    EW_TRY(plan_filter(grid->geom, params, &plan));
    ew_grid* g = const_cast<ew_grid*>(grid);
    const int c = chunk > 0 ? std::min(chunk, nvec) : default_chunk(nvec);
    const int nch = (nvec + c - 1) / c;
    const size_t cb = (size_t)c * N * es;  // bytes of one chunk buffer
    const int nbuf = nch > 1 ? 2 : 1;
    EW_TRY(g->hostio.reserve(2 * nbuf * cb));
    char* din[2] = {(char*)g->hostio.ptr, (char*)g->hostio.ptr + cb};
    char* dout[2] = {(char*)g->hostio.ptr + nbuf * cb, (char*)g->hostio.ptr + (nbuf + 1) * cb};

    StreamH h2d, d2h;
    EW_CUDA_TRY(cudaStreamCreateWithFlags(&h2d.s, cudaStreamNonBlocking));
    EW_CUDA_TRY(cudaStreamCreateWithFlags(&d2h.s, cudaStreamNonBlocking));
    EventH start, end, in_ready[2], done[2], drained[2];
    for (EventH* e : {&start, &end, &in_ready[0], &in_ready[1], &done[0], &done[1], &drained[0], &drained[1]})
        EW_CUDA_TRY(cudaEventCreateWithFlags(&e->e, cudaEventDisableTiming));
    // everything after the work already queued on the caller's stream
    EW_CUDA_TRY(cudaEventRecord(start.e, stream));
    EW_CUDA_TRY(cudaStreamWaitEvent(h2d.s, start.e, 0));
    EW_CUDA_TRY(cudaStreamWaitEvent(d2h.s, start.e, 0));
    for (int k = 0; k < nch; ++k) {
        const int s = k % nbuf;
        const int nv = std::min(c, nvec - k * c);
        const size_t nb = (size_t)nv * N * es;
        // input buffer s: free once the filter application of chunk k - 2 has read it
        if (k >= nbuf) EW_CUDA_TRY(cudaStreamWaitEvent(h2d.s, done[s].e, 0));
        EW_CUDA_TRY(cudaMemcpyAsync(din[s], hin + (size_t)k * cb, nb, cudaMemcpyHostToDevice, h2d.s));
        EW_CUDA_TRY(cudaEventRecord(in_ready[s].e, h2d.s));
        // filter on the caller's stream once the input is in and output buffer s drained
        EW_CUDA_TRY(cudaStreamWaitEvent(stream, in_ready[s].e, 0));
        if (k >= nbuf) EW_CUDA_TRY(cudaStreamWaitEvent(stream, drained[s].e, 0));
        EW_TRY(filter_apply_any(g, params, plan, din[s], dout[s], nv, stream));
        EW_CUDA_TRY(cudaEventRecord(done[s].e, stream));
        EW_CUDA_TRY(cudaStreamWaitEvent(d2h.s, done[s].e, 0));
        EW_CUDA_TRY(cudaMemcpyAsync(hout + (size_t)k * cb, dout[s], nb, cudaMemcpyDeviceToHost, d2h.s));
        EW_CUDA_TRY(cudaEventRecord(drained[s].e, d2h.s));
    }
    // later work on the caller's stream sees the outputs in host memory
    EW_CUDA_TRY(cudaEventRecord(end.e, d2h.s));
    EW_CUDA_TRY(cudaStreamWaitEvent(stream, end.e, 0));
    return EW_OK;
} catch (...) {
    return abi_exception();
}
