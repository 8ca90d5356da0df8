// ew_eigs_batched.cu -- eigen-solves of many independent problems with their
// filter applications batched (no counterpart in the paper: the batching of
// many box problems of uneven size into one launch sequence).
//
// Each problem runs the block Krylov-Schur solver of ew_arnoldi_eigs
// (ew_arnoldi.cu) on a host thread and a stream of its own.  The solver's
// filter applications go through a hook: a problem that asks for S X waits
// until every unfinished problem has asked too (or finished), and then one
// ew_filter_apply_batched call runs all of them together on a batch stream.
// Its graph is kept per batch, so the rounds of an eigen-solve only replay it;
// the tile variant, tuned on the first round, stays pinned for the rest.
// Everything between two rounds (orthogonalisation, the small eigenproblems,
// Rayleigh quotients) runs per problem, concurrently, on the problems' own
// streams.  Ordering between the streams is by events: the batch stream
// waits for each problem's inputs, each problem's stream waits for the batch.
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ew_internal.h"

namespace ew {

class Rendezvous {
   public:
    explicit Rendezvous(int n) : live_(n), req_(n), has_(n, false), result_(n, EW_OK), msg_(n), ready_(n, nullptr) {}
    ~Rendezvous() {
        for (auto e : ready_)
            if (e) cudaEventDestroy(e);
        if (done_) cudaEventDestroy(done_);
        if (bst_) cudaStreamDestroy(bst_);
    }
    ew_status init() {
        EW_CUDA_TRY(cudaStreamCreateWithFlags(&bst_, cudaStreamNonBlocking));
        EW_CUDA_TRY(cudaEventCreateWithFlags(&done_, cudaEventDisableTiming));
        for (auto& e : ready_) EW_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return EW_OK;
    }

    // problem `slot` asks for vout = S vin; returns when the batched call that
    // includes it has been queued (the problem's stream waits for it)
    ew_status submit(int slot, ew_grid* g, const ew_filter_params* p, const void* vin, void* vout, int nvec,
                     cudaStream_t st) {
        std::unique_lock<std::mutex> lk(mu_);
        req_[slot] = Req{g, p, vin, vout, nvec, st};
        cudaError_t e = cudaEventRecord(ready_[slot], st);
        if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
        has_[slot] = true;
        ++pending_;
        const uint64_t my = gen_;
        if (pending_ == live_) run_locked();
        else cv_.wait(lk, [&] { return gen_ != my; });
        if (result_[slot] != EW_OK) return set_error(result_[slot], msg_[slot]);
        return EW_OK;
    }

    // problem `slot` has finished (or failed): the others no longer wait for it
    void leave() {
        std::lock_guard<std::mutex> lk(mu_);
        --live_;
        if (live_ > 0 && pending_ == live_) run_locked();
    }

    int rounds() const { return rounds_; }

   private:
    struct Req {
        ew_grid* g = nullptr;
        const ew_filter_params* p = nullptr;
        const void* vin = nullptr;
        void* vout = nullptr;
        int nvec = 0;
        cudaStream_t st = nullptr;
    };

    // one batched call per group of requests that can share a launch (same
    // precision and order; ew_filter_apply_batched runs any other mix, e.g. a
    // refinement's FP64 images, one problem at a time)
    void run_locked() {
        std::vector<int> slots;
        ew_status s = EW_OK;
        for (int q = 0; q < (int)has_.size(); ++q) {
            if (!has_[q]) continue;
            slots.push_back(q);
            if (s == EW_OK) {
                cudaError_t e = cudaStreamWaitEvent(bst_, ready_[q], 0);
                if (e != cudaSuccess) s = cuda_error(e, "cudaStreamWaitEvent");
            }
        }
        std::vector<bool> taken(slots.size(), false);
        for (size_t i = 0; i < slots.size() && s == EW_OK; ++i) {
            if (taken[i]) continue;
            const ew_grid* g0 = req_[slots[i]].g;
            const int gkey = (int)g0->prec * 16 + g0->geom.order;
            std::vector<const ew_grid*> grids;
            std::vector<ew_filter_params> params;
            std::vector<const void*> vin;
            std::vector<void*> vout;
            std::vector<int> nvec;
            for (size_t j = i; j < slots.size(); ++j) {
                const Req& r = req_[slots[j]];
                if (taken[j] || (int)r.g->prec * 16 + r.g->geom.order != gkey) continue;
                taken[j] = true;
                grids.push_back(r.g);
                params.push_back(*r.p);
                vin.push_back(r.vin);
                vout.push_back(r.vout);
                nvec.push_back(r.nvec);
            }
            int& pin = variant_[gkey];  // tuned on a group's first round, then kept
            if (!pin_set_[gkey]) pin = -1, pin_set_[gkey] = true;
            s = filter_apply_batched_impl((int)grids.size(), grids.data(), params.data(), vin.data(), vout.data(),
                                          nvec.data(), bst_, &pin);
        }
        std::string msg = s == EW_OK ? std::string() : std::string(ew_last_error());
        if (s == EW_OK) {
            cudaError_t e = cudaEventRecord(done_, bst_);
            if (e != cudaSuccess) s = cuda_error(e, "cudaEventRecord"), msg = ew_last_error();
        }
        for (int q : slots) {
            if (s == EW_OK) {
                cudaError_t e = cudaStreamWaitEvent(req_[q].st, done_, 0);
                if (e != cudaSuccess) s = cuda_error(e, "cudaStreamWaitEvent"), msg = ew_last_error();
            }
        }
        for (int q : slots) {
            result_[q] = s;
            msg_[q] = msg;
            has_[q] = false;
        }
        pending_ = 0;
        ++rounds_;
        ++gen_;
        cv_.notify_all();
    }

    std::mutex mu_;
    std::condition_variable cv_;
    int live_;
    int pending_ = 0;
    int rounds_ = 0;
    uint64_t gen_ = 0;
    std::map<int, int> variant_;   // tile variant per (precision, order) group: tuned on its first round, then pinned
    std::map<int, bool> pin_set_;
    std::vector<Req> req_;
    std::vector<bool> has_;
    std::vector<ew_status> result_;
    std::vector<std::string> msg_;
    std::vector<cudaEvent_t> ready_;
    cudaEvent_t done_ = nullptr;
    cudaStream_t bst_ = nullptr;
};

// the hook of one problem's solver
struct ProblemHook final : FilterHook {
    Rendezvous* rv;
    int slot;
    ew_status apply(ew_grid* g, const ew_filter_params* p, const FilterPlan&, const void* vin, void* vout, int nvec,
                    cudaStream_t st) override {
        return rv->submit(slot, g, p, vin, vout, nvec, st);
    }
};

}  // namespace ew

using namespace ew;

extern "C" ew_status ew_arnoldi_eigs_batched(int nprob, const ew_grid* const* grids, const ew_filter_params* params,
                                             const ew_eigs_params* eigs, double* const* lambda_host,
                                             double* const* vecs_dev, ew_eigs_report* reports, ew_status* statuses,
                                             int* rounds_host, cudaStream_t stream) try {
    clear_error();
    if (nprob < 1 || !grids || !params || !eigs || !lambda_host) return set_error(EW_EINVAL, "null argument");
    // one host thread per problem (each solver blocks at the rendezvous until the round's batched call)
    if (nprob > 1024) return set_error(EW_EINVAL, "ew_arnoldi_eigs_batched takes at most 1024 problems");
    for (int q = 0; q < nprob; ++q)
        if (!grids[q] || !lambda_host[q]) return set_error(EW_EINVAL, "null grid or lambda pointer");
    int dev = -1;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    Rendezvous rv(nprob);
    EW_TRY(rv.init());
    // the problems' streams start after the work already queued on `stream`
    cudaEvent_t start = nullptr;
    EW_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    struct EventGuard {
        cudaEvent_t e;
        ~EventGuard() { cudaEventDestroy(e); }
    } start_guard{start};
    EW_CUDA_TRY(cudaEventRecord(start, stream));
    std::vector<cudaStream_t> streams((size_t)nprob, nullptr);
    struct StreamsGuard {
        std::vector<cudaStream_t>& s;
        ~StreamsGuard() {
            for (auto x : s)
                if (x) cudaStreamDestroy(x);
        }
    } streams_guard{streams};
    for (auto& s : streams) {
        EW_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        EW_CUDA_TRY(cudaStreamWaitEvent(s, start, 0));
    }
    std::vector<ew_status> st((size_t)nprob, EW_OK);
    std::vector<std::string> msg((size_t)nprob);
    std::vector<ProblemHook> hooks((size_t)nprob);
    std::vector<std::thread> threads;
    threads.reserve((size_t)nprob);
    for (int q = 0; q < nprob; ++q) {
        hooks[q].rv = &rv;
        hooks[q].slot = q;
        threads.emplace_back([&, q]() {
            ew_status s = EW_OK;
            try {
                if (cudaSetDevice(dev) != cudaSuccess) {
                    s = set_error(EW_ECUDA, "cudaSetDevice failed in a problem thread");
                } else {
                    ew_eigs_report rep;
                    std::memset(&rep, 0, sizeof(rep));
                    s = arnoldi_eigs_impl(grids[q], &params[q], &eigs[q], nullptr, lambda_host[q],
                                          vecs_dev ? vecs_dev[q] : nullptr, &rep, streams[q], &hooks[q]);
                    if (reports) reports[q] = rep;
                }
            } catch (...) {
                s = abi_exception();
            }
            st[q] = s;
            if (s != EW_OK) msg[q] = ew_last_error();
            rv.leave();
        });
    }
    for (auto& t : threads) t.join();
    if (rounds_host) *rounds_host = rv.rounds();
    ew_status first = EW_OK;
    for (int q = 0; q < nprob; ++q) {
        if (statuses) statuses[q] = st[q];
        if (first == EW_OK && st[q] != EW_OK) {
            first = st[q];
            set_error(st[q], "problem " + std::to_string(q) + ": " + msg[q]);
        }
    }
    return first;
} catch (...) {
    return abi_exception();
}
