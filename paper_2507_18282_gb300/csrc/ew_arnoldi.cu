// ew_arnoldi.cu -- matrix-free block Krylov-Schur eigen-solver on S (Arnoldi
// section: Algorithm arnoldi for the basis, the restart of Algorithms IRAM /
// KrylovSchur), driven from the host with the basis in FP64 device memory.
//
//   S V_m = V_{m+b} H        (block Arnoldi relation, b vectors per expansion)
//
// Expansion: W = S V_last (one wave-solve per vector, in the grid precision),
// classical Gram-Schmidt applied twice against the whole basis (FP64 Gram and
// update kernels), then Cholesky-QR applied twice for the new block.
// Rayleigh-Ritz: the projected matrix H_m (symmetric because S is) is
// diagonalised on the host by cyclic Jacobi.  The wanted Ritz pairs are the
// n_wanted largest algebraic Ritz values (the peak of the filter, where
// lambda is near omega).  A pair has converged when its Ritz residual
// ||S x - theta x|| = ||R E^T y|| is below tol.  Thick restart: keep the best
// k Ritz vectors and the residual block (Krylov-Schur form).
//
// Stage 2 (Arnoldi section): lambda from the Rayleigh quotient of L_h
// (eq. simpleRayleighQuotient; on grids with Neumann faces the weighted form
// eq. discreteRayleighQuotient) and the eig-res metric.  With refine_fp64 on an
// FP32 grid the result is refined in FP64: mixed-precision iterative
// refinement of the invariant subspace (refine_ir) or a second Krylov-Schur
// run with FP64 wave-solves.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <memory>
#include <vector>

#include "ew_internal.h"

namespace ew {

ew_status gram(int64_t N, const double* A, int64_t lda, int ma, const double* B, int64_t ldb, int mb,
               double* part, double* C, cudaStream_t st);
size_t gram_part_doubles(int ma, int mb);
ew_status update(int64_t N, const double* A, int64_t lda, int ma, const double* Bin, int64_t ldb, int mb,
                 const double* M, double alpha, double beta, double* Out, int64_t ldo, cudaStream_t st);
template <typename S, typename D>
ew_status convert(int64_t n, const S* x, D* y, cudaStream_t st);
ew_status splitmix_uniform(int64_t n, uint64_t seed, double* out, cudaStream_t st);
ew_status filter_apply_any(ew_grid* g, const ew_filter_params* p, const FilterPlan& plan, const void* vin,
                           void* vout, int nvec, cudaStream_t st);
ew_status rayleigh_any(ew_grid* g, const void* phi, int nvec, double* lam, double* res, cudaStream_t st);

// ---------------------------------------------------------------------------
// cyclic Jacobi for a small symmetric matrix (row-major n x n, destroyed).
// Eigenvalues in w, eigenvectors in the columns of V (row-major).
// ---------------------------------------------------------------------------
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& w) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double fro = 0.0;
    for (double a : A) fro += a * a;
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += 2.0 * A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (sqrt(off) <= 1e-15 * fro || fro == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (fabs(apq) <= 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                // rotation that zeroes A[p][q]: tan = t, cos = c, sin = s
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // V <- V J
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Cholesky of a small SPD matrix (row-major), upper factor R with G = R^T R.
static bool cholesky_upper(int n, const std::vector<double>& G, std::vector<double>& R) {
    R.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = G[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= R[(size_t)k * n + j] * R[(size_t)k * n + j];
        if (!(d > 0.0)) return false;
        double rjj = sqrt(d);
        R[(size_t)j * n + j] = rjj;
        for (int i = j + 1; i < n; ++i) {
            double s = G[(size_t)j * n + i];
            for (int k = 0; k < j; ++k) s -= R[(size_t)k * n + j] * R[(size_t)k * n + i];
            R[(size_t)j * n + i] = s / rjj;
        }
    }
    return true;
}

// inverse of an upper-triangular matrix (row-major)
static void inv_upper(int n, const std::vector<double>& R, std::vector<double>& Ri) {
    Ri.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        Ri[(size_t)j * n + j] = 1.0 / R[(size_t)j * n + j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= j; ++k) s += R[(size_t)i * n + k] * Ri[(size_t)k * n + j];
            Ri[(size_t)i * n + j] = -s / R[(size_t)i * n + i];
        }
    }
}

// ---------------------------------------------------------------------------
// one Krylov-Schur run
// ---------------------------------------------------------------------------
// S applied to nvec vectors: filter_apply_any, or through the hook of a
// caller that gathers the applications of several solvers (the batched
// eigen-solver, ew_eigs_batched.cu)
static ew_status apply_filter(FilterHook* hook, ew_grid* g, const ew_filter_params* p, const FilterPlan& plan,
                              const void* vin, void* vout, int nvec, cudaStream_t st) {
    if (hook) return hook->apply(g, p, plan, vin, vout, nvec, st);
    return filter_apply_any(g, p, plan, vin, vout, nvec, st);
}

struct KSRun {
    ew_grid* g;
    const ew_filter_params* p;
    FilterHook* hook = nullptr;
    FilterPlan plan;
    int64_t N;
    int b, m, nw;
    double tol;
    int max_ws;
    cudaStream_t st;
    // device
    double* V = nullptr;     // N x (m + 2b)
    double* W = nullptr;     // N x b
    void* fin = nullptr;     // filter input (grid precision), N x b
    void* fout = nullptr;    // filter output
    double* symtmp = nullptr;  // FP64 grids with Neumann faces: W^{-1/2} X, N x b
    double* part = nullptr;  // gram partials
    double* dC = nullptr;    // small device matrices
    // host
    double* hC = nullptr;    // pinned small matrix staging
    std::vector<double> H;   // (m + 3b) x (m + 2b), row-major, ldh = m + 2b
    int ldh = 0, mcur = 0;
    int wave_solves = 0, restarts = 0;
    bool lock = false;  // lock converged wanted pairs at restarts
    std::vector<void*> allocs;

    ~KSRun() {
        for (void* a : allocs) cudaFree(a);
        if (hC) cudaFreeHost(hC);
    }
    ew_status alloc(void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(EW_ENOMEM, "Krylov workspace allocation of " + std::to_string(bytes) + " bytes failed");
        }
        allocs.push_back(*p);
        return EW_OK;
    }
    double& h(int i, int j) { return H[(size_t)i * ldh + j]; }

    ew_status setup() {
        size_t es = g->prec == EW_FP32 ? 4 : 8;
        // a restart may leave mcur off a multiple of b, so the basis can reach m + 2b - 1 columns
        EW_TRY(alloc((void**)&V, sizeof(double) * (size_t)N * (m + 2 * b)));
        EW_TRY(alloc((void**)&W, sizeof(double) * (size_t)N * b));
        if (g->prec == EW_FP32) {
            EW_TRY(alloc(&fin, es * (size_t)N * b));
            EW_TRY(alloc(&fout, es * (size_t)N * b));
        } else if (weighted_sums(g->geom)) {
            EW_TRY(alloc((void**)&symtmp, sizeof(double) * (size_t)N * b));
        }
        int wmax = m + 3 * b;
        EW_TRY(alloc((void**)&part, sizeof(double) * gram_part_doubles(wmax, wmax)));
        EW_TRY(alloc((void**)&dC, sizeof(double) * (size_t)wmax * wmax));
        EW_CUDA_TRY(cudaMallocHost((void**)&hC, sizeof(double) * (size_t)wmax * wmax));
        ldh = m + 2 * b;
        H.assign((size_t)(m + 3 * b) * ldh, 0.0);
        return EW_OK;
    }

    // C (host, row-major ma x mb) = A^T B
    ew_status gram_host(const double* A, int ma, const double* B, int mb, std::vector<double>& C) {
        EW_TRY(gram(N, A, N, ma, B, N, mb, part, dC, st));
        EW_CUDA_TRY(cudaMemcpyAsync(hC, dC, sizeof(double) * ma * mb, cudaMemcpyDeviceToHost, st));
        EW_CUDA_TRY(cudaStreamSynchronize(st));
        C.assign(hC, hC + (size_t)ma * mb);
        return EW_OK;
    }
    // Out = beta Bin + alpha A M  (M host row-major ma x mb)
    ew_status update_host(const double* A, int ma, const double* Bin, int mb, const std::vector<double>& M,
                          double alpha, double beta, double* Out) {
        // the staging buffer may still feed the previous copy
        EW_CUDA_TRY(cudaStreamSynchronize(st));
        std::memcpy(hC, M.data(), sizeof(double) * ma * mb);
        EW_CUDA_TRY(cudaMemcpyAsync(dC, hC, sizeof(double) * ma * mb, cudaMemcpyHostToDevice, st));
        return update(N, A, N, ma, Bin, N, mb, dC, alpha, beta, Out, N, st);
    }

    // W = S X (b vectors).  On a grid with Neumann faces S is symmetric in the
    // trapezoid-weighted sums only, so the run works with the similar operator
    // W^{1/2} S W^{-1/2}, symmetric in the plain sums that the Gram kernels and
    // the Rayleigh-Ritz step use (same eigenvalues; eigenvectors W^{1/2} phi).
    ew_status apply_S(const double* X) {
        const bool sym = weighted_sums(g->geom);
        if (g->prec == EW_FP32) {
            const double* Xs = X;
            if (sym) {  // W is free until the result lands in it
                EW_TRY(launch_wsqrt<double>(g->geom, X, W, b, -1, st));
                Xs = W;
            }
            EW_TRY((convert<double, float>(N * b, Xs, (float*)fin, st)));
            EW_TRY(apply_filter(hook, g, p, plan, fin, fout, b, st));
            EW_TRY((convert<float, double>(N * b, (const float*)fout, W, st)));
        } else if (sym) {
            EW_TRY(launch_wsqrt<double>(g->geom, X, symtmp, b, -1, st));
            EW_TRY(apply_filter(hook, g, p, plan, symtmp, W, b, st));
        } else {
            EW_TRY(apply_filter(hook, g, p, plan, X, W, b, st));
        }
        if (sym) EW_TRY(launch_wsqrt<double>(g->geom, W, W, b, 1, st));
        wave_solves += b;
        return EW_OK;
    }

    // orthonormalise the b columns of Y (device) against nothing: Y = Q R, R host upper b x b
    ew_status cholqr2(double* Y, std::vector<double>& R, bool* ok) {
        std::vector<double> G, R1, R2, Ri;
        *ok = true;
        EW_TRY(gram_host(Y, b, Y, b, G));
        if (!cholesky_upper(b, G, R1)) {
            *ok = false;
            return EW_OK;
        }
        inv_upper(b, R1, Ri);
        EW_TRY(update_host(Y, b, nullptr, b, Ri, 1.0, 0.0, Y));
        EW_TRY(gram_host(Y, b, Y, b, G));
        if (!cholesky_upper(b, G, R2)) {
            *ok = false;
            return EW_OK;
        }
        inv_upper(b, R2, Ri);
        EW_TRY(update_host(Y, b, nullptr, b, Ri, 1.0, 0.0, Y));
        R.assign((size_t)b * b, 0.0);  // R = R2 R1
        for (int i = 0; i < b; ++i)
            for (int j = i; j < b; ++j) {
                double s = 0.0;
                for (int k = i; k <= j; ++k) s += R2[(size_t)i * b + k] * R1[(size_t)k * b + j];
                R[(size_t)i * b + j] = s;
            }
        return EW_OK;
    }

    // Cholesky-QR applied twice to n columns of Y (no R returned)
    ew_status orthonormalise(double* Y, int n, bool* ok) {
        std::vector<double> G, R, Ri;
        *ok = true;
        for (int pass = 0; pass < 2; ++pass) {
            EW_TRY(gram_host(Y, n, Y, n, G));
            if (!cholesky_upper(n, G, R)) {
                *ok = false;
                return EW_OK;
            }
            inv_upper(n, R, Ri);
            EW_TRY(update_host(Y, n, nullptr, n, Ri, 1.0, 0.0, Y));
        }
        return EW_OK;
    }

    // SVQB: orthonormalise n columns of Y through the eigen-decomposition of
    // their Gram matrix, dropping directions whose norm is below 1e-12 of the
    // largest (twice, for stability).  The kept columns are packed to the
    // front of Y; *rank receives their number.
    ew_status svqb(double* Y, int n, int* rank) {
        int cur = n;
        for (int pass = 0; pass < 2 && cur > 0; ++pass) {
            std::vector<double> G, U, d;
            EW_TRY(gram_host(Y, cur, Y, cur, G));
            jacobi_eig(cur, G, U, d);
            double dmax = 0.0;
            for (double x : d) dmax = std::max(dmax, x);
            std::vector<int> keep;
            for (int i = 0; i < cur; ++i)
                if (d[i] > 1e-24 * dmax && d[i] > 0.0) keep.push_back(i);
            int r = (int)keep.size();
            std::vector<double> M((size_t)cur * r);
            for (int row = 0; row < cur; ++row)
                for (int c = 0; c < r; ++c) M[(size_t)row * r + c] = U[(size_t)row * cur + keep[c]] / sqrt(d[keep[c]]);
            if (r > 0) EW_TRY(update_host(Y, cur, nullptr, r, M, 1.0, 0.0, Y));
            cur = r;
        }
        *rank = cur;
        return EW_OK;
    }

    // start block: columns 0..b-1 of V, orthonormalised
    // start_dev: a caller's block (grid variables) or, with sym_vars, one
    // already in the variables of the symmetrised operator
    ew_status start(const double* start_dev, uint64_t seed, bool sym_vars = false) {
        if (start_dev && weighted_sums(g->geom) && !sym_vars)
            EW_TRY(launch_wsqrt<double>(g->geom, start_dev, V, b, 1, st));
        else if (start_dev)
            EW_CUDA_TRY(cudaMemcpyAsync(V, start_dev, sizeof(double) * (size_t)N * b, cudaMemcpyDeviceToDevice, st));
        else
            EW_TRY(splitmix_uniform(N * b, seed, V, st));
        std::vector<double> R;
        bool ok = false;
        EW_TRY(cholqr2(V, R, &ok));
        if (!ok) return set_error(EW_EINVAL, "start block is rank deficient");
        mcur = 0;
        return EW_OK;
    }

    // one block expansion: S V[:, mcur:mcur+b] -> new block V[:, mcur+b : mcur+2b]
    ew_status expand() {
        const int nb = mcur + b;  // basis columns present
        EW_TRY(apply_S(V + (size_t)mcur * N));
        std::vector<double> C1, C2;
        EW_TRY(gram_host(V, nb, W, b, C1));
        EW_TRY(update_host(V, nb, W, b, C1, -1.0, 1.0, W));
        EW_TRY(gram_host(V, nb, W, b, C2));
        EW_TRY(update_host(V, nb, W, b, C2, -1.0, 1.0, W));
        for (int i = 0; i < nb; ++i)
            for (int j = 0; j < b; ++j) h(i, mcur + j) = C1[(size_t)i * b + j] + C2[(size_t)i * b + j];
        std::vector<double> R;
        bool ok = false;
        EW_TRY(cholqr2(W, R, &ok));
        if (!ok) return set_error(EW_EBREAKDOWN, "Krylov breakdown: the new block is rank deficient");
        for (int i = 0; i < b; ++i)
            for (int j = 0; j < b; ++j) h(nb + i, mcur + j) = R[(size_t)i * b + j];
        EW_CUDA_TRY(cudaMemcpyAsync(V + (size_t)nb * N, W, sizeof(double) * (size_t)N * b, cudaMemcpyDeviceToDevice, st));
        mcur += b;
        return EW_OK;
    }

    // Rayleigh-Ritz on H_m: theta (descending), Y (row-major mcur x mcur), residual norms
    void ritz(std::vector<double>& theta, std::vector<double>& Y, std::vector<double>& resid) {
        int n = mcur;
        std::vector<double> A((size_t)n * n), Vv, w;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = 0.5 * (h(i, j) + h(j, i));
        jacobi_eig(n, A, Vv, w);
        std::vector<int> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int a, int c) { return w[a] > w[c]; });
        theta.resize(n);
        Y.assign((size_t)n * n, 0.0);
        for (int c = 0; c < n; ++c) {
            theta[c] = w[ord[c]];
            for (int r = 0; r < n; ++r) Y[(size_t)r * n + c] = Vv[(size_t)r * n + ord[c]];
        }
        resid.assign(n, 0.0);
        for (int c = 0; c < n; ++c) {
            double s2 = 0.0;
            for (int i = 0; i < b; ++i) {
                double s = 0.0;
                for (int r = 0; r < n; ++r) s += h(n + i, r) * Y[(size_t)r * n + c];
                s2 += s * s;
            }
            resid[c] = sqrt(s2);
        }
    }

    // thick restart keeping k Ritz vectors and the residual block; with `lock`,
    // the wanted pairs whose residual is below tol are locked: their coupling to
    // the residual block (of norm below tol) is set to zero, so the next
    // Rayleigh-Ritz steps keep their vectors and values as they are
    ew_status restart(int k, const std::vector<double>& theta, const std::vector<double>& Y,
                      const std::vector<double>& resid) {
        int n = mcur;
        std::vector<double> Yk((size_t)n * k);
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < k; ++c) Yk[(size_t)r * k + c] = Y[(size_t)r * n + c];
        std::vector<double> coup((size_t)b * k, 0.0);
        for (int i = 0; i < b; ++i)
            for (int c = 0; c < k; ++c) {
                if (lock && c < nw && resid[c] <= tol) continue;  // locked: no coupling
                double s = 0.0;
                for (int r = 0; r < n; ++r) s += h(n + i, r) * Y[(size_t)r * n + c];
                coup[(size_t)i * k + c] = s;
            }
        EW_TRY(update_host(V, n, nullptr, k, Yk, 1.0, 0.0, V));  // V[:, :k] = V[:, :n] Y_k (in place)
        EW_CUDA_TRY(cudaMemcpyAsync(V + (size_t)k * N, V + (size_t)n * N, sizeof(double) * (size_t)N * b,
                                    cudaMemcpyDeviceToDevice, st));
        std::fill(H.begin(), H.end(), 0.0);
        for (int c = 0; c < k; ++c) h(c, c) = theta[c];
        for (int i = 0; i < b; ++i)
            for (int c = 0; c < k; ++c) h(k + i, c) = coup[(size_t)i * k + c];
        mcur = k;
        ++restarts;
        return EW_OK;
    }

    // run until the nw wanted pairs converge or the budget is spent; the
    // converged Ritz vectors end up in V[:, :nconv] (sorted by theta)
    ew_status run(std::vector<double>& theta_out, int* nconv) {
        std::vector<double> theta, Y, resid;
        for (;;) {
            while (mcur < m) EW_TRY(expand());
            ritz(theta, Y, resid);
            int nc = 0;
            while (nc < nw && resid[nc] <= tol) ++nc;
            if (getenv("EW_KS_LOG")) {
                fprintf(stderr, "[ew ks] %s b=%d m=%d ws=%d restarts=%d conv=%d | theta/resid:",
                        g->prec == EW_FP32 ? "fp32" : "fp64", b, mcur, wave_solves, restarts, nc);
                for (int c = 0; c < std::min(nw + 8, mcur); ++c) fprintf(stderr, " %.9f/%.1e", theta[c], resid[c]);
                fprintf(stderr, "\n");
            }
            bool done = nc >= nw || wave_solves + b > max_ws;
            if (done) {
                // rotate the whole basis into Ritz vectors (descending theta): the
                // wanted ones first, the rest serve the refinement as guard vectors
                EW_TRY(update_host(V, mcur, nullptr, mcur, Y, 1.0, 0.0, V));
                theta_out.assign(theta.begin(), theta.begin() + mcur);
                *nconv = nc;
                return EW_OK;
            }
            int k = std::max(nw, std::min(mcur - b, nw + (mcur - nw) / 2));
            EW_TRY(restart(k, theta, Y, resid));
        }
    }
};

// Trapezoid sum S(mu) = sum_{n=0}^{N_t} sigma_n cos(mu t^n) (sigma_0 = sigma_{N_t}
// = dt/2, else dt) in closed form: with theta = mu dt the cosine sum is the
// Dirichlet kernel, sum_{n=0}^{N} cos(n theta) = sin((N + 1/2) theta) / (2 sin(theta/2))
// + 1/2, so S = dt [sin((N + 1/2) theta) / (2 sin(theta/2)) - cos(N theta) / 2]
// (S(0) = T_f).  O(1) per value instead of N_t + 1 terms.
static double trapezoid_cos_sum(double mu, double dt, int64_t N) {
    const double th = mu * dt, sh = sin(0.5 * th);
    if (fabs(sh) < 1e-300) return dt * (double)N;
    return dt * (sin(((double)N + 0.5) * th) / (2.0 * sh) - 0.5 * cos((double)N * th));
}

// beta_d of the discrete filter at a spatial eigenvalue lambda: eq. betad with
// the time-corrected frequency of eq. discreteExplicitLambdaTilde (explicit)
// or eq. discreteCorr (implicit).  Modes beyond the leapfrog limit get -1.
// With c_n = (2/T_f) sigma_n (cos(omega t^n) - alpha_d/2) (eq. filterQuadrature),
// sum_n c_n cos(lambda~ t^n) = [S(omega - lambda~) + S(omega + lambda~) - alpha_d S(lambda~)] / T_f.
double filter_beta(const FilterPlan& plan, ew_scheme scheme, double lam) {
    const double dt = plan.dt;
    double x;
    if (scheme == EW_EXPLICIT) {
        x = 0.5 * lam * dt;
    } else {
        x = 0.5 * lam * dt / sqrt(1.0 + 0.5 * (lam * dt) * (lam * dt));
    }
    if (x >= 1.0) return -1.0;
    const double lt = 2.0 / dt * asin(x);
    const int64_t N = plan.Nt;
    return (trapezoid_cos_sum(plan.omega - lt, dt, N) + trapezoid_cos_sum(plan.omega + lt, dt, N) -
            plan.alpha_d * trapezoid_cos_sum(lt, dt, N)) /
           plan.Tf;
}

// Mixed-precision iterative refinement of the invariant subspace found by the
// FP32 stage.  Each outer step applies the FP64 filter once to the nw current
// vectors X, which gives the exact (FP64) block relation
//     S X = X Theta + E,   E orthogonal to X,
// and then extends span[X, E] by p block expansions with FP32 wave-solves.
// Their relative error (~1e-5) only touches the small correction directions,
// so the Rayleigh-Ritz step with S (where the wanted eigenvalues are the
// extreme ones) improves X by several digits per outer step.  A last
// Rayleigh-Ritz with L_h inside span[X] separates near-degenerate pairs.
// kr is an FP32 Krylov-Schur run with block nw and basis (1 + p) nw.
// Shape of the mixed-precision refinement for n_wanted nw: p FP32 block
// expansions per outer step and up to nw guard vectors, as many as fit the
// Rayleigh-Ritz rotation of the (p + 2)(nw + guard) basis columns in the
// update kernel (<= 128 columns); p drops from 6 to 3 for large nw.  False
// if not even two guards fit.
static bool refine_shape(int nw, int* p, int* guard) {
    for (int pe = 6; pe >= 3; --pe) {
        int gd = std::min(nw, 128 / (pe + 2) - nw);
        if (gd >= 2) {
            *p = pe;
            *guard = gd;
            return true;
        }
    }
    return false;
}

// gimg: the grid whose filter applications give the images S X (g64, or its
// double-FP32 twin); the images fall back to g64 once an outer step with gimg
// cuts the worst eig-res by less than 10x (its accuracy floor reached)
static ew_status refine_ir(KSRun& ks, KSRun& kr, ew_grid* g64, ew_grid* gimg, int p, int max_outer,
                           double res_tol, std::vector<double>& lam_out, std::vector<double>& beta_out,
                           std::vector<double>& res_out, int* ws64, int* outer_done) {
    const int64_t N = ks.N;
    const int nw = kr.nw;      // wanted + guard vectors refined together
    const int nwant = ks.nw;
    EW_CUDA_TRY(cudaMemcpyAsync(kr.V, ks.V, sizeof(double) * (size_t)N * nw, cudaMemcpyDeviceToDevice, kr.st));
    double* W64 = nullptr;
    EW_TRY(kr.alloc((void**)&W64, sizeof(double) * (size_t)N * nw));
    std::vector<double> sc(nw), lam(nw);
    // Rayleigh-Ritz with L_h inside span[X] (separates pairs that S cannot),
    // rank by beta_d(lambda) of the filter, then eig-res of the wanted pairs:
    // all FP64 and no wave-solve, so it doubles as the stopping test
    const bool sym = weighted_sums(g64->geom);  // the vectors are W^{1/2} phi (see KSRun::apply_S)
    double* Qfree = kr.V + (size_t)nw * N;  // columns nw .. 2 nw - 1, free outside an outer step's expansion
    auto lrr_check = [&](double* worst) -> ew_status {
        if (sym) {  // W^{1/2} L_h W^{-1/2} X
            EW_TRY(launch_wsqrt<double>(g64->geom, kr.V, Qfree, nw, -1, kr.st));
            EW_TRY(launch_apply_L<double>(g64->geom, Qfree, W64, nw, 1.0, kr.st));
            EW_TRY(launch_wsqrt<double>(g64->geom, W64, W64, nw, 1, kr.st));
        } else {
            EW_TRY(launch_apply_L<double>(g64->geom, kr.V, W64, nw, 1.0, kr.st));
        }
        std::vector<double> G, Z, w;
        EW_TRY(kr.gram_host(kr.V, nw, W64, nw, G));
        for (int i = 0; i < nw; ++i)
            for (int j = 0; j < i; ++j) {
                double a = 0.5 * (G[(size_t)i * nw + j] + G[(size_t)j * nw + i]);
                G[(size_t)i * nw + j] = G[(size_t)j * nw + i] = a;
            }
        jacobi_eig(nw, G, Z, w);
        std::vector<double> l(nw), scr(nw);
        for (int i = 0; i < nw; ++i) {
            l[i] = sqrt(std::max(-w[i], 0.0));
            scr[i] = filter_beta(ks.plan, ks.p->scheme, l[i]);
        }
        std::vector<int> ord(nw);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int a, int c) { return scr[a] > scr[c]; });
        std::vector<double> Zo((size_t)nw * nw);
        for (int rr = 0; rr < nw; ++rr)
            for (int c = 0; c < nw; ++c) Zo[(size_t)rr * nw + c] = Z[(size_t)rr * nw + ord[c]];
        // X <- X Z (through W64, then back)
        EW_TRY(kr.update_host(kr.V, nw, nullptr, nw, Zo, 1.0, 0.0, W64));
        EW_CUDA_TRY(cudaMemcpyAsync(kr.V, W64, sizeof(double) * (size_t)N * nw, cudaMemcpyDeviceToDevice, kr.st));
        for (int c = 0; c < nw; ++c) sc[c] = scr[ord[c]];
        lam_out.resize(nwant);
        res_out.resize(nwant);
        if (sym) {  // eig-res of phi = W^{-1/2} x in the grid variables
            EW_TRY(launch_wsqrt<double>(g64->geom, kr.V, W64, nwant, -1, kr.st));
            EW_TRY(rayleigh_any(g64, W64, nwant, lam_out.data(), res_out.data(), kr.st));
        } else {
            EW_TRY(rayleigh_any(g64, kr.V, nwant, lam_out.data(), res_out.data(), kr.st));
        }
        *worst = *std::max_element(res_out.begin(), res_out.end());
        if (getenv("EW_KS_LOG")) fprintf(stderr, "[ew refine] eig-res of the wanted pairs %.3e\n", *worst);
        return EW_OK;
    };
    std::vector<double> theta, Y, resid;
    *outer_done = 0;
    if (!gimg) gimg = g64;
    double prev_worst = INFINITY;
    int p_step = p;  // FP32 block expansions of the current outer step
    for (int outer = 0; outer < max_outer; ++outer) {
        double worst = 0.0;
        EW_TRY(lrr_check(&worst));
        if (worst <= res_tol) break;
        if (gimg != g64 && worst > 0.1 * prev_worst) {
            gimg = g64;
            if (getenv("EW_KS_LOG")) fprintf(stderr, "[ew refine] images in FP64 from here on\n");
        }
        // size the expansions by the contraction the last step achieved with p_step of
        // them, taken as geometric in their number, for 10x below the target
        if (prev_worst < INFINITY && worst < prev_worst) {
            const double got = log(prev_worst / worst), need = log(10.0 * worst / res_tol);
            if (need < got) p_step = std::max(2, std::min(p, (int)ceil(p_step * need / got)));
        }
        prev_worst = worst;
        // image of X at FP64 accuracy: S X = X Theta + E
        for (int c0 = 0; c0 < nw; c0 += 16) {
            int nb = std::min(16, nw - c0);
            if (sym) {
                EW_TRY(launch_wsqrt<double>(g64->geom, kr.V + (size_t)c0 * N, Qfree, nb, -1, kr.st));
                EW_TRY(apply_filter(ks.hook, gimg, ks.p, ks.plan, Qfree, W64 + (size_t)c0 * N, nb, kr.st));
                EW_TRY(launch_wsqrt<double>(g64->geom, W64 + (size_t)c0 * N, W64 + (size_t)c0 * N, nb, 1, kr.st));
            } else {
                EW_TRY(apply_filter(ks.hook, gimg, ks.p, ks.plan, kr.V + (size_t)c0 * N, W64 + (size_t)c0 * N, nb,
                                    kr.st));
            }
        }
        *ws64 += nw;
        std::vector<double> T1, T2;
        EW_TRY(kr.gram_host(kr.V, nw, W64, nw, T1));
        EW_TRY(kr.update_host(kr.V, nw, W64, nw, T1, -1.0, 1.0, W64));
        EW_TRY(kr.gram_host(kr.V, nw, W64, nw, T2));
        EW_TRY(kr.update_host(kr.V, nw, W64, nw, T2, -1.0, 1.0, W64));
        // E = Q R with Q in V[:, nw : 2 nw]
        double* Q = kr.V + (size_t)nw * N;
        EW_CUDA_TRY(cudaMemcpyAsync(Q, W64, sizeof(double) * (size_t)N * nw, cudaMemcpyDeviceToDevice, kr.st));
        int r = 0;
        EW_TRY(kr.svqb(Q, nw, &r));
        if (r == 0) break;
        std::vector<double> R;
        EW_TRY(kr.gram_host(Q, r, W64, nw, R));  // r x nw
        if (r < nw) {  // fill the block with random directions orthogonal to the basis
            EW_TRY(splitmix_uniform(N * (int64_t)(nw - r), 0x5EED0000ull + outer, Q + (size_t)r * N, kr.st));
            double* F = Q + (size_t)r * N;
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<double> C;
                EW_TRY(kr.gram_host(kr.V, nw + r, F, nw - r, C));
                EW_TRY(kr.update_host(kr.V, nw + r, F, nw - r, C, -1.0, 1.0, F));
            }
            int r2 = 0;
            EW_TRY(kr.svqb(F, nw - r, &r2));
            if (r2 < nw - r) return set_error(EW_EBREAKDOWN, "refinement could not complete its block");
        }
        std::fill(kr.H.begin(), kr.H.end(), 0.0);
        for (int i = 0; i < nw; ++i)
            for (int j = 0; j < nw; ++j)
                kr.h(i, j) = 0.5 * (T1[(size_t)i * nw + j] + T2[(size_t)i * nw + j] + T1[(size_t)j * nw + i] +
                                    T2[(size_t)j * nw + i]);
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < nw; ++j) kr.h(nw + i, j) = R[(size_t)i * nw + j];
        kr.mcur = nw;
        for (int e = 0; e < p_step; ++e) {
            const int col0 = kr.mcur;  // S is applied to V[:, col0 : col0 + nw] in this expansion
            EW_TRY(kr.expand());
            // S is symmetric, so X^T S Q_e = (S X)^T Q_e = (X Theta + Q_1 R)^T Q_e, known
            // exactly in FP64: R^T for the first block, 0 beyond; the FP32 images
            // would carry their rounding noise into these entries
            for (int i = 0; i < nw; ++i)
                for (int j = 0; j < nw; ++j) kr.h(i, col0 + j) = (e == 0 && j < r) ? R[(size_t)j * nw + i] : 0.0;
        }
        kr.ritz(theta, Y, resid);
        if (getenv("EW_KS_LOG")) {
            fprintf(stderr, "[ew refine] outer %d rank %d |E_j|:", outer, r);
            for (int j = 0; j < nw; ++j) {
                double s = 0.0;
                for (int i = 0; i < r; ++i) s += R[(size_t)i * nw + j] * R[(size_t)i * nw + j];
                fprintf(stderr, " %.2e", sqrt(s));
            }
            fprintf(stderr, "\n[ew refine]   theta/resid:");
            for (int j = 0; j < nw + 2 && j < kr.mcur; ++j) fprintf(stderr, " %.9f/%.1e", theta[j], resid[j]);
            fprintf(stderr, "\n");
        }
        EW_TRY(kr.update_host(kr.V, kr.mcur, nullptr, kr.mcur, Y, 1.0, 0.0, kr.V));
        *outer_done = outer + 1;
        if (outer + 1 == max_outer) {
            double w2 = 0.0;
            EW_TRY(lrr_check(&w2));
        }
    }
    EW_CUDA_TRY(cudaMemcpyAsync(ks.V, kr.V, sizeof(double) * (size_t)N * nwant, cudaMemcpyDeviceToDevice, kr.st));
    beta_out.assign(sc.begin(), sc.begin() + nwant);
    (void)lam;
    return EW_OK;
}

struct GridDeleter {
    void operator()(ew_grid* g) const { ew_grid_destroy(g); }
};
using GridHandle = std::unique_ptr<ew_grid, GridDeleter>;

static ew_status make_twin_fp64(const ew_grid* g, ew_grid** out) {
    if (g->geom.map) {
        const int64_t n[2] = {g->geom.map->n1, g->geom.map->n2};
        return ew_grid_create_mapped(n, g->geom.map->xy.data(), EW_FP64, out);
    }
    ew_bc bc[6];
    int64_t n[3];
    for (int a = 0; a < 3; ++a) {
        const int lo = (g->geom.bc >> (2 * a)) & 1, hi = (g->geom.bc >> (2 * a + 1)) & 1;
        bc[2 * a] = lo ? EW_BC_NEUMANN : EW_BC_DIRICHLET;
        bc[2 * a + 1] = hi ? EW_BC_NEUMANN : EW_BC_DIRICHLET;
        n[a] = g->geom.n[a] - (a < g->geom.dim ? lo + hi : 0);  // back to interior points
    }
    return ew_grid_create(g->geom.dim, n, g->length, g->geom.order, bc, EW_FP64, out);
}

}  // namespace ew

using namespace ew;

namespace ew {

ew_status arnoldi_eigs_impl(const ew_grid* grid, const ew_filter_params* params, const ew_eigs_params* ep,
                            const double* start_dev, double* lambda_host, double* vecs_dev, ew_eigs_report* rep,
                            cudaStream_t st, FilterHook* hook) {
    auto t0 = std::chrono::steady_clock::now();
    if (!grid || !params || !ep || !lambda_host) return set_error(EW_EINVAL, "null argument");
    int dev = -1;
    EW_CUDA_TRY(cudaGetDevice(&dev));
    if (grid->device >= 0 && grid->device != dev) return set_error(EW_EINVAL, "grid was created on another device");
    const int nw = ep->n_wanted;
    if (nw < 1 || nw > EW_MAX_EIGS) return set_error(EW_EINVAL, "n_wanted must be in [1, EW_MAX_EIGS]");
    int b = ep->block > 0 ? ep->block : 1;
    if (b > 16) return set_error(EW_EINVAL, "block must be <= 16");
    int m = ep->krylov_dim > 0 ? ep->krylov_dim : 2 * nw + b;
    m = ((m + b - 1) / b) * b;
    if (m < nw + b) return set_error(EW_EINVAL, "krylov_dim must be >= n_wanted + block");
    if (m + 2 * b > 160) return set_error(EW_EINVAL, "krylov_dim too large (krylov_dim + 2 block <= 160)");
    int ref_p = 0, ref_guard = 0;
    if (grid->prec == EW_FP32X2) return set_error(EW_EUNSUPPORTED, "double-FP32 grids: ew_filter_apply only");
    if (ep->refine_fp64 < 0 || ep->refine_fp64 > 3) return set_error(EW_EINVAL, "refine_fp64 must be 0..3");
    if ((ep->refine_fp64 == 1 || ep->refine_fp64 == 3) && grid->prec == EW_FP32 && !refine_shape(nw, &ref_p, &ref_guard))
        return set_error(EW_EINVAL, "n_wanted too large for the FP64 refinement (n_wanted <= 23)");
    if ((int64_t)m > grid->geom.N) return set_error(EW_EINVAL, "krylov_dim exceeds the number of active points");
    ew_grid* g = const_cast<ew_grid*>(grid);

    KSRun ks;
    ks.g = g;
    ks.p = params;
    ks.hook = hook;
    EW_TRY(plan_filter(g->geom, params, &ks.plan));
    ks.N = g->geom.N;
    ks.b = b;
    ks.m = m;
    ks.nw = nw;
    ks.tol = ep->tol > 0 ? ep->tol : (g->prec == EW_FP32 ? 1e-4 : 1e-10);
    ks.lock = ep->lock != 0;
    ks.max_ws = ep->max_wave_solves > 0 ? ep->max_wave_solves : 2000;
    ks.st = st;
    EW_TRY(ks.setup());
    EW_TRY(ks.start(start_dev, ep->seed));
    std::vector<double> theta;
    int nconv = 0;
    EW_TRY(ks.run(theta, &nconv));

    ew_eigs_report r;
    std::memset(&r, 0, sizeof(r));
    r.wave_solves = ks.wave_solves;
    r.restarts = ks.restarts;
    // stage 2 on the grid-precision result
    // with Neumann faces the basis holds W^{1/2} phi (KSRun::apply_S): the
    // quotients and eig-res are taken of phi, in the grid variables
    const bool sym = weighted_sums(g->geom);
    double* phis = nullptr;
    if (sym) EW_TRY(ks.alloc((void**)&phis, sizeof(double) * (size_t)ks.N * nw));
    auto rq = [&](ew_grid* g64, const double* X, double* lam_h, double* res_h) -> ew_status {
        if (!sym) return rayleigh_any(g64, X, nw, lam_h, res_h, st);
        EW_TRY(launch_wsqrt<double>(g64->geom, X, phis, nw, -1, st));
        return rayleigh_any(g64, phis, nw, lam_h, res_h, st);
    };
    std::vector<double> lam1(nw), res1(nw);
    {
        ew_grid* raw = nullptr;
        EW_TRY(make_twin_fp64(g, &raw));
        GridHandle twin(raw);
        EW_TRY(rq(twin.get(), ks.V, lam1.data(), res1.data()));
    }
    const double* final_vecs = ks.V;
    std::vector<double> lam(lam1), res(res1), beta(theta.begin(), theta.begin() + nw);
    KSRun ks2;
    GridHandle g64;  // the FP64 twin of the refinement
    ew_status status = nconv >= nw ? EW_OK : EW_ENOCONV;
    if ((ep->refine_fp64 == 1 || ep->refine_fp64 == 3) && g->prec == EW_FP32) {
        ew_grid* raw = nullptr;
        EW_TRY(make_twin_fp64(g, &raw));
        g64.reset(raw);
        GridHandle gdd;  // refine_fp64 3: the images in double-FP32 pairs
        if (ep->refine_fp64 == 3 && g->geom.dim == 2 && !g->geom.map) {
            raw = nullptr;
            EW_TRY(make_twin_fp64(g, &raw));
            gdd.reset(raw);
            gdd->prec = EW_FP32X2;
        }
        // guard vectors: a pair just outside the wanted set can share beta with
        // one inside (lambda on the other side of the peak); refining both and
        // ranking by beta_d(lambda) after the L_h projection keeps the right one.
        // On dense spectra the guards also widen the gap between the refined
        // block and the rest, which sets the contraction of each outer step.
        const int guard = ref_guard, pexp = ref_p;
        const int nr = std::min(nw + guard, (int)theta.size());
        KSRun kr;
        kr.g = g;
        kr.p = params;
        kr.hook = hook;
        kr.plan = ks.plan;
        kr.N = ks.N;
        kr.b = nr;
        kr.nw = nr;
        kr.m = (pexp + 1) * nr;
        kr.tol = 0.0;
        kr.max_ws = 0;
        kr.st = st;
        int ws64 = 0, outer = 0;
        double res_tol = ep->refine_tol > 0 ? ep->refine_tol : 5e-9;
        EW_TRY(kr.setup());
        EW_TRY(refine_ir(ks, kr, g64.get(), gdd.get(), pexp, 6, res_tol, lam, beta, res, &ws64, &outer));
        r.wave_solves += kr.wave_solves;
        r.wave_solves_fp64 = ws64;
        r.restarts += outer;
    } else if (ep->refine_fp64 == 2 && g->prec == EW_FP32) {
        ew_grid* raw = nullptr;
        EW_TRY(make_twin_fp64(g, &raw));
        g64.reset(raw);
        ks2.g = g64.get();
        ks2.p = params;
        ks2.hook = hook;
        ks2.plan = ks.plan;
        ks2.N = ks.N;
        ks2.b = nw;
        ks2.m = 3 * nw;
        ks2.nw = nw;
        ks2.tol = ep->refine_tol > 0 ? ep->refine_tol : 1e-10;
        ks2.max_ws = std::max(ks.max_ws / 2, 8 * nw);
        ks2.st = st;
        EW_TRY(ks2.setup());
        EW_TRY(ks2.start(ks.V, 0, true));
        int nconv2 = 0;
        std::vector<double> theta2;
        EW_TRY(ks2.run(theta2, &nconv2));
        EW_TRY(rq(g64.get(), ks2.V, lam.data(), res.data()));
        final_vecs = ks2.V;
        beta.assign(theta2.begin(), theta2.begin() + nw);
        r.wave_solves_fp64 = ks2.wave_solves;
        r.restarts += ks2.restarts;
        status = nconv2 >= nw ? EW_OK : EW_ENOCONV;
        if (status != EW_OK) set_error(EW_ENOCONV, "FP64 refinement did not reach refine_tol within the budget");
    } else if (status != EW_OK) {
        set_error(EW_ENOCONV, "not every wanted pair converged within max_wave_solves");
    }
    for (int j = 0; j < nw; ++j) {
        lambda_host[j] = lam[j];
        r.beta[j] = beta[j];
        r.eig_res[j] = res[j];
        r.lambda_stage1[j] = lam1[j];
        r.eig_res_stage1[j] = res1[j];
        // the refined pair nearest in lambda to each first-stage pair
        double best = INFINITY;
        for (int i = 0; i < nw; ++i) best = std::min(best, fabs(lam[j] - lam1[i]));
        r.lambda_rel_change[j] = lam[j] > 0 ? best / lam[j] : 0.0;
    }
    r.n_converged = nconv;
    if (vecs_dev && sym) EW_TRY(launch_wsqrt<double>(g->geom, final_vecs, vecs_dev, nw, -1, st));
    if (vecs_dev && !sym)
        EW_CUDA_TRY(cudaMemcpyAsync(vecs_dev, final_vecs, sizeof(double) * (size_t)ks.N * nw,
                                    cudaMemcpyDeviceToDevice, st));
    EW_CUDA_TRY(cudaStreamSynchronize(st));
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    return status;
}

}  // namespace ew

extern "C" ew_status ew_arnoldi_eigs(const ew_grid* grid, const ew_filter_params* params,
                                     const ew_eigs_params* ep, const double* start_dev, double* lambda_host,
                                     double* vecs_dev, ew_eigs_report* rep, cudaStream_t st) try {
    clear_error();
    return arnoldi_eigs_impl(grid, params, ep, start_dev, lambda_host, vecs_dev, rep, st, nullptr);
} catch (...) {
    return abi_exception();
}
