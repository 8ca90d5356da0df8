// ew_periods.cu -- choice of the number of filter periods N_p for an
// eigen-solve (Section "Estimating the EigenWave convergence rate based on
// simultaneous iteration", eq. subSpaceIterationCR; Section "Changing the
// number of filter periods N_p as a function of the number of computed
// eigenpairs").  Host code only.
//
// With the filter values beta_j = beta_d(lambda_j) of the grid's discrete
// eigenvalues sorted in decreasing order (with multiplicity), simultaneous
// iteration on an N_a-dimensional subspace converges to the N_r wanted pairs
// at the rate CR = beta_{N_a+1} / beta_{N_r}.  A longer filter (larger N_p)
// narrows the peak, so fewer eigenvalues share the top of it and CR drops, but
// each wave-solve costs N_p times more.  For N_p = 1, 2, 4, ... the cost of a
// solve is taken as N_p / (-ln CR) (wave-solve length times the iterations per
// factor e of residual reduction), and the cheapest N_p is returned.
//
// On the boxes of this library the discrete spectrum is known exactly: the
// eigenvectors are tensor sine / cosine modes with lambda^2 = sum_a mu_a(k_a),
// mu_a the 1D symbol of the stencil, (4/h^2) s (order 2) or
// (4/h^2)(s + s^2/3) (order 4), s = sin^2(theta / 2), theta set per axis by
// its faces (axis_symbol).  The
// eigenvalues near omega are enumerated from these (per row of modes a binary
// search of the monotone last-axis symbol), so no GPU is needed.
#include <math.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "ew_internal.h"

namespace ew {

double filter_beta(const FilterPlan& plan, ew_scheme scheme, double lam);

// 1D symbol of axis a over its modes, increasing.  With M = (interior points
// + 1) the modes are sin(theta j) / cos(theta j) of the vertex index j, at
//   theta = k pi / M, k = 1 .. M-1      (two Dirichlet faces: sine modes)
//   theta = k pi / M, k = 0 .. M        (two Neumann faces: cosine modes)
//   theta = (k - 1/2) pi / M, k = 1 .. M  (one of each)
// and mu = (4/h^2) s (order 2) or (4/h^2)(s + s^2/3) (order 4), s = sin^2(theta/2).
static std::vector<double> axis_symbol(const GridGeom& g, int a) {
    const int code = (g.bc >> (2 * a)) & 3;
    const int nn = (code & 1) + ((code >> 1) & 1);
    const int64_t M = g.n[a] - nn + 1;
    const double h = g.h[a];
    std::vector<double> mu;
    mu.reserve((size_t)g.n[a]);
    for (int64_t k = 0; k <= M; ++k) {
        double th;
        if (nn == 0) {
            if (k < 1 || k > M - 1) continue;
            th = k * M_PI / M;
        } else if (nn == 2) {
            th = k * M_PI / M;
        } else {
            if (k < 1) continue;
            th = (k - 0.5) * M_PI / M;
        }
        const double sn = sin(0.5 * th);
        const double s2 = sn * sn;
        mu.push_back(4.0 / (h * h) * (g.order == 4 ? s2 + s2 * s2 / 3.0 : s2));
    }
    return mu;
}

// the discrete eigenvalues lambda with lo^2 <= lambda^2 <= hi^2 (with
// multiplicity), at most cap of them (returns false when there are more)
static bool eigenvalues_in(const GridGeom& g, const std::vector<std::vector<double>>& mu, double lo, double hi,
                           size_t cap, std::vector<double>& out) {
    out.clear();
    const double lo2 = lo * lo, hi2 = hi * hi;
    const std::vector<double>& last = mu[(size_t)g.dim - 1];
    auto scan_last = [&](double base) -> bool {  // last-axis modes with base + mu in [lo2, hi2]
        auto b = std::lower_bound(last.begin(), last.end(), lo2 - base);
        auto e = std::upper_bound(last.begin(), last.end(), hi2 - base);
        for (auto it = b; it < e; ++it) {
            if (out.size() >= cap) return false;
            out.push_back(sqrt(base + *it));
        }
        return true;
    };
    for (double mx : mu[0]) {
        if (mx > hi2) break;
        if (g.dim == 2) {
            if (!scan_last(mx)) return false;
        } else {
            for (double my : mu[1]) {
                if (mx + my > hi2) break;
                if (!scan_last(mx + my)) return false;
            }
        }
    }
    return true;
}

}  // namespace ew

using namespace ew;

extern "C" {

ew_status ew_choose_num_periods(const ew_grid* grid, const ew_filter_params* params, int n_wanted, int krylov_dim,
                                int max_periods, int* num_periods, double* cr_host) try {
    clear_error();
    if (!grid || !params || !num_periods) return set_error(EW_EINVAL, "null argument");
    if (n_wanted < 1 || krylov_dim <= n_wanted) return set_error(EW_EINVAL, "need 1 <= n_wanted < krylov_dim");
    if (max_periods < 1 || max_periods > (1 << 20)) return set_error(EW_EINVAL, "max_periods out of range");
    const GridGeom& g = grid->geom;
    if (g.map) return set_error(EW_EUNSUPPORTED, "the spectrum of a mapped grid has no closed form");
    if ((int64_t)krylov_dim + 1 > g.N) return set_error(EW_EINVAL, "krylov_dim + 1 exceeds the number of points");
    std::vector<std::vector<double>> mu;
    for (int a = 0; a < g.dim; ++a) mu.push_back(axis_symbol(g, a));
    const double lam_max = sqrt(mu[0].back() + mu[1].back() + (g.dim == 3 ? mu[2].back() : 0.0));
    const size_t want = (size_t)krylov_dim + 1;
    double best_cost = INFINITY;
    int best = 1, idx = 0;
    for (int np = 1; np <= max_periods; np *= 2, ++idx) {
        ew_filter_params p = *params;
        p.num_periods = np;
        FilterPlan plan;
        // A candidate past the longest wave-solve is not evaluated (CR = 1), nor
        // are the longer ones.  (beta_d costs O(1) per eigenvalue: filter_beta
        // sums the trapezoid rule in closed form.)
        const ew_status ps = plan_filter(g, &p, &plan, false);
        if (np > 1 && ps != EW_OK) {
            clear_error();
            if (cr_host)
                for (int k = np; k <= max_periods; k *= 2) cr_host[idx++] = 1.0;
            break;
        }
        EW_TRY(ps);
        // Widen a window [omega - w, omega + w] until the filter cannot put an
        // eigenvalue outside it among the top N_a + 1: beyond distance d of omega
        // (in time-corrected frequency) the filter's sum of cosines is bounded by
        // 2 [1 / (T d) + 1 / (T omega) + min(0.11, 1 / (2 T lambda~_1))] (Dirichlet-kernel
        // bound with a factor 2 of margin), compared with the window's beta_{N_a+1}.
        const double T = plan.Tf;
        const ew_scheme sch = (ew_scheme)params->scheme;
        auto lt = [&](double l) {  // time-corrected frequency (monotone in l)
            double x = 0.5 * l * plan.dt;
            if (sch != EW_EXPLICIT) x /= sqrt(1.0 + x * x);
            return x >= 1.0 ? M_PI / plan.dt : 2.0 / plan.dt * asin(x);
        };
        const double lt1 = lt(sqrt(mu[0][0] + mu[1][0] + (g.dim == 3 ? mu[2][0] : 0.0)));
        // the positive part of -sinc(x)/2 never exceeds 0.109 (sinc >= -0.2173),
        // which bounds the third term also when lambda_1 = 0 (all faces Neumann)
        const double t3 = lt1 > 0.0 ? std::min(0.11, 0.5 / (T * lt1)) : 0.11;
        std::vector<double> lam, beta;
        double w = 2.0 * plan.omega / np, cr = 1.0;
        for (;;) {
            const double lo = std::max(0.0, plan.omega - w), hi = plan.omega + w;
            const bool all = lo == 0.0 && hi >= lam_max;
            if (!eigenvalues_in(g, mu, lo, hi, (size_t)4000000, lam)) break;  // too many: keep the last estimate
            if (lam.size() < want && !all) {
                w *= 2.0;
                continue;
            }
            if (lam.size() < want) break;
            beta.resize(lam.size());
            for (size_t i = 0; i < lam.size(); ++i) beta[i] = filter_beta(plan, sch, lam[i]);
            std::sort(beta.begin(), beta.end(), std::greater<double>());
            const double bw = beta[(size_t)n_wanted - 1], bn = beta[(size_t)krylov_dim];
            cr = bw > 0.0 ? std::max(0.0, bn) / bw : 1.0;
            if (all) break;
            const double d = std::min(plan.omega - (lo > 0.0 ? lt(lo) : 0.0), lt(hi) - plan.omega);
            const double env =
                d > 0.0 ? 2.0 * (1.0 / (T * d) + 1.0 / (T * plan.omega) + t3) : INFINITY;
            if (env < bn) break;
            w *= 2.0;
        }
        if (cr_host) cr_host[idx] = cr;
        const double cost = cr < 1.0 ? np / std::max(-log(std::max(cr, 1e-300)), 1e-12) : INFINITY;
        if (cost < best_cost) {
            best_cost = cost;
            best = np;
        }
    }
    if (!(best_cost < INFINITY))
        return set_error(EW_EUNSUPPORTED, "no N_p up to max_periods separates the wanted pairs (CR = 1)");
    *num_periods = best;
    return EW_OK;
} catch (...) {
    return abi_exception();
}

}  // extern "C"
