/*
 * ew_oracle_mg.c -- plain FP64 geometric multigrid for the implicit time-step
 * system M x = b, M = I - a L_h, a = dt^2/2 (eq. impMatrix), and the learned
 * convolutional smoother (two 3x3x3 convolutions, 1 -> 8 -> 1 channels).
 *
 * TEST INFRASTRUCTURE ONLY (see ew_oracle.c).
 *
 * The paper solves the implicit systems with its multigrid solver (Section
 * 'An optimal O(N) eigenvalue solver'), naming red-black and line smoothers
 * but giving no cycle details.  This oracle fixes one plain V-cycle, which the
 * CUDA path must reproduce step for step:
 *   - levels: n_c = (n - 1) / 2 per axis (the coarse point I sits on fine
 *     point 2I+1), same box, so h_c = 2 h; stop when some axis has n < 5 or
 *     even n; the coarsest system is solved by CG to 1e-14;
 *   - smoother: damped Jacobi x += wJ (b - M x) / D with the constant interior
 *     diagonal D = 1 + a sum_i d0 / h_i^2, d0 = 2 (order 2) or 5/2 (order 4);
 *     or multi-colour Gauss-Seidel (red-black is one of the smoothers the
 *     paper names): each sweep updates the points colour by colour, each by
 *     x += (b - M x) / D with the current values; the colours are chosen so
 *     that no point's stencil reaches another point of its colour, so a
 *     colour's updates are independent: for the second-order stencil the
 *     parity of i + j + k (red-black), for the fourth-order one (offsets of
 *     1 and 2 along one axis) (i + j + k) mod 3, three colours; or, on the finest
 *     `nlev_learned` levels, the learned correction x += N(b - M x);
 *   - restriction: full weighting, the tensor product of (1/4, 1/2, 1/4);
 *   - prolongation: (multi)linear interpolation, zero on the boundary.
 *
 * The learned correction N (3D only):
 *   h_c(x) = sum_{o in {-1,0,1}^3} W1[c][o] r(x + o),  c = 0..7
 *   N(r)(x) = sum_c sum_o W2[c][o] h_c(x + o)
 * with zero values outside the active box (homogeneous Dirichlet), no bias
 * and no activation: the correction stays linear in r, so the multigrid
 * solve, and hence the filter operator, stays linear.  Tap order of W[c][o]:
 * o = (dz, dy, dx), dz slowest, each from -1 to 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

int og_apply_M(int dim, const long* n, const double* h, int order, double a, const double* x,
               double* y);
int og_cg_solve_M(int dim, const long* n, const double* h, int order, double a, const double* b,
                  double* x, double tol, int maxit);

#define OG_MAX_LEVELS 16
#define OG_NET_C 8
#define OG_NET_W (OG_NET_C * 27)

typedef struct {
    long n[3];
    double h[3];
    long size;
} og_level;

static long og_idx3(const long* n, long i, long j, long k) { return (k * n[1] + j) * n[0] + i; }

/* value of an active vector at (i,j,k), zero outside the active box */
static double og_get(const long* n, const double* v, long i, long j, long k) {
    if (i < 0 || j < 0 || k < 0 || i >= n[0] || j >= n[1] || k >= n[2]) return 0.0;
    return v[og_idx3(n, i, j, k)];
}

static int og_build_levels(int dim, const long* n, const double* h, og_level* lv) {
    int L = 0;
    for (int a = 0; a < 3; ++a) {
        lv[0].n[a] = a < dim ? n[a] : 1;
        lv[0].h[a] = a < dim ? h[a] : 1.0;
    }
    lv[0].size = lv[0].n[0] * lv[0].n[1] * lv[0].n[2];
    for (;;) {
        int ok = L + 1 < OG_MAX_LEVELS;
        for (int a = 0; a < dim; ++a)
            if (lv[L].n[a] < 5 || (lv[L].n[a] % 2) == 0) ok = 0;
        if (!ok) break;
        for (int a = 0; a < 3; ++a) {
            lv[L + 1].n[a] = a < dim ? (lv[L].n[a] - 1) / 2 : 1;
            lv[L + 1].h[a] = a < dim ? 2.0 * lv[L].h[a] : 1.0;
        }
        lv[L + 1].size = lv[L + 1].n[0] * lv[L + 1].n[1] * lv[L + 1].n[2];
        ++L;
    }
    return L + 1;
}

/* full weighting: rc(I) = sum_o w(o) r(2I+1+o), w = prod (1/4, 1/2, 1/4) */
static void og_restrict(int dim, const og_level* f, const og_level* c, const double* r, double* rc) {
    static const double w[3] = {0.25, 0.5, 0.25};
    int oz0 = dim == 3 ? -1 : 0, oz1 = dim == 3 ? 1 : 0;
    for (long K = 0; K < c->n[2]; ++K)
        for (long J = 0; J < c->n[1]; ++J)
            for (long I = 0; I < c->n[0]; ++I) {
                long fi = 2 * I + 1, fj = 2 * J + 1, fk = dim == 3 ? 2 * K + 1 : 0;
                double s = 0.0;
                for (int oz = oz0; oz <= oz1; ++oz)
                    for (int oy = -1; oy <= 1; ++oy)
                        for (int ox = -1; ox <= 1; ++ox) {
                            double wt = w[ox + 1] * w[oy + 1] * (dim == 3 ? w[oz + 1] : 1.0);
                            s += wt * og_get(f->n, r, fi + ox, fj + oy, fk + oz);
                        }
                rc[og_idx3(c->n, I, J, K)] = s;
            }
}

/* linear interpolation of a coarse correction, added to the fine vector:
 * along each axis a fine index i = 2I+1 takes coarse I, an even i = 2I takes
 * the mean of coarse I-1 and I (zero beyond the box). */
static void og_prolong_add(int dim, const og_level* f, const og_level* c, const double* ec,
                           double* x) {
    for (long k = 0; k < f->n[2]; ++k)
        for (long j = 0; j < f->n[1]; ++j)
            for (long i = 0; i < f->n[0]; ++i) {
                long ci[2], cj[2], ck[2];
                double wi[2], wj[2], wk[2];
                int ni, nj, nk;
                /* per-axis stencil */
                if (i % 2 == 1) { ci[0] = (i - 1) / 2; wi[0] = 1.0; ni = 1; }
                else { ci[0] = i / 2 - 1; ci[1] = i / 2; wi[0] = wi[1] = 0.5; ni = 2; }
                if (j % 2 == 1) { cj[0] = (j - 1) / 2; wj[0] = 1.0; nj = 1; }
                else { cj[0] = j / 2 - 1; cj[1] = j / 2; wj[0] = wj[1] = 0.5; nj = 2; }
                if (dim == 2) { ck[0] = 0; wk[0] = 1.0; nk = 1; }
                else if (k % 2 == 1) { ck[0] = (k - 1) / 2; wk[0] = 1.0; nk = 1; }
                else { ck[0] = k / 2 - 1; ck[1] = k / 2; wk[0] = wk[1] = 0.5; nk = 2; }
                double s = 0.0;
                for (int c3 = 0; c3 < nk; ++c3)
                    for (int c2 = 0; c2 < nj; ++c2)
                        for (int c1 = 0; c1 < ni; ++c1)
                            s += wi[c1] * wj[c2] * wk[c3] * og_get(c->n, ec, ci[c1], cj[c2], ck[c3]);
                x[og_idx3(f->n, i, j, k)] += s;
            }
}

/* first layer: hid[c] = conv(W1[c], r) */
static void og_conv1(const long* n, const double* W1, const double* r, double* hid) {
    long N = n[0] * n[1] * n[2];
    for (int c = 0; c < OG_NET_C; ++c)
        for (long k = 0; k < n[2]; ++k)
            for (long j = 0; j < n[1]; ++j)
                for (long i = 0; i < n[0]; ++i) {
                    double s = 0.0;
                    int t = 0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx, ++t)
                                s += W1[c * 27 + t] * og_get(n, r, i + dx, j + dy, k + dz);
                    hid[c * N + og_idx3(n, i, j, k)] = s;
                }
}

/* second layer: y = sum_c conv(W2[c], hid[c]) */
static void og_conv2(const long* n, const double* W2, const double* hid, double* y) {
    long N = n[0] * n[1] * n[2];
    for (long k = 0; k < n[2]; ++k)
        for (long j = 0; j < n[1]; ++j)
            for (long i = 0; i < n[0]; ++i) {
                double s = 0.0;
                for (int c = 0; c < OG_NET_C; ++c) {
                    int t = 0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx, ++t)
                                s += W2[c * 27 + t] * og_get(n, hid + c * N, i + dx, j + dy, k + dz);
                }
                y[og_idx3(n, i, j, k)] = s;
            }
}

/* forward pass: hid (8 x N, may be NULL) and y = N(r) (N).  w = [W1 | W2]. */
int og_conv_net_forward(const long* n, const double* w, const double* r, double* hid, double* y) {
    long N = n[0] * n[1] * n[2];
    double* tmp = hid ? hid : (double*)malloc(sizeof(double) * (size_t)(OG_NET_C * N));
    if (!tmp) return -2;
    og_conv1(n, w, r, tmp);
    og_conv2(n, w + OG_NET_W, tmp, y);
    if (!hid) free(tmp);
    return 0;
}

/* backward pass for a scalar loss with dLoss/dy = gy:
 *   dW2[c][o] = sum_x gy(x) hid_c(x + o)
 *   dhid_c(x) = sum_o W2[c][o] gy(x - o)
 *   dW1[c][o] = sum_x dhid_c(x) r(x + o)
 * `hid` is the forward activation (8 x N); gw receives [dW1 | dW2];
 * dr (may be NULL) receives dLoss/dr = sum_c sum_o W1[c][o] dhid_c(x - o). */
int og_conv_net_backward(const long* n, const double* w, const double* r, const double* hid,
                         const double* gy, double* gw, double* dr) {
    long N = n[0] * n[1] * n[2];
    const double* W1 = w;
    const double* W2 = w + OG_NET_W;
    double* dhid = (double*)malloc(sizeof(double) * (size_t)(OG_NET_C * N));
    if (!dhid) return -2;
    memset(gw, 0, sizeof(double) * 2 * OG_NET_W);
    for (int c = 0; c < OG_NET_C; ++c) {
        int t = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++t) {
                    double s = 0.0;
                    for (long k = 0; k < n[2]; ++k)
                        for (long j = 0; j < n[1]; ++j)
                            for (long i = 0; i < n[0]; ++i)
                                s += gy[og_idx3(n, i, j, k)] *
                                     og_get(n, hid + c * N, i + dx, j + dy, k + dz);
                    gw[OG_NET_W + c * 27 + t] = s;
                }
    }
    for (int c = 0; c < OG_NET_C; ++c)
        for (long k = 0; k < n[2]; ++k)
            for (long j = 0; j < n[1]; ++j)
                for (long i = 0; i < n[0]; ++i) {
                    double s = 0.0;
                    int t = 0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx, ++t)
                                s += W2[c * 27 + t] * og_get(n, gy, i - dx, j - dy, k - dz);
                    dhid[c * N + og_idx3(n, i, j, k)] = s;
                }
    for (int c = 0; c < OG_NET_C; ++c) {
        int t = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++t) {
                    double s = 0.0;
                    for (long k = 0; k < n[2]; ++k)
                        for (long j = 0; j < n[1]; ++j)
                            for (long i = 0; i < n[0]; ++i)
                                s += dhid[c * N + og_idx3(n, i, j, k)] *
                                     og_get(n, r, i + dx, j + dy, k + dz);
                    gw[c * 27 + t] = s;
                }
    }
    if (dr) {
        for (long k = 0; k < n[2]; ++k)
            for (long j = 0; j < n[1]; ++j)
                for (long i = 0; i < n[0]; ++i) {
                    double s = 0.0;
                    for (int c = 0; c < OG_NET_C; ++c) {
                        int t = 0;
                        for (int dz = -1; dz <= 1; ++dz)
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx, ++t)
                                    s += W1[c * 27 + t] *
                                         og_get(n, dhid + c * N, i - dx, j - dy, k - dz);
                    }
                    dr[og_idx3(n, i, j, k)] = s;
                }
    }
    free(dhid);
    return 0;
}

typedef struct {
    int dim, order, nlev, nu1, nu2, nlearn, red_black;
    double a, wJ;
    og_level lv[OG_MAX_LEVELS];
    const double* net; /* nlearn x (2 * OG_NET_W) */
} og_mg;

static double og_jacobi_diag(const og_mg* m, const og_level* l) {
    double d0 = m->order == 2 ? 2.0 : 2.5, s = 0.0;
    for (int a = 0; a < m->dim; ++a) s += d0 / (l->h[a] * l->h[a]);
    return 1.0 + m->a * s;
}

/* (M x)_q = x_q - a sum_i (x(q - e_i) - 2 x_q + x(q + e_i)) / h_i^2 at point
 * (i, j, k) of the second-order system, zero beyond the box */
static double og_Mx_point2(const og_mg* m, const og_level* l, const double* x, long i, long j, long k) {
    const long* n = l->n;
    double xc = og_get(n, x, i, j, k), s = 0.0;
    s += (og_get(n, x, i - 1, j, k) - 2.0 * xc + og_get(n, x, i + 1, j, k)) / (l->h[0] * l->h[0]);
    s += (og_get(n, x, i, j - 1, k) - 2.0 * xc + og_get(n, x, i, j + 1, k)) / (l->h[1] * l->h[1]);
    if (m->dim == 3) s += (og_get(n, x, i, j, k - 1) - 2.0 * xc + og_get(n, x, i, j, k + 1)) / (l->h[2] * l->h[2]);
    return xc - m->a * s;
}

/* value at index p of an axis of length n under the odd (Dirichlet) closure:
 * the wall points -1 and n are 0, beyond them the mirror with a minus sign */
static double og_axis_ext(const double* x, long base, long stride, long p, long n) {
    if (p >= 0 && p < n) return x[base + p * stride];
    if (p == -1 || p == n) return 0.0;
    if (p < -1) return -x[base + (-2 - p) * stride];
    return -x[base + (2 * n - p) * stride];
}

/* (M x)_q at point (i, j, k) of the fourth-order system with the odd-reflection
 * closure: x_q - a sum_i (-x(-2) + 16 x(-1) - 30 x_q + 16 x(+1) - x(+2)) / (12 h_i^2) */
static double og_Mx_point4(const og_mg* m, const og_level* l, const double* x, long i, long j, long k) {
    const long* n = l->n;
    const long q = og_idx3(n, i, j, k);
    const long pos[3] = {i, j, k}, stride[3] = {1, n[0], n[0] * n[1]};
    double s = 0.0;
    for (int a = 0; a < m->dim; ++a) {
        const long base = q - pos[a] * stride[a];
        const double xm2 = og_axis_ext(x, base, stride[a], pos[a] - 2, n[a]);
        const double xm1 = og_axis_ext(x, base, stride[a], pos[a] - 1, n[a]);
        const double xp1 = og_axis_ext(x, base, stride[a], pos[a] + 1, n[a]);
        const double xp2 = og_axis_ext(x, base, stride[a], pos[a] + 2, n[a]);
        s += (-xm2 + 16.0 * xm1 - 30.0 * x[q] + 16.0 * xp1 - xp2) / (12.0 * l->h[a] * l->h[a]);
    }
    return x[q] - m->a * s;
}

static int og_colour(int order, long i, long j, long k) {
    return order == 2 ? (int)((i + j + k) & 1) : (int)((i + j + k) % 3);
}

static void og_smooth(const og_mg* m, int L, const double* b, double* x, double* r, int nu) {
    const og_level* l = &m->lv[L];
    double D = og_jacobi_diag(m, l);
    if (m->red_black && L >= m->nlearn) {
        const long* n = l->n;
        const int ncol = m->order == 2 ? 2 : 3;
        for (int s = 0; s < nu; ++s)
            for (int colour = 0; colour < ncol; ++colour)
                for (long k = 0; k < n[2]; ++k)
                    for (long j = 0; j < n[1]; ++j)
                        for (long i = 0; i < n[0]; ++i) {
                            if (og_colour(m->order, i, j, k) != colour) continue;
                            long q = og_idx3(n, i, j, k);
                            double mx = m->order == 2 ? og_Mx_point2(m, l, x, i, j, k) : og_Mx_point4(m, l, x, i, j, k);
                            x[q] += (b[q] - mx) / D;
                        }
        return;
    }
    double* corr = NULL;
    if (L < m->nlearn) corr = (double*)malloc(sizeof(double) * (size_t)l->size);
    for (int s = 0; s < nu; ++s) {
        og_apply_M(m->dim, l->n, l->h, m->order, m->a, x, r);
        for (long q = 0; q < l->size; ++q) r[q] = b[q] - r[q];
        if (L < m->nlearn) {
            og_conv_net_forward(l->n, m->net + (size_t)L * 2 * OG_NET_W, r, NULL, corr);
            for (long q = 0; q < l->size; ++q) x[q] += corr[q];
        } else {
            for (long q = 0; q < l->size; ++q) x[q] += m->wJ * r[q] / D;
        }
    }
    free(corr);
}

static void og_vcycle(const og_mg* m, int L, const double* b, double* x) {
    const og_level* l = &m->lv[L];
    if (L == m->nlev - 1) {
        og_cg_solve_M(m->dim, l->n, l->h, m->order, m->a, b, x, 1e-14, 100000);
        return;
    }
    const og_level* c = &m->lv[L + 1];
    double* r = (double*)malloc(sizeof(double) * (size_t)l->size);
    double* rc = (double*)malloc(sizeof(double) * (size_t)c->size);
    double* ec = (double*)calloc((size_t)c->size, sizeof(double));
    og_smooth(m, L, b, x, r, m->nu1);
    og_apply_M(m->dim, l->n, l->h, m->order, m->a, x, r);
    for (long q = 0; q < l->size; ++q) r[q] = b[q] - r[q];
    og_restrict(m->dim, l, c, r, rc);
    og_vcycle(m, L + 1, rc, ec);
    og_prolong_add(m->dim, l, c, ec, x);
    og_smooth(m, L, b, x, r, m->nu2);
    free(r);
    free(rc);
    free(ec);
}

static double og_norm2(long N, const double* v) {
    double s = 0.0;
    for (long q = 0; q < N; ++q) s += v[q] * v[q];
    return sqrt(s);
}

/* `ncycles` V(nu1, nu2) cycles on M x = b starting from the x passed in
 * (red_black: the multi-colour Gauss-Seidel smoother instead of damped Jacobi).
 * res_hist (ncycles + 1 entries, may be NULL) receives ||b - M x||_2 before
 * the first and after every cycle.  Returns the number of levels, < 0 on bad
 * arguments. */
int og_mg_solve(int dim, const long* n, const double* h, int order, double a, const double* b,
                double* x, int nu1, int nu2, double wJ, int ncycles, const double* net_w,
                int nlev_learned, double* res_hist, int red_black) {
    og_mg m;
    if ((dim != 2 && dim != 3) || (order != 2 && order != 4) || ncycles < 0) return -1;
    m.red_black = red_black;
    if (net_w && nlev_learned > 0 && dim != 3) return -1;
    m.dim = dim;
    m.order = order;
    m.a = a;
    m.wJ = wJ;
    m.nu1 = nu1;
    m.nu2 = nu2;
    m.nlev = og_build_levels(dim, n, h, m.lv);
    m.nlearn = net_w ? nlev_learned : 0;
    if (m.nlearn > m.nlev - 1) m.nlearn = m.nlev - 1;
    m.net = net_w;
    long N = m.lv[0].size;
    double* r = (double*)malloc(sizeof(double) * (size_t)N);
    if (res_hist) {
        og_apply_M(dim, m.lv[0].n, m.lv[0].h, order, a, x, r);
        for (long q = 0; q < N; ++q) r[q] = b[q] - r[q];
        res_hist[0] = og_norm2(N, r);
    }
    for (int cyc = 0; cyc < ncycles; ++cyc) {
        og_vcycle(&m, 0, b, x);
        if (res_hist) {
            og_apply_M(dim, m.lv[0].n, m.lv[0].h, order, a, x, r);
            for (long q = 0; q < N; ++q) r[q] = b[q] - r[q];
            res_hist[cyc + 1] = og_norm2(N, r);
        }
    }
    free(r);
    return m.nlev;
}
