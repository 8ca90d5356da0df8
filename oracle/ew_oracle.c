/*
 * ew_oracle.c -- plain, slow, FP64 CPU oracle for the EigenWave filter operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the bench
 * use it.  It shares no code, header or table with the CUDA library.
 *
 * Everything here is written for a reader checking it against the paper
 * (Appelo, Banks, Henshaw, Le, Schwendeman, "EigenWave", arXiv 2507.18282):
 *   - grid functions live on a Cartesian box (eq. eigBVPdiscrete) whose
 *     faces carry homogeneous Dirichlet conditions or, as the paper does for
 *     a symmetry plane, Neumann conditions; vectors hold the active points
 *     only, x fastest (Algorithm "matVec", Note 1): the interior points, plus
 *     the wall points of a Neumann face;
 *   - L_h is the 2nd-order (5/7-point) or 4th-order (9/13-point wide cross)
 *     centred Laplacian.  The boundary closure (the paper leaves the
 *     compatibility conditions out) is a reflection about the wall point:
 *     Dirichlet, u = 0 on the wall and the odd reflection u_{-j} = -u_{j}
 *     beyond it (u = 0 and u_xx = 0 on the wall); Neumann, the even
 *     reflection u_{-j} = u_{j} (the centred normal derivative vanishes);
 *   - the explicit scheme is eq. explicitScheme with the first step
 *     eq. explicitStep1, the implicit one eq. implicitScheme with
 *     M = I - (dt^2/2) L_h (eq. impMatrix) and first step eq. implicitStep1;
 *   - the filter is the trapezoidal sum eq. filterQuadrature; the caller
 *     passes the weights c_n = (2/T_f) sigma_n (cos(omega t^n) - alpha_d/2).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * rounding order is the order written below).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_G 2 /* ghost layers kept around the interior (enough for order 4) */

typedef struct {
    int dim;        /* 2 or 3 */
    long n[3];      /* active points per axis (n[2] = 1 in 2D) */
    double h[3];    /* grid spacing per axis */
    int order;      /* 2 or 4 */
    int neu[6];     /* face f = 2 axis + side (0 low, 1 high): 1 Neumann, 0 Dirichlet */
    long p[3];      /* padded extents */
    long npad;      /* padded size */
    long nact;      /* active size */
} og_grid;

/* bc: six face flags (1 = Neumann) or NULL for all Dirichlet */
static int og_init(og_grid* g, int dim, const long* n, const double* h, int order, const int* bc) {
    if (dim != 2 && dim != 3) return -1;
    if (order != 2 && order != 4) return -1;
    g->dim = dim;
    g->order = order;
    g->npad = 1;
    g->nact = 1;
    for (int f = 0; f < 6; ++f) g->neu[f] = (bc && f < 2 * dim) ? (bc[f] != 0) : 0;
    for (int a = 0; a < 3; ++a) {
        if (a < dim) {
            if (n[a] < 1) return -1;
            /* a Neumann ghost mirrors the point two in from the wall */
            if ((g->neu[2 * a] || g->neu[2 * a + 1]) && n[a] < 3) return -1;
            g->n[a] = n[a];
            g->h[a] = h[a];
            g->p[a] = n[a] + 2 * OG_G;
        } else {
            g->n[a] = 1;
            g->h[a] = 1.0;
            g->p[a] = 1;
        }
        g->npad *= g->p[a];
        g->nact *= g->n[a];
    }
    return 0;
}

/* padded index of active point (i, j, k), 0-based active coordinates; i = -1,
 * -2 and i = n, n+1 are the two layers beyond the active points on each side
 * (for a Dirichlet face: the wall point and a ghost; for a Neumann face,
 * whose wall point is active point 0 or n-1: two ghosts). */
static long og_at(const og_grid* g, long i, long j, long k) {
    long gi = i + OG_G;
    long gj = j + OG_G;
    long gk = (g->dim == 3) ? k + OG_G : 0;
    return (gk * g->p[1] + gj) * g->p[0] + gi;
}

/* copy the active vector into the padded grid function and fill the inactive
 * points from the boundary conditions (Algorithm matVec: vector -> grid, then
 * applyBoundaryConditions). */
static void og_scatter(const og_grid* g, const double* v, double* U) {
    memset(U, 0, sizeof(double) * (size_t)g->npad);
    long m = 0;
    for (long k = 0; k < g->n[2]; ++k)
        for (long j = 0; j < g->n[1]; ++j)
            for (long i = 0; i < g->n[0]; ++i) U[og_at(g, i, j, k)] = v[m++];
}

/* the two layers beyond one face of a line of points: U(x) for x = base +
 * t stride, t = -2 .. n+1, active for 0 <= t < n.
 *   Dirichlet low:  U(-1) = 0,      U(-2) = -U(0)     (odd about the wall t = -1)
 *   Neumann low:    U(-1) = U(1),   U(-2) = U(2)      (even about the wall t = 0)
 *   Dirichlet high: U(n) = 0,       U(n+1) = -U(n-1)  (odd about the wall t = n)
 *   Neumann high:   U(n) = U(n-2),  U(n+1) = U(n-3)   (even about the wall t = n-1) */
static void og_fill_line(double* U, long base, long stride, long n, int neu_lo, int neu_hi) {
#define AT(t) U[base + (t) * stride]
    if (neu_lo) {
        AT(-1) = AT(1);
        AT(-2) = AT(2);
    } else {
        AT(-1) = 0.0;
        AT(-2) = -AT(0);
    }
    if (neu_hi) {
        AT(n) = AT(n - 2);
        AT(n + 1) = AT(n - 3);
    } else {
        AT(n) = 0.0;
        AT(n + 1) = -AT(n - 1);
    }
#undef AT
}

/* fill the inactive layers of every line of active points, axis by axis (the
 * cross-shaped stencils never read the corner blocks). */
static void og_fill_bc(const og_grid* g, double* U) {
    long n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    long sy = g->p[0], sz = g->p[0] * g->p[1];
    for (long k = 0; k < n2; ++k)
        for (long j = 0; j < n1; ++j) og_fill_line(U, og_at(g, 0, j, k), 1, n0, g->neu[0], g->neu[1]);
    for (long k = 0; k < n2; ++k)
        for (long i = 0; i < n0; ++i) og_fill_line(U, og_at(g, i, 0, k), sy, n1, g->neu[2], g->neu[3]);
    if (g->dim == 3)
        for (long j = 0; j < n1; ++j)
            for (long i = 0; i < n0; ++i) og_fill_line(U, og_at(g, i, j, 0), sz, n2, g->neu[4], g->neu[5]);
}

/* L_h at one interior point of a padded grid function whose inactive points
 * are filled. */
static double og_lap_point(const og_grid* g, const double* U, long i, long j, long k) {
    long c = og_at(g, i, j, k);
    long stride[3];
    stride[0] = 1;
    stride[1] = g->p[0];
    stride[2] = g->p[0] * g->p[1];
    double sum = 0.0;
    for (int a = 0; a < g->dim; ++a) {
        long s = stride[a];
        double h2 = g->h[a] * g->h[a];
        double d2;
        if (g->order == 2) {
            d2 = (U[c - s] - 2.0 * U[c] + U[c + s]) / h2;
        } else {
            d2 = (-U[c - 2 * s] + 16.0 * U[c - s] - 30.0 * U[c] + 16.0 * U[c + s] - U[c + 2 * s]) /
                 (12.0 * h2);
        }
        sum += d2;
    }
    return sum;
}

/* Lu = L_h u on active vectors; bc: six face flags (1 = Neumann) or NULL. */
int og_apply_L(int dim, const long* n, const double* h, int order, const int* bc, const double* u, double* Lu) {
    og_grid g;
    if (og_init(&g, dim, n, h, order, bc)) return -1;
    double* U = (double*)malloc(sizeof(double) * (size_t)g.npad);
    if (!U) return -2;
    og_scatter(&g, u, U);
    og_fill_bc(&g, U);
    long m = 0;
    for (long k = 0; k < g.n[2]; ++k)
        for (long j = 0; j < g.n[1]; ++j)
            for (long i = 0; i < g.n[0]; ++i) Lu[m++] = og_lap_point(&g, U, i, j, k);
    free(U);
    return 0;
}

/* One application of the discrete EigenWave operator with explicit
 * leapfrog time stepping:
 *   W^0 = V,  W^1 = V + (dt^2/2) L_h V                       (eq. explicitStep1)
 *   W^{n+1} = 2 W^n - W^{n-1} + dt^2 L_h W^n,  n = 1..Nt-1   (eq. explicitScheme)
 *   out = sum_{n=0}^{Nt} c_n W^n                             (eq. filterQuadrature)
 * Arrays hold active points; c has Nt+1 entries. */
int og_filter_explicit(int dim, const long* n, const double* h, int order, const int* bc, long Nt, double dt,
                       const double* c, const double* v, double* out) {
    og_grid g;
    if (og_init(&g, dim, n, h, order, bc) || Nt < 1) return -1;
    size_t bytes = sizeof(double) * (size_t)g.npad;
    double* Wm = (double*)malloc(bytes); /* W^{n-1} */
    double* W0 = (double*)malloc(bytes); /* W^n     */
    double* Wp = (double*)malloc(bytes); /* W^{n+1} */
    if (!Wm || !W0 || !Wp) {
        free(Wm);
        free(W0);
        free(Wp);
        return -2;
    }
    double dt2 = dt * dt;
    og_scatter(&g, v, Wm);
    og_fill_bc(&g, Wm);
    memcpy(W0, Wm, bytes);
    for (long k = 0; k < g.n[2]; ++k)
        for (long j = 0; j < g.n[1]; ++j)
            for (long i = 0; i < g.n[0]; ++i) {
                long q = og_at(&g, i, j, k);
                W0[q] = Wm[q] + 0.5 * dt2 * og_lap_point(&g, Wm, i, j, k);
            }
    og_fill_bc(&g, W0);
    long m = 0;
    for (long k = 0; k < g.n[2]; ++k)
        for (long j = 0; j < g.n[1]; ++j)
            for (long i = 0; i < g.n[0]; ++i) {
                long q = og_at(&g, i, j, k);
                out[m++] = c[0] * Wm[q] + c[1] * W0[q];
            }
    for (long step = 1; step < Nt; ++step) {
        memset(Wp, 0, bytes);
        for (long k = 0; k < g.n[2]; ++k)
            for (long j = 0; j < g.n[1]; ++j)
                for (long i = 0; i < g.n[0]; ++i) {
                    long q = og_at(&g, i, j, k);
                    Wp[q] = 2.0 * W0[q] - Wm[q] + dt2 * og_lap_point(&g, W0, i, j, k);
                }
        og_fill_bc(&g, Wp);
        m = 0;
        for (long k = 0; k < g.n[2]; ++k)
            for (long j = 0; j < g.n[1]; ++j)
                for (long i = 0; i < g.n[0]; ++i) out[m++] += c[step + 1] * Wp[og_at(&g, i, j, k)];
        double* t = Wm;
        Wm = W0;
        W0 = Wp;
        Wp = t;
    }
    free(Wm);
    free(W0);
    free(Wp);
    return 0;
}

/* y = M x with M = I - a L_h, a = dt^2/2 (eq. impMatrix), active vectors. */
int og_apply_M(int dim, const long* n, const double* h, int order, double a, const double* x,
               double* y) {
    og_grid g;
    if (og_init(&g, dim, n, h, order, NULL)) return -1;
    double* L = (double*)malloc(sizeof(double) * (size_t)g.nact);
    if (!L) return -2;
    og_apply_L(dim, n, h, order, NULL, x, L);
    for (long m = 0; m < g.nact; ++m) y[m] = x[m] - a * L[m];
    free(L);
    return 0;
}

static double og_dot(long N, const double* x, const double* y) {
    double s = 0.0;
    for (long m = 0; m < N; ++m) s += x[m] * y[m];
    return s;
}

/* Conjugate gradients on the symmetric positive definite M = I - a L_h,
 * started from x = 0, stopped when ||b - M x|| <= tol ||b||.  Returns the
 * iteration count, or -1 on bad arguments / no convergence in maxit. */
int og_cg_solve_M(int dim, const long* n, const double* h, int order, double a, const double* b,
                  double* x, double tol, int maxit) {
    og_grid g;
    if (og_init(&g, dim, n, h, order, NULL)) return -1;
    long N = g.nact;
    double* r = (double*)malloc(sizeof(double) * (size_t)N);
    double* p = (double*)malloc(sizeof(double) * (size_t)N);
    double* Ap = (double*)malloc(sizeof(double) * (size_t)N);
    if (!r || !p || !Ap) {
        free(r);
        free(p);
        free(Ap);
        return -2;
    }
    for (long m = 0; m < N; ++m) {
        x[m] = 0.0;
        r[m] = b[m];
        p[m] = b[m];
    }
    double bb = og_dot(N, b, b);
    double rr = bb;
    int it = 0;
    if (bb == 0.0) goto done;
    for (it = 1; it <= maxit; ++it) {
        og_apply_M(dim, n, h, order, a, p, Ap);
        double alpha = rr / og_dot(N, p, Ap);
        for (long m = 0; m < N; ++m) {
            x[m] += alpha * p[m];
            r[m] -= alpha * Ap[m];
        }
        double rr_new = og_dot(N, r, r);
        if (sqrt(rr_new) <= tol * sqrt(bb)) {
            rr = rr_new;
            goto done;
        }
        double beta = rr_new / rr;
        rr = rr_new;
        for (long m = 0; m < N; ++m) p[m] = r[m] + beta * p[m];
    }
    it = -1;
done:
    free(r);
    free(p);
    free(Ap);
    return it;
}

/* One application of the discrete EigenWave operator with implicit
 * (trapezoidal-in-time) stepping, each system solved by CG to tol:
 *   M W^1 = W^0                                             (eq. implicitStep1)
 *   M W^{n+1} = 2 W^n - M W^{n-1}, i.e. W^{n+1} = M^{-1}(2 W^n) - W^{n-1}
 *                                                           (eq. implicitScheme)
 *   out = sum_{n=0}^{Nt} c_n W^n                            (eq. filterQuadrature) */
int og_filter_implicit(int dim, const long* n, const double* h, int order, long Nt, double dt,
                       const double* c, const double* v, double* out, double tol) {
    og_grid g;
    if (og_init(&g, dim, n, h, order, NULL) || Nt < 1) return -1;
    long N = g.nact;
    size_t bytes = sizeof(double) * (size_t)N;
    double a = 0.5 * dt * dt;
    double* Wm = (double*)malloc(bytes);
    double* W0 = (double*)malloc(bytes);
    double* rhs = (double*)malloc(bytes);
    double* y = (double*)malloc(bytes);
    int rc = 0;
    if (!Wm || !W0 || !rhs || !y) {
        rc = -2;
        goto out;
    }
    memcpy(Wm, v, bytes);
    if (og_cg_solve_M(dim, n, h, order, a, Wm, W0, tol, 100000) < 0) {
        rc = -3;
        goto out;
    }
    for (long m = 0; m < N; ++m) out[m] = c[0] * Wm[m] + c[1] * W0[m];
    for (long step = 1; step < Nt; ++step) {
        for (long m = 0; m < N; ++m) rhs[m] = 2.0 * W0[m];
        if (og_cg_solve_M(dim, n, h, order, a, rhs, y, tol, 100000) < 0) {
            rc = -3;
            goto out;
        }
        for (long m = 0; m < N; ++m) {
            double wp = y[m] - Wm[m];
            Wm[m] = W0[m];
            W0[m] = wp;
            out[m] += c[step + 1] * wp;
        }
    }
out:
    free(Wm);
    free(W0);
    free(rhs);
    free(y);
    return rc;
}

/* ------------------------------------------------------------------------
 * Single curvilinear grid by the mapping method (Section "Discrete
 * approximations": a smooth invertible map x = G(r) from the unit square,
 * the equations transformed by the chain rule and discretised by
 * conservative centred differences).  Two dimensions, second order, u = 0
 * on the boundary vertices.
 *
 * xy: the (n1 + 2) x (n2 + 2) vertex coordinates, interleaved (x, y), the r1
 * index fastest, boundary vertices included; the active points are the
 * n1 x n2 interior vertices; dr = 1 / (n1 + 1), ds = 1 / (n2 + 1).
 *
 * In the r coordinates
 *   J Lap u = d/dr (A11 u_r + A12 u_s) + d/ds (A12 u_r + A22 u_s),
 *   J = x_r y_s - x_s y_r,  A11 = (x_s^2 + y_s^2) / J,
 *   A22 = (x_r^2 + y_r^2) / J,  A12 = -(x_r x_s + y_r y_s) / J,
 * with the metric derivatives at every vertex by centred differences
 * (second-order one-sided ones on the boundary vertices).  At an active
 * vertex (i, j), with A at half points the average of its two vertices:
 *   J L u = [A11(i+1/2,j)(u(i+1,j) - u) - A11(i-1/2,j)(u - u(i-1,j))] / dr^2
 *         + [A22(i,j+1/2)(u(i,j+1) - u) - A22(i,j-1/2)(u - u(i,j-1))] / ds^2
 *         + [A12(i+1,j)(u(i+1,j+1) - u(i+1,j-1)) - A12(i-1,j)(u(i-1,j+1) - u(i-1,j-1))] / (4 dr ds)
 *         + [A12(i,j+1)(u(i+1,j+1) - u(i-1,j+1)) - A12(i,j-1)(u(i+1,j-1) - u(i-1,j-1))] / (4 dr ds)
 * ------------------------------------------------------------------------ */

typedef struct {
    long n1, n2;             /* active vertices per direction */
    long p1, p2;             /* vertices per direction (n + 2) */
    double dr, ds;
    double *J, *A11, *A12, *A22; /* at every vertex, p1 x p2, r1 fastest */
} om_grid;

static void om_free(om_grid* m) {
    free(m->J);
    free(m->A11);
    free(m->A12);
    free(m->A22);
}

/* derivative along one direction of the vertex line f(t) = xy[(base + t s) 2 + c],
 * t = 0 .. p-1, at t: centred inside, second-order one-sided at the ends */
static double om_diff(const double* xy, long base, long s, long p, long t, int c, double d) {
#define F(k) xy[2 * (base + (k) * s) + c]
    if (t == 0) return (-3.0 * F(0) + 4.0 * F(1) - F(2)) / (2.0 * d);
    if (t == p - 1) return (3.0 * F(p - 1) - 4.0 * F(p - 2) + F(p - 3)) / (2.0 * d);
    return (F(t + 1) - F(t - 1)) / (2.0 * d);
#undef F
}

static int om_init(om_grid* m, long n1, long n2, const double* xy) {
    if (n1 < 1 || n2 < 1) return -1;
    m->n1 = n1;
    m->n2 = n2;
    m->p1 = n1 + 2;
    m->p2 = n2 + 2;
    m->dr = 1.0 / (double)(n1 + 1);
    m->ds = 1.0 / (double)(n2 + 1);
    size_t np = (size_t)m->p1 * (size_t)m->p2;
    m->J = (double*)malloc(sizeof(double) * np);
    m->A11 = (double*)malloc(sizeof(double) * np);
    m->A12 = (double*)malloc(sizeof(double) * np);
    m->A22 = (double*)malloc(sizeof(double) * np);
    if (!m->J || !m->A11 || !m->A12 || !m->A22) {
        om_free(m);
        return -2;
    }
    for (long j = 0; j < m->p2; ++j)
        for (long i = 0; i < m->p1; ++i) {
            long q = j * m->p1 + i;
            double xr = om_diff(xy, j * m->p1, 1, m->p1, i, 0, m->dr);
            double yr = om_diff(xy, j * m->p1, 1, m->p1, i, 1, m->dr);
            double xs = om_diff(xy, i, m->p1, m->p2, j, 0, m->ds);
            double ys = om_diff(xy, i, m->p1, m->p2, j, 1, m->ds);
            double J = xr * ys - xs * yr;
            if (!(J > 0.0)) {
                om_free(m);
                return -3; /* the map must preserve orientation */
            }
            m->J[q] = J;
            m->A11[q] = (xs * xs + ys * ys) / J;
            m->A22[q] = (xr * xr + yr * yr) / J;
            m->A12[q] = -(xr * xs + yr * ys) / J;
        }
    return 0;
}

/* L u at active vertex (i, j) (vertex indices 1..n) of a vertex array U with
 * zeros on the boundary vertices */
static double om_lap_point(const om_grid* m, const double* U, long i, long j) {
    long p = m->p1;
#define V(a, b) U[(b) * p + (a)]
#define A(arr, a, b) m->arr[(b) * p + (a)]
    double u = V(i, j);
    double a11p = 0.5 * (A(A11, i, j) + A(A11, i + 1, j)), a11m = 0.5 * (A(A11, i, j) + A(A11, i - 1, j));
    double a22p = 0.5 * (A(A22, i, j) + A(A22, i, j + 1)), a22m = 0.5 * (A(A22, i, j) + A(A22, i, j - 1));
    double t_rr = (a11p * (V(i + 1, j) - u) - a11m * (u - V(i - 1, j))) / (m->dr * m->dr);
    double t_ss = (a22p * (V(i, j + 1) - u) - a22m * (u - V(i, j - 1))) / (m->ds * m->ds);
    double t_rs = (A(A12, i + 1, j) * (V(i + 1, j + 1) - V(i + 1, j - 1)) -
                   A(A12, i - 1, j) * (V(i - 1, j + 1) - V(i - 1, j - 1))) / (4.0 * m->dr * m->ds);
    double t_sr = (A(A12, i, j + 1) * (V(i + 1, j + 1) - V(i - 1, j + 1)) -
                   A(A12, i, j - 1) * (V(i + 1, j - 1) - V(i - 1, j - 1))) / (4.0 * m->dr * m->ds);
    return (t_rr + t_ss + t_rs + t_sr) / A(J, i, j);
#undef V
#undef A
}

static void om_scatter(const om_grid* m, const double* v, double* U) {
    memset(U, 0, sizeof(double) * (size_t)m->p1 * (size_t)m->p2);
    long q = 0;
    for (long j = 1; j <= m->n2; ++j)
        for (long i = 1; i <= m->n1; ++i) U[j * m->p1 + i] = v[q++];
}

/* Lu = L u on active vectors of the mapped grid */
int og_mapped_apply_L(long n1, long n2, const double* xy, const double* u, double* Lu) {
    om_grid m;
    int rc = om_init(&m, n1, n2, xy);
    if (rc) return rc;
    double* U = (double*)malloc(sizeof(double) * (size_t)m.p1 * (size_t)m.p2);
    if (!U) {
        om_free(&m);
        return -2;
    }
    om_scatter(&m, u, U);
    long q = 0;
    for (long j = 1; j <= n2; ++j)
        for (long i = 1; i <= n1; ++i) Lu[q++] = om_lap_point(&m, U, i, j);
    free(U);
    om_free(&m);
    return 0;
}

/* J at the active vertices: the weights of the discrete L2 inner product in
 * which the conservative L is symmetric */
int og_mapped_jacobian(long n1, long n2, const double* xy, double* J) {
    om_grid m;
    int rc = om_init(&m, n1, n2, xy);
    if (rc) return rc;
    long q = 0;
    for (long j = 1; j <= n2; ++j)
        for (long i = 1; i <= n1; ++i) J[q++] = m.J[j * m.p1 + i];
    om_free(&m);
    return 0;
}

/* S v on the mapped grid with explicit leapfrog (eqs. explicitScheme,
 * explicitStep1, filterQuadrature), as og_filter_explicit */
int og_mapped_filter_explicit(long n1, long n2, const double* xy, long Nt, double dt, const double* c,
                              const double* v, double* out) {
    om_grid m;
    int rc = om_init(&m, n1, n2, xy);
    if (rc) return rc;
    if (Nt < 1) {
        om_free(&m);
        return -1;
    }
    size_t np = (size_t)m.p1 * (size_t)m.p2;
    double* Wm = (double*)malloc(sizeof(double) * np);
    double* W0 = (double*)malloc(sizeof(double) * np);
    double* Wp = (double*)malloc(sizeof(double) * np);
    if (!Wm || !W0 || !Wp) {
        free(Wm);
        free(W0);
        free(Wp);
        om_free(&m);
        return -2;
    }
    double dt2 = dt * dt;
    om_scatter(&m, v, Wm);
    memcpy(W0, Wm, sizeof(double) * np);
    for (long j = 1; j <= n2; ++j)
        for (long i = 1; i <= n1; ++i) W0[j * m.p1 + i] = Wm[j * m.p1 + i] + 0.5 * dt2 * om_lap_point(&m, Wm, i, j);
    long q = 0;
    for (long j = 1; j <= n2; ++j)
        for (long i = 1; i <= n1; ++i, ++q) out[q] = c[0] * Wm[j * m.p1 + i] + c[1] * W0[j * m.p1 + i];
    memset(Wp, 0, sizeof(double) * np);
    for (long step = 1; step < Nt; ++step) {
        for (long j = 1; j <= n2; ++j)
            for (long i = 1; i <= n1; ++i) {
                long k = j * m.p1 + i;
                Wp[k] = 2.0 * W0[k] - Wm[k] + dt2 * om_lap_point(&m, W0, i, j);
            }
        q = 0;
        for (long j = 1; j <= n2; ++j)
            for (long i = 1; i <= n1; ++i, ++q) out[q] += c[step + 1] * Wp[j * m.p1 + i];
        double* t = Wm;
        Wm = W0;
        W0 = Wp;
        Wp = t;
    }
    free(Wm);
    free(W0);
    free(Wp);
    om_free(&m);
    return 0;
}
