/*
 * Plain FP64 CPU oracle of the Flow-Opt Safety-Filter (SF) iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code;
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code with the CUDA path.
 *
 * What it computes (paper: Sec. IV-B "Fast Inference-Time Refinement" and the
 * Appendix "Derivation of Fixed-Point Iteration Form"):
 *   the projection problem  min 1/2 ||xi_bar - xi||^2  s.t.  A xi_bar = b,
 *   G xi_bar <= h,  g(xi_bar) <= 0  (eqs. proj_cost..proj_robot), rewritten with
 *   the spherical form of the collision constraints (eqs. inter_robot_polar,
 *   workspace_polar, reformulated problem, f_e) and solved by alternating
 *   minimisation of the augmented Lagrangian (eq. aug_lag) in the step order
 *   alpha, beta, d, s, lambda, xi_bar (eqs. alpha_step..xi_step).
 *
 * Everything is written out from the definitions: the constraint matrices F, G,
 * A are applied row by row exactly as the Appendix builds them, the xi_bar step
 * solves the equality-constrained QP by a Cholesky factorisation of its Hessian
 * and the Schur complement of A (no explicit inverse), and the alpha/beta/d
 * steps use the trigonometric closed forms.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  R1  basis: Bernstein polynomials of degree n_xi-1 at tau_k = k/(H-1); the paper
 *      names no family.  A selects coefficient 0 and n_xi-1 (start/goal).
 *  R2  F_r = D (x) W with D the pair incidence (row e_i - e_j, i<j, pairs ordered
 *      i-major), F_o = blockdiag_i(stack_m W); the dimension table's "P" is W.
 *  R3  G = [I (x) W; -I (x) W], h = [p_max; -p_min]: a two-sided box.
 *  R4  slack step s = max(0, h - G xi_bar); the printed sign (-G xi_bar - h) is a garble.
 *  R5  r_1 uses the current iterate xi_bar (printed "F xi").
 *  R6  xi_bar step: argmin of the full augmented Lagrangian, so the Hessian is
 *      I + rho F'F + rho G'G and the right-hand side carries rho G'(h - s);
 *      ws_hess = 0 gives the matrix and eta as printed (no G terms).
 *  R7  beta: the minimiser in M^-1-scaled coordinates,
 *        beta = atan2((dx cos a + dy sin a)/a, dz/b);
 *      d: the clamped least-squares minimiser given alpha, beta,
 *        d = max(1, (a sin b (dx cos a + dy sin a) + b cos b dz)/(a^2 sin^2 b + b^2 cos^2 b)).
 *      2D rows have beta = pi/2 and no z component.
 *  R8  residuals: ||r_p|| = sqrt(||r_1||^2 + ||r_2||^2) (eq. primal_residual adds
 *      vectors of different length); "max residual" = max over constraint rows
 *      of the Euclidean norm of the row's r_1 block and over workspace rows of r_2;
 *      fixed-point residual = ||z^{l+1} - z^l||_2 (eq. fixed_point_residual as printed
 *      is identically zero).
 *  R9  derivative conventions: d/dx max(1,x) = [x > 1], d/dx max(0,x) = [x > 0],
 *      atan2(0,0) = 0 with zero derivative.
 *
 * Cost modes.  cost = 0: the SF projection cost above.  cost = 1: the trajectory
 * optimiser of eq. eq::form with the smoothness cost of eq. cost,
 * 1/2 sum_i sum_k ||p''_{i|k}||^2 = 1/2 xi' Q xi with Q = blockdiag(Wdd' Wdd) and q = 0,
 * solved by the same alternating minimisation: the Hessian of the xi_bar step becomes
 * Q + rho F'F + rho G'G and its right-hand side loses the candidate term.
 *  R13 time scale: p'' is taken with respect to time t = tau (H - 1) dt, dt a parameter
 *      (the paper gives no time step); the smoothness mode needs the workspace terms in
 *      the Hessian (ws_hess = 1), which make it positive definite.
 *  R14 initial-velocity boundary rows (Sec. V, hardware experiments: the planner is
 *      conditioned on the robots' initial velocities): with nbc = 3 each robot and axis
 *      adds the row p'(t = 0) = v_0 to A, the first time derivative of the basis at
 *      tau = 0 in the time of R13; the boundary values per robot and axis are then
 *      (start, goal, v_0).  For Bernstein the row fixes coefficient 1 as well.
 *  R15 self-supervised loss (eq. NN_loss): sum over l = 0..L-1 of
 *      L_FP = ||z^{l+1} - z^l||^2 with z = (xi_bar, lambda) (the fixed-point residual of
 *      eq. fixed_point_residual read as in R8), weighted by g_fp in the reverse pass;
 *      the term ||xi_bar^L - xi||^2 enters through the ordinary output seed.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SFO_NHIST 4 /* per-iteration history: ||r_p||, max residual, FP residual, kink margin */

typedef struct {
    int nd, nxi, n, nobs, H, dyn, ws_hess, cost, nbc;
    double rho, a, b, dt;
    const double *pmin, *pmax, *obs_c, *obs_ab, *bnd, *xi;
} prob_t;

typedef struct {
    int N, npair, rows_pair, rows_obs, rows_F, rows_G;
    double *W;   /* H x nxi basis                                   */
    double *L;   /* Cholesky factor of the xi_bar-step Hessian, N x N */
    double *Y;   /* H^-1 A^T, N x nbc n                              */
    double *LS;  /* Cholesky factor of S = A H^-1 A^T, nbc n square */
    double *Wd0; /* first time derivative of the basis at tau = 0 (R14) */
    int *pi, *pj; /* pair list in F_r row order                     */
} ctx_t;

/* ---------------------------------------------------------------- basis (R1) */
static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; i++) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* W[k][c] = C(n_xi-1, c) tau^c (1-tau)^(n_xi-1-c), tau = k/(H-1)  (eq. poly, reading R1) */
int sfo_basis(int H, int nxi, double *W)
{
    if (H < 2 || nxi < 2) return -1;
    int deg = nxi - 1;
    for (int k = 0; k < H; k++) {
        double tau = (double)k / (double)(H - 1);
        for (int c = 0; c < nxi; c++)
            W[k * nxi + c] = binom(deg, c) * pow(tau, c) * pow(1.0 - tau, deg - c);
    }
    return 0;
}

/* Wdd[k][c] = d^2/dt^2 of the c-th basis polynomial at t_k = tau_k T, T = (H-1) dt:
   the second derivative of a degree-d Bernstein polynomial is d (d-1) times the second
   difference of the degree-(d-2) polynomials, scaled by 1/T^2 (reading R13). */
int sfo_basis_dd(int H, int nxi, double dt, double *Wdd)
{
    if (H < 2 || nxi < 3 || !(dt > 0.0)) return -1;
    int deg = nxi - 1;
    double T = (double)(H - 1) * dt;
    double scale = (double)deg * (double)(deg - 1) / (T * T);
    for (int k = 0; k < H; k++) {
        const double tau = k / (H - 1.0);
        for (int c = 0; c < nxi; c++) {
            double v = 0.0;
            for (int j = c - 2; j <= c; j++) {
                if (j < 0 || j > deg - 2) continue;
                double w = j == c - 1 ? -2.0 : 1.0;
                v += w * binom(deg - 2, j) * pow(tau, j) * pow(1.0 - tau, deg - 2 - j);
            }
            Wdd[k * nxi + c] = scale * v;
        }
    }
    return 0;
}

/* Wd[k][c] = d/dt of the c-th basis polynomial at t_k = tau_k T, T = (H-1) dt: a
   degree-d Bernstein polynomial's derivative is d times the first difference of the
   degree-(d-1) polynomials, scaled by 1/T (readings R13, R14). */
int sfo_basis_d(int H, int nxi, double dt, double *Wd)
{
    if (H < 2 || nxi < 2 || !(dt > 0.0)) return -1;
    int deg = nxi - 1;
    double T = (double)(H - 1) * dt;
    for (int k = 0; k < H; k++) {
        const double tau = k / (H - 1.0);
        for (int c = 0; c < nxi; c++) {
            double v = 0.0;
            for (int j = c - 1; j <= c; j++) {
                if (j < 0 || j > deg - 1) continue;
                double w = j == c - 1 ? 1.0 : -1.0;
                v += w * binom(deg - 1, j) * pow(tau, j) * pow(1.0 - tau, deg - 1 - j);
            }
            Wd[k * nxi + c] = (double)deg * v / T;
        }
    }
    return 0;
}

/* ------------------------------------------------------- dense linear algebra */
static int cholesky(int m, double *A) /* in place, lower; returns 0 on success */
{
    for (int j = 0; j < m; j++) {
        double s = A[j * m + j];
        for (int k = 0; k < j; k++) s -= A[j * m + k] * A[j * m + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        A[j * m + j] = d;
        for (int i = j + 1; i < m; i++) {
            double t = A[i * m + j];
            for (int k = 0; k < j; k++) t -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = t / d;
        }
        for (int i = 0; i < j; i++) A[i * m + j] = 0.0;
    }
    return 0;
}

static void chol_solve(int m, const double *L, double *x) /* solves L L^T x = x */
{
    for (int i = 0; i < m; i++) {
        double t = x[i];
        for (int k = 0; k < i; k++) t -= L[i * m + k] * x[k];
        x[i] = t / L[i * m + i];
    }
    for (int i = m - 1; i >= 0; i--) {
        double t = x[i];
        for (int k = i + 1; k < m; k++) t -= L[k * m + i] * x[k];
        x[i] = t / L[i * m + i];
    }
}

/* --------------------------------------------------------- constraint rows (R2, R3) */
/* Row r of one axis block of F (eq. f_e): pair rows first (F_r), then obstacle rows (F_o).
   Pair row (p, k): +W[k] on robot pi[p], -W[k] on robot pj[p].
   Obstacle row ((i, m), k): +W[k] on robot i. */
static void F_row(const prob_t *P, const ctx_t *C, int r, int *bi, int *bj, int *k, int *m)
{
    if (r < C->rows_pair) {
        int p = r / P->H;
        *k = r % P->H;
        *bi = C->pi[p];
        *bj = C->pj[p];
        *m = -1;
    } else {
        int q = r - C->rows_pair;
        *k = q % P->H;
        int im = q / P->H;
        *bi = im / P->nobs;
        *m = im % P->nobs;
        *bj = -1;
    }
}

/* y = F_axis xi_axis */
static void F_apply(const prob_t *P, const ctx_t *C, const double *x, double *y)
{
    for (int r = 0; r < C->rows_F; r++) {
        int bi, bj, k, m;
        F_row(P, C, r, &bi, &bj, &k, &m);
        double s = 0.0;
        for (int c = 0; c < P->nxi; c++) {
            double v = x[bi * P->nxi + c];
            if (bj >= 0) v -= x[bj * P->nxi + c];
            s += C->W[k * P->nxi + c] * v;
        }
        y[r] = s;
    }
}

/* out += F_axis^T z */
static void FT_apply(const prob_t *P, const ctx_t *C, const double *z, double *out)
{
    for (int r = 0; r < C->rows_F; r++) {
        int bi, bj, k, m;
        F_row(P, C, r, &bi, &bj, &k, &m);
        for (int c = 0; c < P->nxi; c++) {
            out[bi * P->nxi + c] += C->W[k * P->nxi + c] * z[r];
            if (bj >= 0) out[bj * P->nxi + c] -= C->W[k * P->nxi + c] * z[r];
        }
    }
}

/* G rows of one axis: upper row (i,k) = +W[k] on robot i, lower row (i,k) = -W[k] on robot i */
static void G_apply(const prob_t *P, const ctx_t *C, const double *x, double *q)
{
    int nH = P->n * P->H;
    for (int i = 0; i < P->n; i++)
        for (int k = 0; k < P->H; k++) {
            double s = 0.0;
            for (int c = 0; c < P->nxi; c++) s += C->W[k * P->nxi + c] * x[i * P->nxi + c];
            q[i * P->H + k] = s;
            q[nH + i * P->H + k] = -s;
        }
}

static void GT_apply(const prob_t *P, const ctx_t *C, const double *z, double *out)
{
    int nH = P->n * P->H;
    for (int i = 0; i < P->n; i++)
        for (int k = 0; k < P->H; k++)
            for (int c = 0; c < P->nxi; c++)
                out[i * P->nxi + c] += C->W[k * P->nxi + c] * (z[i * P->H + k] - z[nH + i * P->H + k]);
}

static double h_of(const prob_t *P, int ax, int g) /* h = [p_max; -p_min] */
{
    return g < P->n * P->H ? P->pmax[ax] : -P->pmin[ax];
}

/* Boundary row s of one robot (eq. boundary_con): s = 0 the start W[0], s = 1 the goal
   W[H-1], s = 2 the initial velocity p'(0) (reading R14). */
static const double *A_row(const prob_t *P, const ctx_t *C, int s)
{
    return s == 2 ? C->Wd0 : C->W + (size_t)(s ? P->H - 1 : 0) * P->nxi;
}

/* A rows of one axis: row nbc i + s is boundary row s on robot i */
static void A_apply(const prob_t *P, const ctx_t *C, const double *x, double *y)
{
    for (int i = 0; i < P->n; i++)
        for (int s = 0; s < P->nbc; s++) {
            const double *w = A_row(P, C, s);
            double t = 0.0;
            for (int c = 0; c < P->nxi; c++) t += w[c] * x[i * P->nxi + c];
            y[P->nbc * i + s] = t;
        }
}

static void AT_apply(const prob_t *P, const ctx_t *C, const double *nu, double *out)
{
    for (int i = 0; i < P->n; i++)
        for (int s = 0; s < P->nbc; s++) {
            const double *w = A_row(P, C, s);
            for (int c = 0; c < P->nxi; c++) out[i * P->nxi + c] += w[c] * nu[P->nbc * i + s];
        }
}

/* ------------------------------------------------------ alpha, beta, d steps (R7) */
/* For one constraint row with line-of-sight vector D (relative to the row's centre),
   the closed-form alpha, beta, d minimisers (eqs. alpha_step, beta_step, d_step) and
   e = d (A cos a sin b, A sin a sin b, Bz cos b) (eq. inter_robot_polar).  If J is
   given, J[r*nd+q] = d e_r / d D_q (forward-mode chain rule, conventions R9).
   tmargin (optional) returns |t - 1| for the d clamp. */
static void estep(int nd, const double *D, double A, double Bz, double *e, double *J, double *tmargin)
{
    double dx = D[0], dy = D[1], dz = nd == 3 ? D[2] : 0.0;
    double alpha = atan2(dy, dx);
    double ca = cos(alpha), sa = sin(alpha);
    double w = dx * ca + dy * sa;
    double sb = 1.0, cb = 0.0, u1 = 0.0, u2 = 0.0;
    if (nd == 3) {
        u1 = w / A;
        u2 = dz / Bz;
        double beta = atan2(u1, u2);
        sb = sin(beta);
        cb = cos(beta);
    }
    double num = A * sb * w + Bz * cb * dz;
    double den = A * A * sb * sb + Bz * Bz * cb * cb;
    double t = num / den;
    double d = t > 1.0 ? t : 1.0;
    e[0] = d * A * ca * sb;
    e[1] = d * A * sa * sb;
    if (nd == 3) e[2] = d * Bz * cb;
    if (tmargin) *tmargin = fabs(t - 1.0);
    if (!J) return;
    double r2 = dx * dx + dy * dy;
    for (int q = 0; q < nd; q++) {
        double ddx = q == 0, ddy = q == 1, ddz = q == 2;
        double dal = r2 > 0.0 ? (-dy * ddx + dx * ddy) / r2 : 0.0;
        double dca = -sa * dal, dsa = ca * dal;
        double dw = ddx * ca + dx * dca + ddy * sa + dy * dsa;
        double dsb = 0.0, dcb = 0.0;
        if (nd == 3) {
            double q2 = u1 * u1 + u2 * u2;
            double du1 = dw / A, du2 = ddz / Bz;
            double dbe = q2 > 0.0 ? (u2 * du1 - u1 * du2) / q2 : 0.0;
            dsb = cb * dbe;
            dcb = -sb * dbe;
        }
        double dnum = A * (dsb * w + sb * dw) + Bz * (dcb * dz + cb * ddz);
        double dden = 2.0 * A * A * sb * dsb + 2.0 * Bz * Bz * cb * dcb;
        double dt = (dnum * den - num * dden) / (den * den);
        double dd = t > 1.0 ? dt : 0.0;
        J[0 * nd + q] = A * (dd * ca * sb + d * dca * sb + d * ca * dsb);
        J[1 * nd + q] = A * (dd * sa * sb + d * dsa * sb + d * sa * dsb);
        if (nd == 3) J[2 * nd + q] = Bz * (dd * cb + d * dcb);
    }
}

/* exported for the brute-force and geometry pins */
int sfo_estep(int nd, const double *D, double A, double Bz, double *e, double *J)
{
    estep(nd, D, A, Bz, e, J, NULL);
    return 0;
}

/* centre of obstacle m at timestep k (static or per-timestep) */
static const double *obs_at(const prob_t *P, int m, int k)
{
    return P->dyn ? P->obs_c + ((size_t)m * P->H + k) * P->nd : P->obs_c + (size_t)m * P->nd;
}

/* ------------------------------------------------------------------ set-up */
static void ctx_free(ctx_t *C)
{
    free(C->W); free(C->L); free(C->Y); free(C->LS); free(C->pi); free(C->pj); free(C->Wd0);
    memset(C, 0, sizeof(*C));
}

/* Builds W, the Hessian H = I + rho F'F (+ rho G'G) of the xi_bar step by accumulating
   the outer products of the constraint rows, its Cholesky factor, Y = H^-1 A^T and the
   Cholesky factor of S = A Y (eq. xi_step and the KKT matrix M). */
static int ctx_init(const prob_t *P, ctx_t *C)
{
    memset(C, 0, sizeof(*C));
    int nxi = P->nxi, n = P->n, H = P->H;
    int N = n * nxi;
    C->N = N;
    C->npair = n * (n - 1) / 2;
    C->rows_pair = C->npair * H;
    C->rows_obs = n * P->nobs * H;
    C->rows_F = C->rows_pair + C->rows_obs;
    C->rows_G = 2 * n * H;
    const int m = P->nbc * n;
    C->W = malloc(sizeof(double) * H * nxi);
    C->L = calloc((size_t)N * N, sizeof(double));
    C->Y = calloc((size_t)N * m, sizeof(double));
    C->LS = calloc((size_t)m * m, sizeof(double));
    C->pi = malloc(sizeof(int) * (C->npair + 1));
    C->pj = malloc(sizeof(int) * (C->npair + 1));
    C->Wd0 = calloc(nxi, sizeof(double));
    if (!C->W || !C->L || !C->Y || !C->LS || !C->pi || !C->pj || !C->Wd0) { ctx_free(C); return -2; }
    sfo_basis(H, nxi, C->W);
    if (P->nbc == 3) {
        double *Wd = malloc(sizeof(double) * H * nxi);
        if (!Wd || sfo_basis_d(H, nxi, P->dt, Wd)) { free(Wd); ctx_free(C); return -1; }
        memcpy(C->Wd0, Wd, sizeof(double) * nxi);   /* row tau = 0 */
        free(Wd);
    }
    int p = 0;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) { C->pi[p] = i; C->pj[p] = j; p++; }

    double *Hm = C->L;
    double *f = malloc(sizeof(double) * N);
    for (int r = 0; r < C->rows_F; r++) {
        int bi, bj, k, m;
        F_row(P, C, r, &bi, &bj, &k, &m);
        memset(f, 0, sizeof(double) * N);
        for (int c = 0; c < nxi; c++) {
            f[bi * nxi + c] += C->W[k * nxi + c];
            if (bj >= 0) f[bj * nxi + c] -= C->W[k * nxi + c];
        }
        for (int u = 0; u < N; u++)
            if (f[u] != 0.0)
                for (int v = 0; v < N; v++) Hm[u * N + v] += P->rho * f[u] * f[v];
    }
    if (P->ws_hess) {
        for (int i = 0; i < n; i++)
            for (int k = 0; k < H; k++)
                for (int side = 0; side < 2; side++) {
                    double sg = side ? -1.0 : 1.0;
                    for (int u = 0; u < nxi; u++)
                        for (int v = 0; v < nxi; v++)
                            Hm[(i * nxi + u) * N + i * nxi + v] +=
                                P->rho * (sg * C->W[k * nxi + u]) * (sg * C->W[k * nxi + v]);
                }
    }
    if (P->cost == 0) {
        for (int u = 0; u < N; u++) Hm[u * N + u] += 1.0;   /* 1/2 ||xi_bar - xi||^2 */
    } else {                                                /* 1/2 xi' Q xi, one block per robot */
        double *Wdd = malloc(sizeof(double) * H * nxi);
        if (!Wdd || sfo_basis_dd(H, nxi, P->dt, Wdd)) { free(Wdd); free(f); ctx_free(C); return -1; }
        for (int i = 0; i < n; i++)
            for (int u = 0; u < nxi; u++)
                for (int v = 0; v < nxi; v++) {
                    double q = 0.0;
                    for (int k = 0; k < H; k++) q += Wdd[k * nxi + u] * Wdd[k * nxi + v];
                    Hm[(i * nxi + u) * N + i * nxi + v] += q;
                }
        free(Wdd);
    }
    free(f);
    if (cholesky(N, C->L)) { ctx_free(C); return -3; }

    /* Y = H^-1 A^T, column by column */
    double *col = malloc(sizeof(double) * N);
    double *unit = calloc(m, sizeof(double));
    for (int q = 0; q < m; q++) {
        memset(col, 0, sizeof(double) * N);
        unit[q] = 1.0;
        AT_apply(P, C, unit, col);
        unit[q] = 0.0;
        chol_solve(N, C->L, col);
        for (int u = 0; u < N; u++) C->Y[u * m + q] = col[u];
    }
    /* S = A Y */
    double *ay = malloc(sizeof(double) * m);
    for (int q = 0; q < m; q++) {
        for (int u = 0; u < N; u++) col[u] = C->Y[u * m + q];
        A_apply(P, C, col, ay);
        for (int r = 0; r < m; r++) C->LS[r * m + q] = ay[r];
    }
    free(col); free(unit); free(ay);
    if (cholesky(m, C->LS)) { ctx_free(C); return -3; }
    return 0;
}

/* x = argmin 1/2 x'Hx - eta'x  s.t.  A x = bb   (eq. xi_step; KKT with Schur complement)
   bb may be NULL for b = 0. */
static void kkt_solve(const prob_t *P, const ctx_t *C, const double *eta, const double *bb, double *x)
{
    int N = C->N, m = P->nbc * P->n;
    double *u = malloc(sizeof(double) * m);
    memcpy(x, eta, sizeof(double) * N);
    chol_solve(N, C->L, x);             /* t = H^-1 eta            */
    A_apply(P, C, x, u);                /* u = A t - b             */
    if (bb) for (int r = 0; r < m; r++) u[r] -= bb[r];
    chol_solve(m, C->LS, u);            /* nu = S^-1 (A t - b)      */
    for (int v = 0; v < N; v++) {       /* x = t - H^-1 A^T nu      */
        double s = 0.0;
        for (int r = 0; r < m; r++) s += C->Y[v * m + r] * u[r];
        x[v] -= s;
    }
    free(u);
}

/* ------------------------------------------------------------ one T application */
typedef struct {
    double *y, *e, *r1;   /* per axis x rows_F */
    double *q, *s, *r2;   /* per axis x rows_G */
    double *v1, *v2;      /* per axis x N       */
} buf_t;

static int buf_init(const prob_t *P, const ctx_t *C, buf_t *B)
{
    size_t RF = (size_t)P->nd * C->rows_F, RG = (size_t)P->nd * C->rows_G, NN = (size_t)P->nd * C->N;
    B->y = malloc(sizeof(double) * RF);
    B->e = malloc(sizeof(double) * RF);
    B->r1 = malloc(sizeof(double) * RF);
    B->q = malloc(sizeof(double) * RG);
    B->s = malloc(sizeof(double) * RG);
    B->r2 = malloc(sizeof(double) * RG);
    B->v1 = malloc(sizeof(double) * NN);
    B->v2 = malloc(sizeof(double) * NN);
    return (B->y && B->e && B->r1 && B->q && B->s && B->r2 && B->v1 && B->v2) ? 0 : -2;
}

static void buf_free(buf_t *B)
{
    free(B->y); free(B->e); free(B->r1); free(B->q); free(B->s); free(B->r2); free(B->v1); free(B->v2);
}

/* Evaluates, at xi_bar: y = F xi_bar, the alpha/beta/d steps giving e, s = max(0, h - G xi_bar),
   r_1 = y - e and r_2 = G xi_bar - h + s.  Returns ||r_p||^2 in st[0], max residual in st[1],
   kink margin in st[2]. */
static void evaluate(const prob_t *P, const ctx_t *C, const double *xib, buf_t *B, double *st)
{
    int nd = P->nd, RF = C->rows_F, RG = C->rows_G, N = C->N;
    for (int ax = 0; ax < nd; ax++) {
        F_apply(P, C, xib + (size_t)ax * N, B->y + (size_t)ax * RF);
        G_apply(P, C, xib + (size_t)ax * N, B->q + (size_t)ax * RG);
    }
    double rp2 = 0.0, mx = 0.0, kink = INFINITY;
    for (int r = 0; r < RF; r++) {
        int bi, bj, k, m;
        F_row(P, C, r, &bi, &bj, &k, &m);
        double D[3], ev[3], tm;
        const double *po = m >= 0 ? obs_at(P, m, k) : NULL;
        for (int ax = 0; ax < nd; ax++) D[ax] = B->y[(size_t)ax * RF + r] - (po ? po[ax] : 0.0);
        double A = m >= 0 ? P->obs_ab[2 * m] : P->a;
        double Bz = m >= 0 ? P->obs_ab[2 * m + 1] : P->b;
        estep(nd, D, A, Bz, ev, NULL, &tm);
        if (tm < kink) kink = tm;
        double rn = 0.0;
        for (int ax = 0; ax < nd; ax++) {
            double e = ev[ax] + (po ? po[ax] : 0.0);
            B->e[(size_t)ax * RF + r] = e;
            double r1 = B->y[(size_t)ax * RF + r] - e;
            B->r1[(size_t)ax * RF + r] = r1;
            rn += r1 * r1;
        }
        rp2 += rn;
        if (sqrt(rn) > mx) mx = sqrt(rn);
    }
    for (int ax = 0; ax < nd; ax++)
        for (int g = 0; g < RG; g++) {
            size_t o = (size_t)ax * RG + g;
            double h = h_of(P, ax, g);
            double s = h - B->q[o];
            if (fabs(s) < kink) kink = fabs(s);
            s = s > 0.0 ? s : 0.0;
            B->s[o] = s;
            double r2 = B->q[o] - h + s;
            B->r2[o] = r2;
            rp2 += r2 * r2;
            if (r2 > mx) mx = r2;
        }
    st[0] = rp2;
    st[1] = mx;
    st[2] = kink;
}

/* T(xi_bar, lambda) -> (xi_bar', lambda')  (eq. fixed_point; steps alpha..xi in order) */
static void T_apply(const prob_t *P, const ctx_t *C, const double *xib, const double *lam,
                    double *xib_new, double *lam_new, buf_t *B, double *st)
{
    int nd = P->nd, RF = C->rows_F, RG = C->rows_G, N = C->N;
    evaluate(P, C, xib, B, st);
    /* lambda step (eq. lambda_step): lambda - rho F'r_1 - rho G'r_2 */
    for (int ax = 0; ax < nd; ax++) {
        double *g = B->v1 + (size_t)ax * N;
        memset(g, 0, sizeof(double) * N);
        FT_apply(P, C, B->r1 + (size_t)ax * RF, g);
        GT_apply(P, C, B->r2 + (size_t)ax * RG, g);
        for (int u = 0; u < N; u++) lam_new[(size_t)ax * N + u] = lam[(size_t)ax * N + u] - P->rho * g[u];
    }
    /* xi_bar step (eq. xi_step): eta = xi + lambda' + rho F'e (+ rho G'(h - s)), KKT solve
       (the smoothness cost has no linear term: eta = lambda' + ...) */
    double *hs = malloc(sizeof(double) * RG);
    double *bb = malloc(sizeof(double) * P->nbc * P->n);
    for (int ax = 0; ax < nd; ax++) {
        double *eta = B->v2 + (size_t)ax * N;
        for (int u = 0; u < N; u++)
            eta[u] = (P->cost == 0 ? P->xi[(size_t)ax * N + u] : 0.0) + lam_new[(size_t)ax * N + u];
        double *fe = B->v1 + (size_t)ax * N;
        memset(fe, 0, sizeof(double) * N);
        FT_apply(P, C, B->e + (size_t)ax * RF, fe);
        if (P->ws_hess) {
            for (int g = 0; g < RG; g++) hs[g] = h_of(P, ax, g) - B->s[(size_t)ax * RG + g];
            GT_apply(P, C, hs, fe);
        }
        for (int u = 0; u < N; u++) eta[u] += P->rho * fe[u];
        for (int i = 0; i < P->n; i++)
            for (int s = 0; s < P->nbc; s++) bb[P->nbc * i + s] = P->bnd[((size_t)ax * P->n + i) * P->nbc + s];
        kkt_solve(P, C, eta, bb, xib_new + (size_t)ax * N);
    }
    free(hs);
    free(bb);
}

/* ------------------------------------------------------------ exported API */
static void fill_prob(prob_t *P, int nd, int nxi, double rho, int n, int nobs, int H, int dyn,
                      double a, double b, const double *pmin, const double *pmax, const double *obs_c,
                      const double *obs_ab, const double *bnd, const double *xi, int ws_hess, int cost,
                      double dt, int nbc)
{
    P->nd = nd; P->nxi = nxi; P->rho = rho; P->n = n; P->nobs = nobs; P->H = H; P->dyn = dyn;
    P->a = a; P->b = b; P->pmin = pmin; P->pmax = pmax; P->obs_c = obs_c; P->obs_ab = obs_ab;
    P->bnd = bnd; P->xi = xi; P->ws_hess = ws_hess; P->cost = cost; P->dt = dt; P->nbc = nbc;
}

static int check_prob(const prob_t *P)
{
    if (P->nd < 2 || P->nd > 3 || P->nxi < 2 || P->n < 1 || P->nobs < 0 || P->H < 2) return -1;
    if (!(P->rho > 0.0) || !(P->a > 0.0) || !(P->b > 0.0)) return -1;
    if (P->cost != 0 && (P->cost != 1 || !P->ws_hess || P->nxi < 3 || !(P->dt > 0.0))) return -1;
    if (P->nbc != 2 && (P->nbc != 3 || P->nxi < 4 || !(P->dt > 0.0))) return -1;
    return 0;
}

/* Explicit pieces of the KKT system for one axis (pins only):
   Hm = I + rho F'F (+ rho G'G)  (N x N), Peta (N x N) and Pb (N x nbc n) with
   argmin_{Ax=b} 1/2 x'Hx - eta'x = Peta eta + Pb b. */
int sfo_kkt(int nd, int nxi, double rho, int n, int nobs, int H, int ws_hess, int cost, double dt, int nbc,
            double *Hm, double *Peta, double *Pb)
{
    prob_t P;
    double zeros[3] = {0, 0, 0};
    fill_prob(&P, nd, nxi, rho, n, nobs, H, 0, 1.0, 1.0, zeros, zeros, NULL, NULL, NULL, NULL, ws_hess, cost, dt,
              nbc);
    if (check_prob(&P)) return -1;
    ctx_t C;
    int rc = ctx_init(&P, &C);
    if (rc) return rc;
    int N = C.N, m = nbc * n;
    if (Hm) {
        /* reassemble H = L L^T */
        for (int u = 0; u < N; u++)
            for (int v = 0; v < N; v++) {
                double s = 0.0;
                for (int k = 0; k < N; k++) s += C.L[u * N + k] * C.L[v * N + k];
                Hm[u * N + v] = s;
            }
    }
    double *col = malloc(sizeof(double) * N);
    double *bb = calloc(m, sizeof(double));
    double *x = malloc(sizeof(double) * N);
    if (Peta)
        for (int q = 0; q < N; q++) {
            memset(col, 0, sizeof(double) * N);
            col[q] = 1.0;
            kkt_solve(&P, &C, col, bb, x);
            for (int u = 0; u < N; u++) Peta[u * N + q] = x[u];
        }
    if (Pb)
        for (int q = 0; q < m; q++) {
            memset(col, 0, sizeof(double) * N);
            bb[q] = 1.0;
            kkt_solve(&P, &C, col, bb, x);
            bb[q] = 0.0;
            for (int u = 0; u < N; u++) Pb[u * m + q] = x[u];
        }
    free(col); free(bb); free(x);
    ctx_free(&C);
    return 0;
}

/* Residuals of xi_bar (reading R8): out[0] = ||r_p||_2, out[1] = max residual (m),
   out[2] = kink margin.  g (optional, nd x N) receives F'r_1 + G'r_2. */
int sfo_residual(int nd, int nxi, double rho, int n, int nobs, int H, int dyn, double a, double b,
                 const double *pmin, const double *pmax, const double *obs_c, const double *obs_ab,
                 const double *xib, double *out, double *g)
{
    prob_t P;
    fill_prob(&P, nd, nxi, rho, n, nobs, H, dyn, a, b, pmin, pmax, obs_c, obs_ab, NULL, NULL, 1, 0, 0.0, 2);
    if (check_prob(&P)) return -1;
    ctx_t C;
    memset(&C, 0, sizeof(C));
    /* the residual needs only the basis and the row structure, not the factorisation */
    C.N = n * nxi;
    C.npair = n * (n - 1) / 2;
    C.rows_pair = C.npair * H;
    C.rows_obs = n * nobs * H;
    C.rows_F = C.rows_pair + C.rows_obs;
    C.rows_G = 2 * n * H;
    C.W = malloc(sizeof(double) * H * nxi);
    C.pi = malloc(sizeof(int) * (C.npair + 1));
    C.pj = malloc(sizeof(int) * (C.npair + 1));
    sfo_basis(H, nxi, C.W);
    int p = 0;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) { C.pi[p] = i; C.pj[p] = j; p++; }
    buf_t B;
    if (buf_init(&P, &C, &B)) { ctx_free(&C); return -2; }
    double st[3];
    evaluate(&P, &C, xib, &B, st);
    out[0] = sqrt(st[0]);
    out[1] = st[1];
    out[2] = st[2];
    if (g) {
        for (int ax = 0; ax < nd; ax++) {
            double *ga = g + (size_t)ax * C.N;
            memset(ga, 0, sizeof(double) * C.N);
            FT_apply(&P, &C, B.r1 + (size_t)ax * C.rows_F, ga);
            GT_apply(&P, &C, B.r2 + (size_t)ax * C.rows_G, ga);
        }
    }
    buf_free(&B);
    ctx_free(&C);
    return 0;
}

/* Runs `iters` applications of T from (xi0, lam0) (NULL: xi0 = candidate, lam0 = 0).
   hist (optional): iters x SFO_NHIST, row l = (||r_p||, max residual, kink margin) of the
   l-th iterate and ||z^{l+1} - z^l||.
   traj (optional): (iters+1) x 2 x nd x N, the iterates (xi_bar, lambda) including z^0. */
int sfo_solve(int nd, int nxi, double rho, int n, int nobs, int H, int dyn, double a, double b,
              const double *pmin, const double *pmax, const double *obs_c, const double *obs_ab,
              const double *bnd, const double *xi, const double *xi0, const double *lam0,
              int iters, int ws_hess, int cost, double dt, int nbc, double *xi_out, double *lam_out,
              double *hist, double *traj)
{
    prob_t P;
    fill_prob(&P, nd, nxi, rho, n, nobs, H, dyn, a, b, pmin, pmax, obs_c, obs_ab, bnd, xi, ws_hess, cost, dt, nbc);
    if (check_prob(&P) || iters < 0) return -1;
    ctx_t C;
    int rc = ctx_init(&P, &C);
    if (rc) return rc;
    buf_t B;
    if (buf_init(&P, &C, &B)) { ctx_free(&C); return -2; }
    size_t NN = (size_t)nd * C.N;
    double *x = malloc(sizeof(double) * NN), *l = malloc(sizeof(double) * NN);
    double *xn = malloc(sizeof(double) * NN), *ln = malloc(sizeof(double) * NN);
    memcpy(x, xi0 ? xi0 : xi, sizeof(double) * NN);
    if (lam0) memcpy(l, lam0, sizeof(double) * NN); else memset(l, 0, sizeof(double) * NN);
    if (traj) { memcpy(traj, x, sizeof(double) * NN); memcpy(traj + NN, l, sizeof(double) * NN); }
    for (int it = 0; it < iters; it++) {
        double st[3];
        T_apply(&P, &C, x, l, xn, ln, &B, st);
        double fp = 0.0;
        for (size_t u = 0; u < NN; u++) fp += (xn[u] - x[u]) * (xn[u] - x[u]) + (ln[u] - l[u]) * (ln[u] - l[u]);
        if (hist) {
            hist[it * SFO_NHIST + 0] = sqrt(st[0]);
            hist[it * SFO_NHIST + 1] = st[1];
            hist[it * SFO_NHIST + 2] = sqrt(fp);
            hist[it * SFO_NHIST + 3] = st[2];
        }
        double *t;
        t = x; x = xn; xn = t;
        t = l; l = ln; ln = t;
        if (traj) {
            memcpy(traj + (size_t)(it + 1) * 2 * NN, x, sizeof(double) * NN);
            memcpy(traj + (size_t)(it + 1) * 2 * NN + NN, l, sizeof(double) * NN);
        }
    }
    memcpy(xi_out, x, sizeof(double) * NN);
    if (lam_out) memcpy(lam_out, l, sizeof(double) * NN);
    free(x); free(l); free(xn); free(ln);
    buf_free(&B);
    ctx_free(&C);
    return 0;
}

/* Reverse mode through `iters` applications of T (hand-written adjoint of each step,
   conventions R9).  Seeds: g_xi_out, g_lam_out (nd x N, either may be NULL); g_rp2, the
   weight of ||r_p(xi_out)||^2 in the loss; g_fp, the weight of the self-supervised
   fixed-point term sum_{l<iters} ||z^{l+1} - z^l||^2, z = (xi_bar, lambda) (reading R15).
   Outputs (nd x N each, any may be NULL): gradients with respect to the candidate xi,
   the initial xi_bar and the initial lambda.  The candidate also enters through xi0 when
   xi0 is NULL; that path is added to g_xi. */
int sfo_solve_backward(int nd, int nxi, double rho, int n, int nobs, int H, int dyn, double a, double b,
                       const double *pmin, const double *pmax, const double *obs_c, const double *obs_ab,
                       const double *bnd, const double *xi, const double *xi0, const double *lam0,
                       int iters, int ws_hess, int cost, double dt, int nbc, const double *g_xi_out,
                       const double *g_lam_out, double g_rp2, double g_fp, double *g_xi, double *g_xi0,
                       double *g_lam0)
{
    prob_t P;
    fill_prob(&P, nd, nxi, rho, n, nobs, H, dyn, a, b, pmin, pmax, obs_c, obs_ab, bnd, xi, ws_hess, cost, dt, nbc);
    if (check_prob(&P) || iters < 0) return -1;
    ctx_t C;
    int rc = ctx_init(&P, &C);
    if (rc) return rc;
    buf_t B;
    if (buf_init(&P, &C, &B)) { ctx_free(&C); return -2; }
    int N = C.N, RF = C.rows_F, RG = C.rows_G;
    size_t NN = (size_t)nd * N;
    /* forward pass, keeping every iterate */
    double *X = malloc(sizeof(double) * NN * (iters + 1));
    double *Lm = malloc(sizeof(double) * NN * (iters + 1));
    memcpy(X, xi0 ? xi0 : xi, sizeof(double) * NN);
    if (lam0) memcpy(Lm, lam0, sizeof(double) * NN); else memset(Lm, 0, sizeof(double) * NN);
    for (int it = 0; it < iters; it++) {
        double st[3];
        T_apply(&P, &C, X + NN * it, Lm + NN * it, X + NN * (it + 1), Lm + NN * (it + 1), &B, st);
    }
    double *xb = calloc(NN, sizeof(double)), *lb = calloc(NN, sizeof(double));
    double *gx = calloc(NN, sizeof(double));
    if (g_xi_out) memcpy(xb, g_xi_out, sizeof(double) * NN);
    if (g_lam_out) memcpy(lb, g_lam_out, sizeof(double) * NN);
    double *yb = malloc(sizeof(double) * RF * nd), *eb = malloc(sizeof(double) * RF * nd);
    double *qb = malloc(sizeof(double) * RG * nd), *hsb = malloc(sizeof(double) * RG * nd);
    double *tmp = malloc(sizeof(double) * N), *etab = malloc(sizeof(double) * NN), *lt = malloc(sizeof(double) * NN);
    double J[9];

    /* d/d xi_out of g_rp2 * ||r_p(xi_out)||^2, by the chain rule through r_1 = y - e(y),
       r_2 = q - h + max(0, h - q) */
    if (g_rp2 != 0.0) {
        double st[3];
        evaluate(&P, &C, X + NN * iters, &B, st);
        for (int r = 0; r < RF; r++) {
            int bi, bj, k, m;
            F_row(&P, &C, r, &bi, &bj, &k, &m);
            const double *po = m >= 0 ? obs_at(&P, m, k) : NULL;
            double D[3], ev[3], rb[3];
            for (int ax = 0; ax < nd; ax++) {
                D[ax] = B.y[(size_t)ax * RF + r] - (po ? po[ax] : 0.0);
                rb[ax] = 2.0 * g_rp2 * B.r1[(size_t)ax * RF + r];
            }
            estep(nd, D, m >= 0 ? P.obs_ab[2 * m] : a, m >= 0 ? P.obs_ab[2 * m + 1] : b, ev, J, NULL);
            for (int q = 0; q < nd; q++) {
                double s = rb[q];
                for (int rr = 0; rr < nd; rr++) s -= J[rr * nd + q] * rb[rr];
                yb[(size_t)q * RF + r] = s;
            }
        }
        for (int ax = 0; ax < nd; ax++) {
            for (int gq = 0; gq < RG; gq++) {
                size_t o = (size_t)ax * RG + gq;
                double act = (h_of(&P, ax, gq) - B.q[o]) > 0.0 ? 1.0 : 0.0;
                qb[o] = 2.0 * g_rp2 * B.r2[o] * (1.0 - act);
            }
            FT_apply(&P, &C, yb + (size_t)ax * RF, xb + (size_t)ax * N);
            GT_apply(&P, &C, qb + (size_t)ax * RG, xb + (size_t)ax * N);
        }
    }

    for (int it = iters - 1; it >= 0; it--) {
        double st[3];
        /* the fixed-point term's share of z^{it+1}: d/dz^{it+1} of g_fp ||z^{it+1} - z^it||^2 */
        if (g_fp != 0.0)
            for (size_t u = 0; u < NN; u++) {
                xb[u] += 2.0 * g_fp * (X[NN * (it + 1) + u] - X[NN * it + u]);
                lb[u] += 2.0 * g_fp * (Lm[NN * (it + 1) + u] - Lm[NN * it + u]);
            }
        evaluate(&P, &C, X + NN * it, &B, st); /* recompute y, e, q, s of iterate it */
        for (int ax = 0; ax < nd; ax++) {
            /* eta_bar = Peta^T xi_bar'_bar (Peta symmetric: one KKT solve with b = 0) */
            kkt_solve(&P, &C, xb + (size_t)ax * N, NULL, etab + (size_t)ax * N);
            for (int u = 0; u < N; u++) {
                if (P.cost == 0) gx[(size_t)ax * N + u] += etab[(size_t)ax * N + u];   /* d eta / d xi = I */
                lt[(size_t)ax * N + u] = lb[(size_t)ax * N + u] + etab[(size_t)ax * N + u];
            }
            /* e_bar = rho F eta_bar - r1_bar, r1_bar = -rho F lt;  y_bar = r1_bar */
            double *ybx = yb + (size_t)ax * RF, *ebx = eb + (size_t)ax * RF;
            F_apply(&P, &C, etab + (size_t)ax * N, ebx);
            F_apply(&P, &C, lt + (size_t)ax * N, ybx);
            for (int r = 0; r < RF; r++) {
                double r1b = -rho * ybx[r];
                ebx[r] = rho * ebx[r] - r1b;
                ybx[r] = r1b;
            }
            /* (h - s)_bar = rho G eta_bar (R6), r2_bar = -rho G lt, q_bar = r2_bar,
               s_bar = r2_bar - (h - s)_bar, q_bar -= s_bar [h - q > 0] */
            double *qbx = qb + (size_t)ax * RG, *hsbx = hsb + (size_t)ax * RG;
            G_apply(&P, &C, etab + (size_t)ax * N, hsbx);
            G_apply(&P, &C, lt + (size_t)ax * N, qbx);
            for (int gq = 0; gq < RG; gq++) {
                size_t o = (size_t)ax * RG + gq;
                double hs_b = ws_hess ? rho * hsbx[gq] : 0.0;
                double r2b = -rho * qbx[gq];
                double sb = r2b - hs_b;
                double act = (h_of(&P, ax, gq) - B.q[o]) > 0.0 ? 1.0 : 0.0;
                qbx[gq] = r2b - sb * act;
            }
            memcpy(lb + (size_t)ax * N, lt + (size_t)ax * N, sizeof(double) * N);
        }
        /* y_bar += J_e^T e_bar, row by row */
        for (int r = 0; r < RF; r++) {
            int bi, bj, k, m;
            F_row(&P, &C, r, &bi, &bj, &k, &m);
            const double *po = m >= 0 ? obs_at(&P, m, k) : NULL;
            double D[3], ev[3];
            for (int ax = 0; ax < nd; ax++) D[ax] = B.y[(size_t)ax * RF + r] - (po ? po[ax] : 0.0);
            estep(nd, D, m >= 0 ? P.obs_ab[2 * m] : a, m >= 0 ? P.obs_ab[2 * m + 1] : b, ev, J, NULL);
            for (int q = 0; q < nd; q++) {
                double s = 0.0;
                for (int rr = 0; rr < nd; rr++) s += J[rr * nd + q] * eb[(size_t)rr * RF + r];
                yb[(size_t)q * RF + r] += s;
            }
        }
        /* xi_bar_bar = F^T y_bar + G^T q_bar */
        for (int ax = 0; ax < nd; ax++) {
            memset(xb + (size_t)ax * N, 0, sizeof(double) * N);
            FT_apply(&P, &C, yb + (size_t)ax * RF, xb + (size_t)ax * N);
            GT_apply(&P, &C, qb + (size_t)ax * RG, xb + (size_t)ax * N);
        }
        /* and its share of z^it */
        if (g_fp != 0.0)
            for (size_t u = 0; u < NN; u++) {
                xb[u] -= 2.0 * g_fp * (X[NN * (it + 1) + u] - X[NN * it + u]);
                lb[u] -= 2.0 * g_fp * (Lm[NN * (it + 1) + u] - Lm[NN * it + u]);
            }
    }
    if (g_xi) {
        memcpy(g_xi, gx, sizeof(double) * NN);
        if (!xi0) for (size_t u = 0; u < NN; u++) g_xi[u] += xb[u];
    }
    if (g_xi0) memcpy(g_xi0, xb, sizeof(double) * NN);
    if (g_lam0) memcpy(g_lam0, lb, sizeof(double) * NN);
    free(X); free(Lm); free(xb); free(lb); free(gx); free(yb); free(eb); free(qb); free(hsb);
    free(tmp); free(etab); free(lt);
    buf_free(&B);
    ctx_free(&C);
    return 0;
}

/* Batch of independent instances (packed arrays, per-instance offsets), OpenMP over
   instances.  Offsets are in doubles.  shp[i] = (n, nobs, H, dyn); ab[i] = (a, b);
   box[i] = (pmin[3], pmax[3]).  Returns the first non-zero status, or 0. */
int sfo_solve_batch(int B, int nd, int nxi, double rho, const int *shp, const double *ab,
                    const double *box, const double *obs_c, const long long *off_obs,
                    const double *obs_ab, const long long *off_oab, const double *bnd,
                    const long long *off_bnd, const double *xi, const long long *off_xi,
                    int iters, int ws_hess, int cost, double dt, int nbc, double *xi_out, double *lam_out,
                    double *resid)
{
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < B; i++) {
        const int *s = shp + 4 * i;
        int rc = sfo_solve(nd, nxi, rho, s[0], s[1], s[2], s[3], ab[2 * i], ab[2 * i + 1],
                           box + 6 * i, box + 6 * i + 3, obs_c + off_obs[i], obs_ab + off_oab[i],
                           bnd + off_bnd[i], xi + off_xi[i], NULL, NULL, iters, ws_hess, cost, dt, nbc,
                           xi_out + off_xi[i], lam_out ? lam_out + off_xi[i] : NULL, NULL, NULL);
        if (rc == 0 && resid) {
            double out[3];
            rc = sfo_residual(nd, nxi, rho, s[0], s[1], s[2], s[3], ab[2 * i], ab[2 * i + 1],
                              box + 6 * i, box + 6 * i + 3, obs_c + off_obs[i], obs_ab + off_oab[i],
                              xi_out + off_xi[i], out, NULL);
            resid[2 * i] = out[0];
            resid[2 * i + 1] = out[1];
        }
        if (rc) {
#pragma omp critical
            if (!status) status = rc;
        }
    }
    return status;
}
