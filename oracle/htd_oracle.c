/*
 * htd_oracle.c -- plain, slow, FP64 CPU oracle for the time-domain Helmholtz
 * preconditioner of C. C. Stolk, "A time-domain preconditioner for the
 * Helmholtz equation" (arXiv 2006.16861).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists so that the CUDA path can be
 * checked against something obviously correct.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant with the CUDA library, and the CUDA library
 * must never call it.
 *
 * Everything is double precision, IEEE round-to-nearest, compiled without
 * fast-math.  Loops follow the paper's definitions in the paper's order; no
 * blocking, fusion or reordering beyond that.
 *
 * Contents (paper passages in brackets):
 *   ora_tables          Hamming-distance cell kernels f~_s = S~_s - (hk)^2 M~_s
 *                       [App. A cell form; Sec. 3.1 5-point example].  The
 *                       paper's optimized f_s are not printed in the paper;
 *                       the stencil "Q1MIX" is the stated stand-in (textbook Q1
 *                       stiffness, half consistent plus half lumped Q1 mass).
 *   ora_tables_family   the two-parameter family between FD5 and Q1MIX
 *                       (stiffness and mass weights a, gamma).
 *   ora_setup           omega = sqrt(-lambda_min(Re H)) via the per-cell bound
 *                       (App. A), lambda_max bound (Sec. 3.2, generalised to the
 *                       maximum of the constant-coefficient symbol), the CFL
 *                       rule [Eq. define_Deltat_ImH_diagonal], n_P a multiple of
 *                       4 [Sec. 2.3], alpha and beta [Eq. define_alpha_beta].
 *   ora_apply_reH /
 *   ora_apply_H         Re H by the cell loop of App. A; Im H diagonal,
 *                       (Im H)_ii = omega_phys R_i [Eq. damped_Helmholtz_equation].
 *   ora_assemble_H      the same matrix as triplets, for tiny grids.
 *   ora_window          sine-squared window with parameter rho [Sec. 2.3].
 *   ora_acd_step        one step of I_acd [Def. of I_acd, Eq. acd_integrator,
 *                       Eq. K_L_frequency_adapted_central_differences].
 *   ora_setup_abd /
 *   ora_abd_step        parameters [Sec. 6.1] and one step of I_abd [Def. of
 *                       I_abd, Eq. K_L_frequency_adapted_backward_differences],
 *                       explicit also for non-diagonal damping (damping per
 *                       cell with the cell mass: ORA_DAMP_CELL).
 *   ora_precond         Table 1 (TimeDomainPreconditioner, real fields) and the
 *                       exact operator S_T^acd [Def. approx_solver] as a complex
 *                       recurrence.
 *   ora_precond_project the windowed e^{-i omega t} projection: the real-field
 *                       run of Table 1, read out by projecting its last whole
 *                       periods of states onto e^{-i omega t} (not in the
 *                       paper; it reads U off the same time-harmonic ansatz
 *                       u(t) = Re(U e^{i omega t}) that Table 1 samples).
 *   ora_project_states  that projection for given states (pinned directly).
 *   ora_grad            receiver misfit 0.5 sum_s |P U_s - d_s|^2 of exact
 *                       solutions and its gradient with respect to c^-2 per cell
 *                       and R per node, by one adjoint solve per source (H is
 *                       complex symmetric; not in the paper).
 *   ora_apply_imH       Im H alone (diagonal, or the cell-mass form).
 *   ora_grad_td         misfit of the preconditioner's own approximate solution
 *                       and its gradient through the recurrence (discrete
 *                       adjoint run backwards in time; not in the paper).
 *   ora_direct_solve    banded LU with partial pivoting (exact H^{-1} F).
 *   ora_gmres           restarted GMRES, left-preconditioned [Sec. 2.4] or
 *                       flexible right-preconditioned (FGMRES), modified
 *                       Gram-Schmidt and Givens rotations.
 *
 * Grid: n_a unknown nodes per axis at x_i = i h, a zero ghost ring at i = -1
 * and i = n_a.  Nodes are stored row-major, last axis fastest.  Cells carry
 * the index of their lower corner a = -1..n_a-1 and are stored at a+1, so the
 * cell array has prod(n_a + 1) entries.  Complex vectors are interleaved
 * (re, im) = C99 double complex.
 *
 * Parity unpinned: the paper's own optimized f_s coefficients (not printed in
 * the paper).  Everything else here is pinned by tests.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORA_PI 3.14159265358979323846

enum { ORA_Q1MIX = 0, ORA_FD5 = 1, ORA_FAMILY = 2 };
enum { ORA_MODE_TABLE1 = 0, ORA_MODE_EXACT = 1 };
enum { ORA_P_IDENTITY = 0, ORA_P_TABLE1 = 1, ORA_P_EXACT = 2, ORA_P_DIRECT = 3 };
enum { ORA_FGMRES = 0, ORA_LEFT_GMRES = 1 };
enum { ORA_DAMP_NODE = 0, ORA_DAMP_CELL = 1 };
enum { ORA_ACD = 0, ORA_ABD = 1 };

typedef struct {
    int ndim;            /* 2 or 3 */
    long long n[3];      /* unknown nodes per axis (n[2] ignored for ndim 2) */
    double h;            /* grid spacing */
    int stencil;         /* ORA_Q1MIX, ORA_FD5 or ORA_FAMILY */
    const double *c_cell;  /* wave speed per cell, prod(n_a + 1) */
    const double *R_node;  /* damping per node, prod(n_a), >= 0 */
    double omega_phys;   /* physical angular frequency */
    int damping;         /* ORA_DAMP_NODE: (Im H)_ii = omega_phys R_i (diagonal);
                            ORA_DAMP_CELL: Im H = omega_phys sum over cells of
                            R_cell times the cell mass M (non-diagonal), R_cell
                            the mean of R over the cell's grid corners */
    double stencil_a;    /* ORA_FAMILY: weight of the consistent Q1 mass */
    double stencil_gamma;  /* ORA_FAMILY: weight of the Q1 element stiffness */
} ora_problem;

typedef struct {
    double k_min, k_max;        /* min / max of omega_phys / c over cells */
    double omega;               /* computational omega = k_max */
    double lam_max_reH;         /* upper bound for lambda_max(Re H) */
    double lam_max_A;           /* lambda_max(Re H) + omega^2 */
    int nP;                     /* time steps per period */
    double dt, alpha, beta;
    int T;                      /* periods */
    double rho;                 /* window parameter actually used */
    long long nsteps;           /* T * nP */
    int integrator;             /* ORA_ACD (Def. of I_acd) or ORA_ABD (Def. of I_abd) */
    double lam_max_imH;         /* upper bound for lambda_max(Im H) */
} ora_params;

typedef struct {
    int iterations;             /* Arnoldi steps taken */
    int restarts;               /* cycles started */
    int precond_applies;
    int converged;
    double rel_res_true;        /* ||F - H U|| / ||F|| at exit */
    double rel_res_est;         /* last Arnoldi estimate */
    int hist_len;
    double hist[4096];          /* estimate after every Arnoldi step */
} ora_info;

/* ------------------------------------------------------------------------- */
/* grid helpers                                                               */
/* ------------------------------------------------------------------------- */

static long long n_nodes(const ora_problem *p)
{
    long long N = 1;
    for (int a = 0; a < p->ndim; ++a) N *= p->n[a];
    return N;
}

static long long n_cells(const ora_problem *p)
{
    long long N = 1;
    for (int a = 0; a < p->ndim; ++a) N *= p->n[a] + 1;
    return N;
}

/* linear node index of multi-index i (row-major, last axis fastest) */
static long long node_lin(const ora_problem *p, const long long *i)
{
    long long l = 0;
    for (int a = 0; a < p->ndim; ++a) l = l * p->n[a] + i[a];
    return l;
}

/* linear cell index of the cell whose lower corner is node a (a_k >= -1) */
static long long cell_lin(const ora_problem *p, const long long *a)
{
    long long l = 0;
    for (int k = 0; k < p->ndim; ++k) l = l * (p->n[k] + 1) + (a[k] + 1);
    return l;
}

static int popcount_small(unsigned x)
{
    int c = 0;
    while (x) { c += (int)(x & 1u); x >>= 1; }
    return c;
}

/* ------------------------------------------------------------------------- */
/* stencil tables                                                             */
/* ------------------------------------------------------------------------- */

/*
 * Per-cell kernel of the bilinear form of App. A: for two corners beta, gamma
 * of a cell with Hamming distance s = Delta(beta, gamma),
 *     h^2 * H_cell entry = f~_s(hk/2pi) = S[s] - (h k_cell)^2 * M[s].
 * (Scaled by h^{-2} when assembled, as the paper's coefficients h^{-2} f_s.)
 *
 * Q1MIX, d = 2: S = Q1 element stiffness (2/3, -1/6, -1/3);
 *   consistent Q1 mass (4, 2, 1)/36, lumped mass 1/4 on the diagonal;
 *   M = (consistent + lumped) / 2 = (13/72, 1/36, 1/72).
 * Q1MIX, d = 3: S = (1/3, 0, -1/12, -1/12);
 *   consistent (8, 4, 2, 1)/216, lumped 1/8; M = half of each.
 * FD5: S = (d w, -w, 0, 0) with w = 2^{1-d} (each grid edge is shared by
 *   2^{d-1} cells), M = lumped 2^{-d}: with constant k it assembles to the
 *   5-point (7-point) operator of Sec. 3.1.
 */
int ora_tables(int ndim, int stencil, double S[4], double M[4])
{
    for (int s = 0; s < 4; ++s) { S[s] = 0.0; M[s] = 0.0; }
    if (ndim != 2 && ndim != 3) return -1;
    if (stencil == ORA_Q1MIX) {
        if (ndim == 2) {
            S[0] = 2.0 / 3.0; S[1] = -1.0 / 6.0; S[2] = -1.0 / 3.0;
            M[0] = 0.5 * (4.0 / 36.0) + 0.5 * 0.25;
            M[1] = 0.5 * (2.0 / 36.0);
            M[2] = 0.5 * (1.0 / 36.0);
        } else {
            S[0] = 1.0 / 3.0; S[1] = 0.0; S[2] = -1.0 / 12.0; S[3] = -1.0 / 12.0;
            M[0] = 0.5 * (8.0 / 216.0) + 0.5 * 0.125;
            M[1] = 0.5 * (4.0 / 216.0);
            M[2] = 0.5 * (2.0 / 216.0);
            M[3] = 0.5 * (1.0 / 216.0);
        }
        return 0;
    }
    if (stencil == ORA_FD5) {
        double w = (ndim == 2) ? 0.5 : 0.25;
        S[0] = ndim * w; S[1] = -w;
        M[0] = (ndim == 2) ? 0.25 : 0.125;
        return 0;
    }
    return -1;
}

/*
 * FAMILY(a, gamma): the cell stiffness gamma S(Q1) + (1 - gamma) S(FD5) and the
 * cell mass a M(consistent Q1) + (1 - a) M(lumped), both per Hamming distance
 * with the tables written out above; a, gamma in [0, 1].  Convex combinations
 * of PSD kernels stay PSD and of masses within [0, 2^-d] stay within it, so
 * App. A's bounds hold for every member.
 */
int ora_tables_family(int ndim, double a, double gamma, double S[4], double M[4])
{
    for (int s = 0; s < 4; ++s) { S[s] = 0.0; M[s] = 0.0; }
    if (ndim != 2 && ndim != 3) return -1;
    if (!(a >= 0.0 && a <= 1.0) || !(gamma >= 0.0 && gamma <= 1.0)) return -1;
    double sq1[4] = {0, 0, 0, 0}, sfd[4] = {0, 0, 0, 0}, mc[4] = {0, 0, 0, 0};
    if (ndim == 2) {
        sq1[0] = 2.0 / 3.0; sq1[1] = -1.0 / 6.0; sq1[2] = -1.0 / 3.0;
        mc[0] = 4.0 / 36.0; mc[1] = 2.0 / 36.0; mc[2] = 1.0 / 36.0;
        sfd[0] = 1.0; sfd[1] = -0.5;
    } else {
        sq1[0] = 1.0 / 3.0; sq1[1] = 0.0; sq1[2] = -1.0 / 12.0; sq1[3] = -1.0 / 12.0;
        mc[0] = 8.0 / 216.0; mc[1] = 4.0 / 216.0; mc[2] = 2.0 / 216.0; mc[3] = 1.0 / 216.0;
        sfd[0] = 0.75; sfd[1] = -0.25;
    }
    double lumped = (ndim == 2) ? 0.25 : 0.125;
    for (int s = 0; s <= ndim; ++s) {
        S[s] = gamma * sq1[s] + (1.0 - gamma) * sfd[s];
        M[s] = a * mc[s] + (1.0 - a) * (s == 0 ? lumped : 0.0);
    }
    return 0;
}

/* the tables of a problem's stencil */
static int problem_tables(const ora_problem *p, double S[4], double M[4])
{
    if (p->stencil == ORA_FAMILY)
        return ora_tables_family(p->ndim, p->stencil_a, p->stencil_gamma, S, M);
    return ora_tables(p->ndim, p->stencil, S, M);
}

/* ------------------------------------------------------------------------- */
/* parameters                                                                 */
/* ------------------------------------------------------------------------- */

/*
 * Sec. 2.2 with the bounds of App. A:
 *   omega = sqrt(-lambda_min(Re H)) -> per-cell bound lambda_min >= -k_max^2,
 *   so omega = k_max.
 *   lambda_max(Re H) <= h^{-2} max over theta in {0, pi}^d of the symbol of the
 *   constant-coefficient operator with k = k_min (the symbol is multilinear in
 *   cos theta_a, so the maximum is at a vertex).
 *   lambda_max(A) = lambda_max(Re H) + omega^2.
 *   n_P = smallest multiple of 4 with sin^2(pi / n_P) < omega^2 / lambda_max(A)
 *   (strict CFL of Eq. define_Deltat_ImH_diagonal with dt = 2 pi / (omega n_P)).
 *   alpha, beta from Eq. define_alpha_beta.
 * Returns 0, or -1 on bad input, -2 if a requested nP is not a multiple of 4
 * or violates the CFL bound.
 */
int ora_setup(const ora_problem *p, int T, double rho, int nP_req, ora_params *out)
{
    if (p->ndim != 2 && p->ndim != 3) return -1;
    if (T <= 0 || rho > 1.0 || p->h <= 0.0 || p->omega_phys <= 0.0) return -1;
    double S[4], M[4];
    if (problem_tables(p, S, M)) return -1;
    long long Nc = n_cells(p);
    double kmin = INFINITY, kmax = 0.0;
    for (long long c = 0; c < Nc; ++c) {
        double k = p->omega_phys / p->c_cell[c];
        if (!(k > 0.0) || !isfinite(k)) return -1;
        if (k < kmin) kmin = k;
        if (k > kmax) kmax = k;
    }
    int d = p->ndim;
    double kap = (p->h * kmin) * (p->h * kmin);
    double best = -INFINITY;
    int nvert = 1 << d;
    for (int v = 0; v < nvert; ++v) {
        /* sum over offsets o in {-1,0,1}^d */
        double sym = 0.0;
        int noff = (d == 2) ? 9 : 27;
        for (int t = 0; t < noff; ++t) {
            int o[3], tt = t, s = 0, sign = 1;
            for (int a = 0; a < d; ++a) { o[a] = tt % 3 - 1; tt /= 3; }
            for (int a = 0; a < d; ++a) {
                if (o[a] != 0) {
                    ++s;
                    if ((v >> a) & 1) sign = -sign;   /* cos(pi * o_a) = -1 */
                }
            }
            double ncell = (double)(1 << (d - s));   /* cells holding both nodes */
            sym += sign * ncell * (S[s] - kap * M[s]);
        }
        if (sym > best) best = sym;
    }
    double omega = kmax;
    double lam_reH = best / (p->h * p->h);
    double lam_A = lam_reH + omega * omega;
    double ratio = omega * omega / lam_A;
    int nP = 0;
    if (nP_req > 0) {
        if (nP_req % 4) return -2;
        double s = sin(ORA_PI / nP_req);
        if (!(s * s < ratio)) return -2;
        nP = nP_req;
    } else {
        for (int q = 4; q < 1 << 20; q += 4) {
            double s = sin(ORA_PI / q);
            if (s * s < ratio) { nP = q; break; }
        }
        if (!nP) return -1;
    }
    double dt = 2.0 * ORA_PI / (omega * nP);
    double x = omega * dt;
    out->k_min = kmin;
    out->k_max = kmax;
    out->omega = omega;
    out->lam_max_reH = lam_reH;
    out->lam_max_A = lam_A;
    out->nP = nP;
    out->dt = dt;
    out->alpha = x * x / (4.0 * sin(0.5 * x) * sin(0.5 * x));
    out->beta = x / sin(x);
    out->T = T;
    /* rho = 0 in the paper's experiments meant a ramp over one period (Sec. 5.1) */
    out->rho = (rho <= 0.0) ? 1.0 / T : rho;
    out->nsteps = (long long)T * nP;
    out->integrator = ORA_ACD;
    out->lam_max_imH = 0.0;
    for (long long i = 0; i < n_nodes(p); ++i)
        if (p->omega_phys * p->R_node[i] > out->lam_max_imH) out->lam_max_imH = p->omega_phys * p->R_node[i];
    return 0;
}

/*
 * Parameters of the frequency-adapted backward-differences scheme (Sec. 6.1,
 * Def. of I_abd).  With theta = omega dt = 2 pi / n_P:
 *   omega^2 = -lambda_min(Re H) + (beta / theta)(1 - cos theta) lambda_max(Im H)
 * (K positive semidefinite; -lambda_min(Re H) <= k_max^2 by the App. A bound,
 * lambda_max(Im H) <= omega_phys max R), and n_P the smallest multiple of 4 with
 *   (theta^2 / alpha)(lambda_max(Re H) / omega^2 + 1)
 *     + (beta / alpha)(1 + cos theta) lambda_max(Im H) / omega^2 < 4
 * (4 I - K - 2 L positive definite).  alpha, beta as for I_acd.
 */
static int abd_ok(double theta, double lam_reH, double lam_imH, double kmax2, double *omega2)
{
    double a = theta * theta / (4.0 * sin(0.5 * theta) * sin(0.5 * theta));
    double b = theta / sin(theta);
    double w2 = kmax2 + b / theta * (1.0 - cos(theta)) * lam_imH;
    *omega2 = w2;
    double lhs = theta * theta / a * (lam_reH / w2 + 1.0) + b / a * (1.0 + cos(theta)) * lam_imH / w2;
    return lhs < 4.0;
}

int ora_setup_abd(const ora_problem *p, int T, double rho, int nP_req, ora_params *out)
{
    ora_params q;
    int rc = ora_setup(p, T, rho, 0, &q);    /* k range, lambda bounds, window */
    if (rc) return rc;
    double kmax2 = q.k_max * q.k_max, w2 = 0.0;
    int nP = 0;
    if (nP_req > 0) {
        if (nP_req % 4) return -2;
        if (!abd_ok(2.0 * ORA_PI / nP_req, q.lam_max_reH, q.lam_max_imH, kmax2, &w2)) return -2;
        nP = nP_req;
    } else {
        for (int c = 4; c < 1 << 20; c += 4)
            if (abd_ok(2.0 * ORA_PI / c, q.lam_max_reH, q.lam_max_imH, kmax2, &w2)) { nP = c; break; }
        if (!nP) return -1;
    }
    double theta = 2.0 * ORA_PI / nP;
    q.omega = sqrt(w2);
    q.lam_max_A = q.lam_max_reH + w2;
    q.nP = nP;
    q.dt = theta / q.omega;
    q.alpha = theta * theta / (4.0 * sin(0.5 * theta) * sin(0.5 * theta));
    q.beta = theta / sin(theta);
    q.nsteps = (long long)T * nP;
    q.integrator = ORA_ABD;
    *out = q;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* the operator H                                                             */
/* ------------------------------------------------------------------------- */

/*
 * out = Re H u for a real field u read with element stride `stride`
 * (1 for a real array, 2 for the real or imaginary part of a complex array);
 * out written with the same stride.  The bilinear form of App. A:
 *   (Re H u)_beta = h^{-2} sum over cells alpha containing beta
 *                   sum over corners gamma of alpha
 *                   f~_{Delta(beta,gamma)}(h k_alpha) u_gamma,
 * with u = 0 on the ghost ring.
 */
void ora_apply_reH(const ora_problem *p, const double *u, long long stride, double *out)
{
    double S[4], M[4];
    problem_tables(p, S, M);
    int d = p->ndim;
    long long N = n_nodes(p);
    for (long long i = 0; i < N; ++i) out[i * stride] = 0.0;
    double ih2 = 1.0 / (p->h * p->h);
    long long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) { lo[a] = -1; hi[a] = p->n[a] - 1; }
    long long a3[3];
    int ncorner = 1 << d;
    for (a3[0] = lo[0]; a3[0] <= hi[0]; ++a3[0])
    for (a3[1] = lo[1]; a3[1] <= hi[1]; ++a3[1])
    for (a3[2] = (d == 3 ? lo[2] : 0); a3[2] <= (d == 3 ? hi[2] : 0); ++a3[2]) {
        double k = p->omega_phys / p->c_cell[cell_lin(p, a3)];
        double kap = (p->h * k) * (p->h * k);
        /* the cell's corners: node index, or -1 for a ghost node (u = 0 there) */
        long long corner[8];
        for (int b = 0; b < ncorner; ++b) {
            long long ib[3];
            int inside = 1;
            for (int t = 0; t < d; ++t) {
                ib[t] = a3[t] + ((b >> (d - 1 - t)) & 1);
                if (ib[t] < 0 || ib[t] >= p->n[t]) inside = 0;
            }
            corner[b] = inside ? node_lin(p, ib) : -1;
        }
        for (int b = 0; b < ncorner; ++b) {
            if (corner[b] < 0) continue;
            double acc = 0.0;
            for (int g = 0; g < ncorner; ++g) {
                if (corner[g] < 0) continue;
                int s = popcount_small((unsigned)(b ^ g));
                acc += (S[s] - kap * M[s]) * u[corner[g] * stride];
            }
            out[corner[b] * stride] += ih2 * acc;
        }
    }
}

/* out = H U = Re H U + i (omega_phys R) U, complex vectors */
/* R of a cell for ORA_DAMP_CELL: the mean of R over the cell's corners inside
 * the grid (every cell has at least one) */
static double cell_R(const ora_problem *p, const long long *a3)
{
    int d = p->ndim;
    double sum = 0.0;
    int cnt = 0;
    for (int b = 0; b < (1 << d); ++b) {
        long long ib[3];
        int inside = 1;
        for (int t = 0; t < d; ++t) {
            ib[t] = a3[t] + ((b >> (d - 1 - t)) & 1);
            if (ib[t] < 0 || ib[t] >= p->n[t]) inside = 0;
        }
        if (inside) { sum += p->R_node[node_lin(p, ib)]; ++cnt; }
    }
    return sum / cnt;
}

/*
 * out = Im H u (real field, element stride `stride`).  ORA_DAMP_NODE:
 * omega_phys R_i u_i.  ORA_DAMP_CELL: the cell loop of App. A with the mass
 * weights only, R_cell in place of kappa:
 *   (Im H u)_beta = omega_phys sum_{cells alpha containing beta}
 *                   R_alpha sum_{corners gamma} M_{Delta(beta,gamma)} u_gamma.
 * The mass row sums are 1, so for constant R both forms agree on constants.
 */
void ora_apply_imH(const ora_problem *p, const double *u, long long stride, double *out)
{
    long long N = n_nodes(p);
    if (p->damping != ORA_DAMP_CELL) {
        for (long long i = 0; i < N; ++i) out[i * stride] = p->omega_phys * p->R_node[i] * u[i * stride];
        return;
    }
    double S[4], M[4];
    problem_tables(p, S, M);
    int d = p->ndim;
    for (long long i = 0; i < N; ++i) out[i * stride] = 0.0;
    long long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) { lo[a] = -1; hi[a] = p->n[a] - 1; }
    long long a3[3];
    int ncorner = 1 << d;
    for (a3[0] = lo[0]; a3[0] <= hi[0]; ++a3[0])
    for (a3[1] = lo[1]; a3[1] <= hi[1]; ++a3[1])
    for (a3[2] = (d == 3 ? lo[2] : 0); a3[2] <= (d == 3 ? hi[2] : 0); ++a3[2]) {
        double r = p->omega_phys * cell_R(p, a3);
        long long corner[8];
        for (int b = 0; b < ncorner; ++b) {
            long long ib[3];
            int inside = 1;
            for (int t = 0; t < d; ++t) {
                ib[t] = a3[t] + ((b >> (d - 1 - t)) & 1);
                if (ib[t] < 0 || ib[t] >= p->n[t]) inside = 0;
            }
            corner[b] = inside ? node_lin(p, ib) : -1;
        }
        for (int b = 0; b < ncorner; ++b) {
            if (corner[b] < 0) continue;
            double acc = 0.0;
            for (int g = 0; g < ncorner; ++g)
                if (corner[g] >= 0) acc += M[popcount_small((unsigned)(b ^ g))] * u[corner[g] * stride];
            out[corner[b] * stride] += r * acc;
        }
    }
}

void ora_apply_H(const ora_problem *p, const cplx *U, cplx *out)
{
    long long N = n_nodes(p);
    const double *Ud = (const double *)U;
    double *Od = (double *)out;
    ora_apply_reH(p, Ud, 2, Od);          /* real parts */
    ora_apply_reH(p, Ud + 1, 2, Od + 1);  /* imaginary parts */
    double *t = malloc(sizeof(double) * 2 * N);   /* interleaved: Im H Re U, Im H Im U */
    ora_apply_imH(p, Ud, 2, t);
    ora_apply_imH(p, Ud + 1, 2, t + 1);
    for (long long i = 0; i < N; ++i) out[i] += -t[2 * i + 1] + I * t[2 * i];
    free(t);
}

/*
 * Triplets of H (tiny grids).  Writes at most `cap` entries (duplicates summed
 * by the caller, e.g. scipy COO -> CSR).  Returns the number of entries that
 * the full matrix needs.
 */
long long ora_assemble_H(const ora_problem *p, long long cap, long long *rows,
                         long long *cols, double *re, double *im)
{
    double S[4], M[4];
    problem_tables(p, S, M);
    int d = p->ndim;
    long long cnt = 0;
    double ih2 = 1.0 / (p->h * p->h);
    long long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) { lo[a] = -1; hi[a] = p->n[a] - 1; }
    long long a3[3];
    int ncorner = 1 << d;
    for (a3[0] = lo[0]; a3[0] <= hi[0]; ++a3[0])
    for (a3[1] = lo[1]; a3[1] <= hi[1]; ++a3[1])
    for (a3[2] = (d == 3 ? lo[2] : 0); a3[2] <= (d == 3 ? hi[2] : 0); ++a3[2]) {
        double k = p->omega_phys / p->c_cell[cell_lin(p, a3)];
        double kap = (p->h * k) * (p->h * k);
        for (int b = 0; b < ncorner; ++b)
        for (int g = 0; g < ncorner; ++g) {
            long long ib[3], ig[3];
            int ok = 1;
            for (int t = 0; t < d; ++t) {
                ib[t] = a3[t] + ((b >> (d - 1 - t)) & 1);
                ig[t] = a3[t] + ((g >> (d - 1 - t)) & 1);
                if (ib[t] < 0 || ib[t] >= p->n[t] || ig[t] < 0 || ig[t] >= p->n[t]) ok = 0;
            }
            if (!ok) continue;
            int s = popcount_small((unsigned)(b ^ g));
            if (cnt < cap) {
                rows[cnt] = node_lin(p, ib);
                cols[cnt] = node_lin(p, ig);
                re[cnt] = ih2 * (S[s] - kap * M[s]);
                im[cnt] = (p->damping == ORA_DAMP_CELL) ? p->omega_phys * cell_R(p, a3) * M[s] : 0.0;
            }
            ++cnt;
        }
    }
    long long N = n_nodes(p);
    if (p->damping == ORA_DAMP_CELL) return cnt;
    for (long long i = 0; i < N; ++i) {
        if (cnt < cap) {
            rows[cnt] = i; cols[cnt] = i; re[cnt] = 0.0;
            im[cnt] = p->omega_phys * p->R_node[i];
        }
        ++cnt;
    }
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* window and one step of I_acd                                               */
/* ------------------------------------------------------------------------- */

/*
 * Sine-squared window of Sec. 2.3, read as an even function:
 *   chi(s) = 1                            for |s| <= 1 - rho,
 *            sin^2(pi (1 - |s|) / (2 rho)) for 1 - rho < |s| < 1,
 *            0                            for |s| >= 1.
 */
double ora_window(double s, double rho)
{
    double a = fabs(s);
    if (a >= 1.0) return 0.0;
    if (a <= 1.0 - rho) return 1.0;
    double v = sin(ORA_PI * (1.0 - a) / (2.0 * rho));
    return v * v;
}

/*
 * One step of frequency-adapted central-differences damped leapfrog
 * (Def. of I_acd):
 *   u_{n+1} = (I + L/2)^{-1} ((2 - K) u_n - (I - L/2) u_{n-1} + g_n),
 *   K = (dt^2/alpha) A,  A = Re H + omega^2 I,
 *   L = (beta dt/alpha) B,  B = omega^{-1} Im H,
 *   g_n = (dt^2/alpha) f_n.
 * Real version; the arrays are read and written with element stride `stride`
 * (so the real and imaginary parts of a complex recurrence can be stepped by
 * the same routine: K and L are real).  `work` holds N doubles.
 */
static void acd_step_real(const ora_problem *p, const ora_params *q,
                          const double *un, const double *unm1, const double *fn,
                          double *unp1, long long stride, double *work)
{
    long long N = n_nodes(p);
    double c = q->dt * q->dt / q->alpha;
    double lc = q->beta * q->dt / q->alpha;
    ora_apply_reH(p, un, stride, work);   /* Re H u_n, same stride */
    for (long long i = 0; i < N; ++i) {
        double Ku = c * (work[i * stride] + q->omega * q->omega * un[i * stride]);
        double B = p->omega_phys * p->R_node[i] / q->omega;
        double L = lc * B;
        double g = c * fn[i * stride];
        unp1[i * stride] = ((2.0 * un[i * stride] - Ku)
                            - (1.0 - 0.5 * L) * unm1[i * stride] + g) / (1.0 + 0.5 * L);
    }
}

/*
 * One step of frequency-adapted backward-differences damped leapfrog
 * (Def. of I_abd), explicit for any symmetric B:
 *   u_{n+1} = (2 - K - L) u_n - (I - L) u_{n-1} + g_n,
 *   K = (dt^2/alpha) A - (dt beta (1 - cos(omega dt)) / alpha) B,
 *   L = (beta dt / alpha) B,  A = Re H + omega^2 I,  B = omega^{-1} Im H,
 *   g_n = (dt^2/alpha) f_n.
 * Real fields with element stride `stride`; `work` holds 3 N stride doubles.
 */
static void abd_step_real(const ora_problem *p, const ora_params *q,
                          const double *un, const double *unm1, const double *fn,
                          double *unp1, long long stride, double *work)
{
    long long N = n_nodes(p);
    double cA = q->dt * q->dt / q->alpha;
    double cBK = q->dt * q->beta * (1.0 - cos(q->omega * q->dt)) / q->alpha / q->omega;
    double cBL = q->beta * q->dt / q->alpha / q->omega;
    double *reH = work, *imHu = work + N * stride, *imHp = work + 2 * N * stride;
    ora_apply_reH(p, un, stride, reH);
    ora_apply_imH(p, un, stride, imHu);
    ora_apply_imH(p, unm1, stride, imHp);
    for (long long i = 0; i < N; ++i) {
        double u = un[i * stride], up = unm1[i * stride];
        double Ku = cA * (reH[i * stride] + q->omega * q->omega * u) - cBK * imHu[i * stride];
        double Lu = cBL * imHu[i * stride], Lup = cBL * imHp[i * stride];
        unp1[i * stride] = 2.0 * u - Ku - Lu - (up - Lup) + cA * fn[i * stride];
    }
}

void ora_abd_step(const ora_problem *p, const ora_params *q, const cplx *un,
                  const cplx *unm1, const cplx *fn, cplx *unp1)
{
    long long N = n_nodes(p);
    double *work = (double *)malloc(sizeof(double) * 6 * N);
    for (int part = 0; part < 2; ++part)
        abd_step_real(p, q, (const double *)un + part, (const double *)unm1 + part,
                      (const double *)fn + part, (double *)unp1 + part, 2, work + part);
    free(work);
}

/* the step of the parameters' integrator */
static void any_step_real(const ora_problem *p, const ora_params *q,
                          const double *un, const double *unm1, const double *fn,
                          double *unp1, long long stride, double *work)
{
    if (q->integrator == ORA_ABD) abd_step_real(p, q, un, unm1, fn, unp1, stride, work);
    else acd_step_real(p, q, un, unm1, fn, unp1, stride, work);
}

/* complex step: real and imaginary parts stepped separately (K, L real) */
void ora_acd_step(const ora_problem *p, const ora_params *q, const cplx *un,
                  const cplx *unm1, const cplx *fn, cplx *unp1)
{
    long long N = n_nodes(p);
    double *work = (double *)malloc(sizeof(double) * 2 * N);
    for (int part = 0; part < 2; ++part)
        acd_step_real(p, q, (const double *)un + part, (const double *)unm1 + part,
                      (const double *)fn + part, (double *)unp1 + part, 2, work + part);
    free(work);
}

/* ------------------------------------------------------------------------- */
/* the preconditioner                                                         */
/* ------------------------------------------------------------------------- */

/*
 * Table 1, TimeDomainPreconditioner(F, K, L, T, n_P), with real fields:
 *   u_{-1} = u_0 = 0
 *   for j = 0 .. T n_P - 1:
 *       u_{j+1} = I_acd(u_j, u_{j-1},
 *                       chi(1 - j/(T n_P)) [cos(2 pi j/n_P) Re F - sin(2 pi j/n_P) Im F])
 *   U = u_{T n_P} + i u_{(T - 1/4) n_P}
 */
static void precond_table1(const ora_problem *p, const ora_params *q, const cplx *F, cplx *U)
{
    long long N = n_nodes(p);
    long long nsteps = q->nsteps;
    long long j_im = nsteps - q->nP / 4;
    double *um1 = calloc(N, sizeof(double));
    double *u0 = calloc(N, sizeof(double));
    double *u1 = calloc(N, sizeof(double));
    double *f = malloc(sizeof(double) * N);
    double *snap = calloc(N, sizeof(double));
    double *work = malloc(sizeof(double) * 3 * N);
    for (long long j = 0; j < nsteps; ++j) {
        double chi = ora_window(1.0 - (double)j / (double)nsteps, q->rho);
        double cs = cos(2.0 * ORA_PI * (double)j / q->nP);
        double sn = sin(2.0 * ORA_PI * (double)j / q->nP);
        for (long long i = 0; i < N; ++i)
            f[i] = chi * (cs * creal(F[i]) - sn * cimag(F[i]));
        any_step_real(p, q, u0, um1, f, u1, 1, work);
        if (j + 1 == j_im) memcpy(snap, u1, sizeof(double) * N);
        double *t = um1; um1 = u0; u0 = u1; u1 = t;
    }
    for (long long i = 0; i < N; ++i) U[i] = u0[i] + I * snap[i];
    free(um1); free(u0); free(u1); free(f); free(snap); free(work);
}

/*
 * S_T^acd F = e^{-i 2 pi T} u_{n_steps} (Def. approx_solver), with the complex
 * recurrence u_{n+1} = I_acd(u_n, u_{n-1}, f_n), u_0 = 0 (and u_{-1} = 0),
 * f_n = chi(1 - n dt / (2 pi T / omega)) e^{i omega n dt} F.
 */
static void precond_exact(const ora_problem *p, const ora_params *q, const cplx *F, cplx *U)
{
    long long N = n_nodes(p);
    long long nsteps = q->nsteps;
    cplx *um1 = calloc(N, sizeof(cplx));
    cplx *u0 = calloc(N, sizeof(cplx));
    cplx *u1 = calloc(N, sizeof(cplx));
    cplx *f = malloc(sizeof(cplx) * N);
    double *work = malloc(sizeof(double) * 6 * N);
    double Ttilde = 2.0 * ORA_PI * q->T / q->omega;
    for (long long n = 0; n < nsteps; ++n) {
        double t = n * q->dt;
        cplx e = cexp(I * q->omega * t);
        double chi = ora_window(1.0 - t / Ttilde, q->rho);
        for (long long i = 0; i < N; ++i) f[i] = chi * e * F[i];
        for (int part = 0; part < 2; ++part)
            any_step_real(p, q, (const double *)u0 + part, (const double *)um1 + part,
                          (const double *)f + part, (double *)u1 + part, 2, work + part);
        cplx *tmp = um1; um1 = u0; u0 = u1; u1 = tmp;
    }
    cplx ph = cexp(-I * 2.0 * ORA_PI * q->T);
    for (long long i = 0; i < N; ++i) U[i] = ph * u0[i];
    free(um1); free(u0); free(u1); free(f); free(work);
}

/*
 * Projection read-out.  The real-field run of Table 1 approaches the
 * time-harmonic state u_j = Re(U e^{i 2 pi j / n_P}) (at j = T n_P the phase
 * is 0, so Re U = u_{T n_P} as in Table 1).  Over whole periods
 * sum_j e^{-i 2 pi j/n_P} Re(U e^{i 2 pi j/n_P}) = (n_acc / 2) U, because
 * sum_j e^{-i 4 pi j/n_P} vanishes for n_P > 2, so
 *   U = (2 / n_acc) sum_{j = j_first}^{j_first + n_acc - 1} e^{-i 2 pi j / n_P} u_j,
 * with n_acc = (periods) n_P equal weights (a rectangular window of whole
 * periods keeps that cancellation exact).
 */
static void project_add(long long N, int nP, long long j, const double *u, cplx *acc)
{
    double th = 2.0 * ORA_PI * (double)(j % nP) / nP;
    cplx e = cos(th) - I * sin(th);
    for (long long i = 0; i < N; ++i) acc[i] += e * u[i];
}

/* states: n_acc consecutive real states u_{j_first} .. u_{j_first + n_acc - 1},
 * N values each; U = (2 / n_acc) sum e^{-i 2 pi j / n_P} u_j */
void ora_project_states(long long N, int nP, long long j_first, long long n_acc,
                        const double *states, cplx *U)
{
    for (long long i = 0; i < N; ++i) U[i] = 0.0;
    for (long long k = 0; k < n_acc; ++k) project_add(N, nP, j_first + k, states + k * N, U);
    for (long long i = 0; i < N; ++i) U[i] *= 2.0 / (double)n_acc;
}

/* Table 1's recurrence, read out by projecting the states u_j of the last
 * `periods` periods (j = T n_P - periods n_P + 1 .. T n_P); 1 <= periods <= T */
int ora_precond_project(const ora_problem *p, const ora_params *q, int periods, const cplx *F,
                        cplx *U)
{
    if (periods < 1 || periods > q->T) return -1;
    if (q->integrator == ORA_ACD && p->damping == ORA_DAMP_CELL) return -1;
    long long N = n_nodes(p);
    long long nsteps = q->nsteps;
    long long n_acc = (long long)periods * q->nP;
    double *um1 = calloc(N, sizeof(double));
    double *u0 = calloc(N, sizeof(double));
    double *u1 = calloc(N, sizeof(double));
    double *f = malloc(sizeof(double) * N);
    double *work = malloc(sizeof(double) * 3 * N);
    for (long long i = 0; i < N; ++i) U[i] = 0.0;
    for (long long j = 0; j < nsteps; ++j) {
        double chi = ora_window(1.0 - (double)j / (double)nsteps, q->rho);
        double cs = cos(2.0 * ORA_PI * (double)j / q->nP);
        double sn = sin(2.0 * ORA_PI * (double)j / q->nP);
        for (long long i = 0; i < N; ++i)
            f[i] = chi * (cs * creal(F[i]) - sn * cimag(F[i]));
        any_step_real(p, q, u0, um1, f, u1, 1, work);
        if (j + 1 > nsteps - n_acc) project_add(N, q->nP, j + 1, u1, U);   /* state u_{j+1} */
        double *t = um1; um1 = u0; u0 = u1; u1 = t;
    }
    for (long long i = 0; i < N; ++i) U[i] *= 2.0 / (double)n_acc;
    free(um1); free(u0); free(u1); free(f); free(work);
    return 0;
}

int ora_precond(const ora_problem *p, const ora_params *q, int mode, const cplx *F, cplx *U)
{
    /* I_acd inverts I + L/2, which is only explicit for diagonal damping */
    if (q->integrator == ORA_ACD && p->damping == ORA_DAMP_CELL) return -1;
    if (mode == ORA_MODE_TABLE1) precond_table1(p, q, F, U);
    else if (mode == ORA_MODE_EXACT) precond_exact(p, q, F, U);
    else return -1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* banded LU with partial pivoting                                            */
/* ------------------------------------------------------------------------- */

typedef struct {
    long long N, kl, ku, W;    /* W = 2 kl + ku + 1 band width stored per row */
    cplx *B;                   /* row i holds columns i-kl .. i+ku+kl */
    long long *piv;
} band_lu;

static cplx *band_at(band_lu *f, long long i, long long j)
{
    return &f->B[i * f->W + (j - i + f->kl)];
}

static void band_free(band_lu *f) { free(f->B); free(f->piv); f->B = 0; f->piv = 0; }

/* assemble H into band storage and factor it; returns 0, or -1 if singular */
static int band_factor(const ora_problem *p, band_lu *f)
{
    long long N = n_nodes(p);
    long long bw = 0, stride = 1;
    for (int a = p->ndim - 1; a >= 0; --a) { bw += stride; stride *= p->n[a]; }
    f->N = N; f->kl = bw; f->ku = bw; f->W = 2 * bw + bw + 1;
    f->B = calloc((size_t)(N * f->W), sizeof(cplx));
    f->piv = malloc(sizeof(long long) * N);
    long long cap = 0;
    {
        long long per = (p->ndim == 2) ? 16 : 64;
        cap = n_cells(p) * per + N;
    }
    long long *rows = malloc(sizeof(long long) * cap), *cols = malloc(sizeof(long long) * cap);
    double *re = malloc(sizeof(double) * cap), *im = malloc(sizeof(double) * cap);
    long long cnt = ora_assemble_H(p, cap, rows, cols, re, im);
    for (long long e = 0; e < cnt; ++e) *band_at(f, rows[e], cols[e]) += re[e] + I * im[e];
    free(rows); free(cols); free(re); free(im);
    for (long long k = 0; k < N; ++k) {
        long long last = k + f->kl < N - 1 ? k + f->kl : N - 1;
        long long pr = k;
        double best = cabs(*band_at(f, k, k));
        for (long long i = k + 1; i <= last; ++i) {
            double v = cabs(*band_at(f, i, k));
            if (v > best) { best = v; pr = i; }
        }
        f->piv[k] = pr;
        if (best == 0.0) return -1;
        long long jend = k + f->ku + f->kl < N - 1 ? k + f->ku + f->kl : N - 1;
        if (pr != k)
            for (long long j = k; j <= jend; ++j) {
                cplx t = *band_at(f, k, j);
                *band_at(f, k, j) = *band_at(f, pr, j);
                *band_at(f, pr, j) = t;
            }
        cplx piv = *band_at(f, k, k);
        for (long long i = k + 1; i <= last; ++i) {
            cplx l = *band_at(f, i, k) / piv;
            *band_at(f, i, k) = l;
            if (l != 0.0)
                for (long long j = k + 1; j <= jend; ++j)
                    *band_at(f, i, j) -= l * *band_at(f, k, j);
        }
    }
    return 0;
}

static void band_solve(band_lu *f, const cplx *b, cplx *x)
{
    long long N = f->N;
    cplx *y = malloc(sizeof(cplx) * N);
    memcpy(y, b, sizeof(cplx) * N);
    for (long long k = 0; k < N; ++k) {
        long long pr = f->piv[k];
        if (pr != k) { cplx t = y[k]; y[k] = y[pr]; y[pr] = t; }
        long long last = k + f->kl < N - 1 ? k + f->kl : N - 1;
        for (long long i = k + 1; i <= last; ++i) y[i] -= *band_at(f, i, k) * y[k];
    }
    for (long long k = N - 1; k >= 0; --k) {
        long long jend = k + f->ku + f->kl < N - 1 ? k + f->ku + f->kl : N - 1;
        cplx s = y[k];
        for (long long j = k + 1; j <= jend; ++j) s -= *band_at(f, k, j) * x[j];
        x[k] = s / *band_at(f, k, k);
    }
    free(y);
}

/* U = H^{-1} F by banded LU (tiny grids only: memory ~ N * 3 * bandwidth) */
int ora_direct_solve(const ora_problem *p, const cplx *F, cplx *U)
{
    band_lu f;
    if (band_factor(p, &f)) { band_free(&f); return -1; }
    band_solve(&f, F, U);
    band_free(&f);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* GMRES                                                                      */
/* ------------------------------------------------------------------------- */

static cplx dotc(long long N, const cplx *x, const cplx *y)  /* sum conj(x) y */
{
    cplx s = 0.0;
    for (long long i = 0; i < N; ++i) s += conj(x[i]) * y[i];
    return s;
}

static double nrm2(long long N, const cplx *x) { return sqrt(creal(dotc(N, x, x))); }

typedef struct {
    const ora_problem *p;
    const ora_params *q;
    int precond;
    band_lu *lu;
    int applies;
} gm_ctx;

static void apply_P(gm_ctx *c, const cplx *x, cplx *y)
{
    long long N = n_nodes(c->p);
    switch (c->precond) {
    case ORA_P_TABLE1: precond_table1(c->p, c->q, x, y); break;
    case ORA_P_EXACT: precond_exact(c->p, c->q, x, y); break;
    case ORA_P_DIRECT: band_solve(c->lu, x, y); break;
    default: memcpy(y, x, sizeof(cplx) * N); break;
    }
    c->applies++;
}

/*
 * Restarted GMRES(m) (Sec. 2.4).
 *   krylov = ORA_LEFT_GMRES: GMRES on P H U = P F (the paper's proposal).
 *   krylov = ORA_FGMRES: flexible right preconditioning, H P V = F with the
 *            preconditioned vectors Z_j = P V_j stored, U = U0 + Z y.
 * Arnoldi by modified Gram-Schmidt, least squares by Givens rotations.
 * Stops when the Arnoldi residual estimate (relative to ||P F|| for left, to
 * ||F|| for flexible) is <= tol and the true relative residual ||F - H U|| / ||F||
 * is <= tol, or after maxit Arnoldi steps.  fixed != 0: no early exit, exactly
 * maxit Arnoldi steps.  U holds the initial guess on entry.
 */
int ora_gmres(const ora_problem *p, const ora_params *q, int krylov, int precond,
              const cplx *F, cplx *U, double tol, int m, int maxit, int fixed, ora_info *info)
{
    long long N = n_nodes(p);
    if (m < 1 || maxit < 0) return -1;
    band_lu lu = {0};
    gm_ctx c = {p, q, precond, &lu, 0};
    if (precond == ORA_P_DIRECT && band_factor(p, &lu)) { band_free(&lu); return -1; }
    cplx *V = malloc(sizeof(cplx) * N * (m + 1));
    cplx *Z = (krylov == ORA_FGMRES) ? malloc(sizeof(cplx) * N * m) : NULL;
    cplx *w = malloc(sizeof(cplx) * N);
    cplx *t = malloc(sizeof(cplx) * N);
    cplx *Hm = malloc(sizeof(cplx) * (m + 1) * m);    /* column-major (m+1) x m */
    cplx *cs = malloc(sizeof(cplx) * m), *g = malloc(sizeof(cplx) * (m + 1));
    double *sn = malloc(sizeof(double) * m);
    cplx *y = malloc(sizeof(cplx) * m);
    memset(info, 0, sizeof(*info));

    double fnorm = nrm2(N, F);
    double bnorm = fnorm;
    cplx *PF = NULL;
    if (krylov == ORA_LEFT_GMRES) {
        PF = malloc(sizeof(cplx) * N);
        apply_P(&c, F, PF);
        bnorm = nrm2(N, PF);
    }
    if (fnorm == 0.0) {
        for (long long i = 0; i < N; ++i) U[i] = 0.0;
        info->converged = 1;
        goto done;
    }
    int its = 0;
    for (;;) {
        /* true residual r = F - H U */
        ora_apply_H(p, U, t);
        for (long long i = 0; i < N; ++i) t[i] = F[i] - t[i];
        double true_rel = nrm2(N, t) / fnorm;
        info->rel_res_true = true_rel;
        if (!fixed && true_rel <= tol) { info->converged = 1; break; }
        if (its >= maxit) break;
        /* Krylov residual: P r (left) or r (flexible) */
        if (krylov == ORA_LEFT_GMRES) apply_P(&c, t, w); else memcpy(w, t, sizeof(cplx) * N);
        double beta = nrm2(N, w);
        if (beta == 0.0) break;
        info->restarts++;
        for (long long i = 0; i < N; ++i) V[i] = w[i] / beta;
        for (int k = 0; k <= m; ++k) g[k] = 0.0;
        g[0] = beta;
        int j = 0;
        while (j < m && its < maxit) {
            cplx *vj = V + (long long)j * N;
            if (krylov == ORA_FGMRES) {
                cplx *zj = Z + (long long)j * N;
                apply_P(&c, vj, zj);
                ora_apply_H(p, zj, w);
            } else {
                ora_apply_H(p, vj, t);
                apply_P(&c, t, w);
            }
            cplx *col = Hm + (long long)j * (m + 1);
            for (int i = 0; i <= j; ++i) {       /* modified Gram-Schmidt */
                cplx *vi = V + (long long)i * N;
                cplx hij = dotc(N, vi, w);
                col[i] = hij;
                for (long long l = 0; l < N; ++l) w[l] -= hij * vi[l];
            }
            double hn = nrm2(N, w);
            col[j + 1] = hn;
            if (hn != 0.0) {
                cplx *vn = V + (long long)(j + 1) * N;
                for (long long l = 0; l < N; ++l) vn[l] = w[l] / hn;
            }
            /* apply the previous rotations to column j */
            for (int i = 0; i < j; ++i) {
                cplx a = col[i], b = col[i + 1];
                col[i] = conj(cs[i]) * a + sn[i] * b;
                col[i + 1] = -sn[i] * a + cs[i] * b;
            }
            /* new rotation [conj(c) s; -s c] with real s, zeroing col[j+1] */
            {
                cplx a = col[j];
                double b = creal(col[j + 1]);
                double r = sqrt(creal(a * conj(a)) + b * b);
                if (r == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
                else { cs[j] = a / r; sn[j] = b / r; }
                col[j] = conj(cs[j]) * a + sn[j] * b;
                col[j + 1] = 0.0;
                cplx gj = g[j];
                g[j] = conj(cs[j]) * gj;
                g[j + 1] = -sn[j] * gj;
            }
            ++its;
            ++j;
            double est = cabs(g[j]) / bnorm;
            info->rel_res_est = est;
            if (info->hist_len < 4096) info->hist[info->hist_len++] = est;
            if (!fixed && est <= tol) break;
            if (hn == 0.0) break;
        }
        /* y = R^{-1} g, U += basis * y */
        for (int i = j - 1; i >= 0; --i) {
            cplx s = g[i];
            for (int k = i + 1; k < j; ++k) s -= Hm[(long long)k * (m + 1) + i] * y[k];
            y[i] = s / Hm[(long long)i * (m + 1) + i];
        }
        for (int k = 0; k < j; ++k) {
            const cplx *bk = (krylov == ORA_FGMRES) ? Z + (long long)k * N : V + (long long)k * N;
            for (long long l = 0; l < N; ++l) U[l] += y[k] * bk[l];
        }
    }
    info->iterations = its;
done:
    info->precond_applies = c.applies;
    free(V); free(Z); free(w); free(t); free(Hm); free(cs); free(g); free(sn); free(y);
    free(PF);
    band_free(&lu);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* receiver misfit and its gradient (adjoint state)                           */
/* ------------------------------------------------------------------------- */

/*
 * J = 1/2 sum_s || P U_s - d_s ||^2 with H U_s = F_s (direct solves), P the
 * sampling at the nodes rec_idx[0..nrec-1].  Gradient with respect to
 * m = c^{-2} per cell and R per node.  With r_s = P^T (P U_s - d_s) and the
 * adjoint field mu_s = H^{-1} conj(r_s) (H is complex symmetric, so this is the
 * conjugate of the solution of H^H lambda = r):
 *   dJ/dm_alpha = omega^2 sum_s Re sum_{beta,gamma in cell alpha}
 *                 mu_{s,beta} M_{Delta(beta,gamma)} U_{s,gamma}
 *   (Re H depends on m through -(h k)^2 M_cell h^{-2} = -omega^2 m M_cell),
 *   dJ/dR_i = omega sum_s Im(mu_{s,i} U_{s,i})   ((Im H)_ii = omega R_i).
 * F: nsrc x N complex, d: nsrc x nrec complex; grad_m: prod(n+1), grad_R: N.
 * Returns 0, or -1 if H is singular.
 */
int ora_grad(const ora_problem *p, int nsrc, const cplx *F, int nrec, const long long *rec_idx,
             const cplx *d, double *grad_m, double *grad_R, double *misfit)
{
    long long N = n_nodes(p), Nc = n_cells(p);
    band_lu lu;
    if (band_factor(p, &lu)) { band_free(&lu); return -1; }
    double S[4], M[4];
    problem_tables(p, S, M);
    cplx *U = malloc(sizeof(cplx) * N), *r = malloc(sizeof(cplx) * N), *mu = malloc(sizeof(cplx) * N);
    for (long long c = 0; c < Nc; ++c) grad_m[c] = 0.0;
    for (long long i = 0; i < N; ++i) grad_R[i] = 0.0;
    double J = 0.0;
    double w = p->omega_phys;
    int d3 = p->ndim;
    for (int s = 0; s < nsrc; ++s) {
        band_solve(&lu, F + (long long)s * N, U);
        for (long long i = 0; i < N; ++i) r[i] = 0.0;
        for (int k = 0; k < nrec; ++k) {
            cplx res = U[rec_idx[k]] - d[(long long)s * nrec + k];
            J += 0.5 * creal(res * conj(res));
            r[rec_idx[k]] += conj(res);
        }
        band_solve(&lu, r, mu);
        /* cell loop: omega^2 Re sum mu_beta M U_gamma */
        long long a3[3], lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int t = 0; t < d3; ++t) { lo[t] = -1; hi[t] = p->n[t] - 1; }
        int ncorner = 1 << d3;
        for (a3[0] = lo[0]; a3[0] <= hi[0]; ++a3[0])
        for (a3[1] = lo[1]; a3[1] <= hi[1]; ++a3[1])
        for (a3[2] = (d3 == 3 ? lo[2] : 0); a3[2] <= (d3 == 3 ? hi[2] : 0); ++a3[2]) {
            long long corner[8];
            for (int b = 0; b < ncorner; ++b) {
                long long ib[3];
                int inside = 1;
                for (int t = 0; t < d3; ++t) {
                    ib[t] = a3[t] + ((b >> (d3 - 1 - t)) & 1);
                    if (ib[t] < 0 || ib[t] >= p->n[t]) inside = 0;
                }
                corner[b] = inside ? node_lin(p, ib) : -1;
            }
            cplx acc = 0.0;
            for (int b = 0; b < ncorner; ++b) {
                if (corner[b] < 0) continue;
                for (int g = 0; g < ncorner; ++g) {
                    if (corner[g] < 0) continue;
                    acc += mu[corner[b]] * M[popcount_small((unsigned)(b ^ g))] * U[corner[g]];
                }
            }
            grad_m[cell_lin(p, a3)] += w * w * creal(acc);
        }
        for (long long i = 0; i < N; ++i) grad_R[i] += w * cimag(mu[i] * U[i]);
    }
    *misfit = J;
    free(U); free(r); free(mu);
    band_free(&lu);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* misfit of the time-domain approximate solution and its gradient through    */
/* the recurrence (discrete adjoint, reverse time)                             */
/* ------------------------------------------------------------------------- */

/*
 * J = 1/2 sum_s sum_r |(P F_s)[rec_r] - d_{s,r}|^2 with P the preconditioner
 * (mode Table 1 or EXACT): the approximate solution of one application, not
 * H^{-1} F.  Each real run of P is the recurrence R_j(u) = (1 + L/2) u_{j+1}
 * - (2 - K) u_j + (1 - L/2) u_{j-1} - g_j = 0, j = 0 .. N-1, u_0 = u_{-1} = 0
 * (Def. of I_acd), read out at its output steps.  With multipliers lam_{j+1}
 * for R_j, stationarity in u_k gives the same recurrence backwards in time,
 *   (1 + L/2) lam_k = (2 - K) lam_{k+1} - (1 - L/2) lam_{k+2} - dJ/du_k,
 * lam_{N+1} = lam_{N+2} = 0 (K and L symmetric), and
 *   dJ/dtheta = sum_j lam_{j+1}^T dR_j/dtheta
 *             = sum_j lam_{j+1}^T [ (dL/2 / dtheta)(u_{j+1} - u_{j-1}) + (dK/dtheta) u_j ].
 * K depends on m = c^-2 per cell through Re H (Eq. damped Helmholtz equation,
 * App. A cell mass M): dK/dm_alpha = -(dt^2/alpha) omega_phys^2 M on the
 * cell's corners; L/2 = (beta dt / (2 alpha omega)) omega_phys R per node.
 * omega, dt, n_P (chosen from c) are held fixed.  All states are kept.
 */
int ora_grad_td(const ora_problem *p, const ora_params *q, int mode, int nsrc, const cplx *F,
                int nrec, const long long *rec_idx, const cplx *d, double *grad_m, double *grad_R,
                double *misfit)
{
    if (mode != ORA_MODE_TABLE1 && mode != ORA_MODE_EXACT) return -1;
    if (q->integrator != ORA_ACD || p->damping != ORA_DAMP_NODE) return -1;
    long long N = n_nodes(p), Nc = n_cells(p);
    long long ns = q->nsteps;
    long long jim = ns - q->nP / 4;
    double S[4], M[4];
    problem_tables(p, S, M);
    double c = q->dt * q->dt / q->alpha;
    double w = p->omega_phys;
    double cm = -c * w * w;
    double cR = q->beta * q->dt / (2.0 * q->alpha * q->omega) * w;
    int runs = (mode == ORA_MODE_EXACT) ? 2 : 1;
    double *u = malloc(sizeof(double) * (size_t)(ns + 2) * N);   /* u_{-1} .. u_N */
    double *lam = malloc(sizeof(double) * (size_t)(ns + 3) * N); /* lam_0 .. lam_{N+2} */
    double *f = malloc(sizeof(double) * N), *work = malloc(sizeof(double) * N);
    double *dj = malloc(sizeof(double) * (size_t)2 * N);        /* dJ/du at two output steps */
    cplx *U = malloc(sizeof(cplx) * N);
    for (long long a = 0; a < Nc; ++a) grad_m[a] = 0.0;
    for (long long i = 0; i < N; ++i) grad_R[i] = 0.0;
    double J = 0.0;
#define UST(j) (u + (size_t)((j) + 1) * N)
#define LAM(k) (lam + (size_t)(k) * N)
    for (int s = 0; s < nsrc; ++s) {
        const cplx *Fs = F + (long long)s * N;
        ora_precond(p, q, mode, Fs, U);
        double *dre = dj, *dim = dj + N;                       /* Re / Im of U - d at receivers */
        for (long long i = 0; i < 2 * N; ++i) dj[i] = 0.0;
        for (int k = 0; k < nrec; ++k) {
            cplx res = U[rec_idx[k]] - d[(long long)s * nrec + k];
            J += 0.5 * creal(res * conj(res));
            dre[rec_idx[k]] += creal(res);
            dim[rec_idx[k]] += cimag(res);
        }
        for (int run = 0; run < runs; ++run) {
            /* forward: the real run with forcing Re(e^{i theta_j} F) (Table 1), or
             * Re / Im parts of the complex run of S_T (EXACT, phase e^{-i 2 pi T} = 1) */
            for (long long i = 0; i < N; ++i) { UST(-1)[i] = 0.0; UST(0)[i] = 0.0; }
            for (long long j = 0; j < ns; ++j) {
                double chi = ora_window(1.0 - (double)j / (double)ns, q->rho);
                double cs = cos(2.0 * ORA_PI * (double)j / q->nP);
                double sn = sin(2.0 * ORA_PI * (double)j / q->nP);
                for (long long i = 0; i < N; ++i) {
                    double fr = creal(Fs[i]), fi = cimag(Fs[i]);
                    if (run == 1) { double t = fr; fr = fi; fi = -t; }   /* forcing -i F */
                    f[i] = chi * (cs * fr - sn * fi);
                }
                acd_step_real(p, q, UST(j), UST(j - 1), f, UST(j + 1), 1, work);
            }
            /* backward: lam_k for k = N .. 1 with -dJ/du_k at the output steps */
            for (long long i = 0; i < N; ++i) { LAM(ns + 1)[i] = 0.0; LAM(ns + 2)[i] = 0.0; }
            for (long long k = ns; k >= 1; --k) {
                for (long long i = 0; i < N; ++i) f[i] = 0.0;
                if (mode == ORA_MODE_TABLE1) {
                    if (k == ns) for (long long i = 0; i < N; ++i) f[i] -= dre[i] / c;
                    if (k == jim) for (long long i = 0; i < N; ++i) f[i] -= dim[i] / c;
                } else if (k == ns) {
                    const double *g = (run == 0) ? dre : dim;
                    for (long long i = 0; i < N; ++i) f[i] = -g[i] / c;
                }
                acd_step_real(p, q, LAM(k + 1), LAM(k + 2), f, LAM(k), 1, work);
                /* term of R_{k-1}: lam_k with u_k, u_{k-1}, u_{k-2} */
                const double *lk = LAM(k), *uk = UST(k), *uk1 = UST(k - 1), *uk2 = UST(k - 2);
                for (long long i = 0; i < N; ++i) grad_R[i] += cR * lk[i] * (uk[i] - uk2[i]);
                long long a3[3], lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
                int d3 = p->ndim;
                for (int t = 0; t < d3; ++t) { lo[t] = -1; hi[t] = p->n[t] - 1; }
                int ncorner = 1 << d3;
                for (a3[0] = lo[0]; a3[0] <= hi[0]; ++a3[0])
                for (a3[1] = lo[1]; a3[1] <= hi[1]; ++a3[1])
                for (a3[2] = (d3 == 3 ? lo[2] : 0); a3[2] <= (d3 == 3 ? hi[2] : 0); ++a3[2]) {
                    long long corner[8];
                    for (int b = 0; b < ncorner; ++b) {
                        long long ib[3];
                        int inside = 1;
                        for (int t = 0; t < d3; ++t) {
                            ib[t] = a3[t] + ((b >> (d3 - 1 - t)) & 1);
                            if (ib[t] < 0 || ib[t] >= p->n[t]) inside = 0;
                        }
                        corner[b] = inside ? node_lin(p, ib) : -1;
                    }
                    double acc = 0.0;
                    for (int b = 0; b < ncorner; ++b) {
                        if (corner[b] < 0) continue;
                        for (int g = 0; g < ncorner; ++g) {
                            if (corner[g] < 0) continue;
                            acc += lk[corner[b]] * M[popcount_small((unsigned)(b ^ g))] * uk1[corner[g]];
                        }
                    }
                    grad_m[cell_lin(p, a3)] += cm * acc;
                }
            }
        }
    }
#undef UST
#undef LAM
    *misfit = J;
    free(u); free(lam); free(f); free(work); free(dj); free(U);
    return 0;
}
