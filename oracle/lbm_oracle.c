/*
 * FP64 CPU oracle of the pseudopotential MRT lattice Boltzmann step (D2Q9).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method of R. Huang, J. Huang, Q. Li, "Improved third-order
 * scheme in pseudopotential lattice Boltzmann model for multiphase flows" (2026).
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant with the CUDA library:
 * every table below is written out here on its own.
 *
 * Every stage follows the paper in the paper's order (Sec. 2):
 *   1. streaming in pull form, Eq. (lbe.str), with wall links closed by bounce-back
 *   2. moments rho = sum f_i, j = sum e_i f_i, Eq. (rho.rhou)
 *   3. pseudopotential psi = sqrt(2 (p_EOS - rho c_s^2) / (G dx^2)), Sec. 2 (EOS inversion)
 *   4. pairwise force F_int = -G psi(x) sum_i w(|e_i|^2) psi(x+e_i) e_i, Eq. (fint)
 *   5. velocity rho u = j + F/2, Eq. (rho.rhou)
 *   6. m = M f; m_eq and F_m of Sec. 2; Q_m original or improved, Eqs. (qm.improved),
 *      (qm46.improved)
 *   7. relaxation rates of Sec. 3: s_0 = s_j = 1, s_e = s_eps = s_p = 1/tau,
 *      (1/s_q - 1/2)(1/s_p - 1/2) = Lambda
 *   8. collision m_bar = m + F_m - S (m - m_eq + F_m/2) + S Q_m, Eq. (lbe.col);
 *      f_bar = M^-1 m_bar
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 9

/* D2Q9 velocities.  The numbering (1..4 axis vectors counter-clockwise from +x,
 * 5..8 diagonals counter-clockwise from (1,1)) is the one the sums of
 * Eqs. (ali.2) and (obl.3) require. */
static const int EX[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[NQ] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WEQ[NQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Orthogonal transformation matrix of Lallemand & Luo (cited in Sec. 2), moment order
 * [rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy].  Its rows are fixed by m_eq and F_m of
 * Sec. 2 and by Eq. (ali.3). */
static const double MM[NQ][NQ] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},          {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},      {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},       {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},       {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
/* squared row norms: M^-1 = M^T diag(1 / MNORM) */
static const double MNORM[NQ] = {9, 36, 36, 6, 12, 6, 12, 4, 4};

/* Eq. (fint): nearest-neighbour weights w(1) = 1/3, w(2) = 1/12 */
static double omega_sc(int i) { return (i == 0) ? 0.0 : (i <= 4 ? 1.0 / 3.0 : 1.0 / 12.0); }

typedef struct {
    int32_t nx, ny, periodic_x, periodic_y;
    int32_t scheme;      /* 0 original Q_m (Huang & Wu), 1 improved Q_m (this paper) */
    int32_t q2_original; /* debug reading: improved Q4, Q6 with the original Q2 = -Q1 */
    int32_t eos;         /* 0 van der Waals (Sec. 3), 1 Carnahan-Starling */
    int32_t force_mode;  /* 0 constant force density, 1 (rho - rho_g) g, 2 per-node field */
    double a, b, R, T, K_eos;
    double G;
    double k1, k2; /* epsilon = -8 (k1 + k2) */
    double tau_l, tau_g, rho_l, rho_g;
    double Lambda;
    double Fx, Fy;
    double rho_s;
} or_params;

typedef struct {
    or_params p;
    int64_t n;
    double *A, *B;       /* 9 planes [i][y][x]: stored post-collision populations */
    uint8_t *solid;      /* n, or NULL */
    double *wall_u;      /* 2n (x plane then y plane), velocity of solid nodes, or NULL */
    double *q;           /* 8n: q[(d-1) n + node] = wall distance fraction on link d, or NULL */
    double *fext;        /* 2n: external force density field (force_mode 2), or NULL */
    double *wall_rho;    /* n: virtual density of each solid node, or NULL (all walls rho_s) */
    double *fpull;       /* 9n scratch: pulled (pre-collision) populations */
    double *rho, *jx, *jy, *psi;
    double drag[2];
    int64_t step;
} or_sim;

/* ---------------------------------------------------------------- EOS ----- */

/* van der Waals, Sec. 3: p = K (rho R T / (1 - b rho) - a rho^2).
 * Carnahan-Starling (named in Sec. 2 as an example; standard published form):
 * p = K (rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2), eta = b rho / 4. */
double or_p_eos(const or_params *p, double rho)
{
    if (p->eos == 0) {
        return p->K_eos * (rho * p->R * p->T / (1.0 - p->b * rho) - p->a * rho * rho);
    }
    double eta = p->b * rho / 4.0;
    double num = 1.0 + eta + eta * eta - eta * eta * eta;
    double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
    return p->K_eos * (rho * p->R * p->T * num / den - p->a * rho * rho);
}

/* Sec. 2: psi = sqrt(2 (p_EOS - rho c_s^2) / (G dx^2)), c_s^2 = 1/3, dx = 1 */
double or_psi(const or_params *p, double rho)
{
    return sqrt(2.0 * (or_p_eos(p, rho) - rho / 3.0) / p->G);
}

/* ------------------------------------------------------------ geometry ---- */

static int64_t node_of(const or_sim *s, int x, int y) { return (int64_t)y * s->p.nx + x; }

/* Wrap (x, y) into the domain along periodic directions; return 0 when the point
 * lies outside along a non-periodic direction (it is then a wall). */
static int wrap(const or_sim *s, int *x, int *y)
{
    int nx = s->p.nx, ny = s->p.ny;
    if (*x < 0 || *x >= nx) {
        if (!s->p.periodic_x) return 0;
        *x = ((*x % nx) + nx) % nx;
    }
    if (*y < 0 || *y >= ny) {
        if (!s->p.periodic_y) return 0;
        *y = ((*y % ny) + ny) % ny;
    }
    return 1;
}

/* 1 when (x, y) is a wall: outside a non-periodic edge, or a solid node */
static int is_wall(const or_sim *s, int x, int y)
{
    if (!wrap(s, &x, &y)) return 1;
    return s->solid ? (s->solid[node_of(s, x, y)] != 0) : 0;
}

/* velocity of the wall at (x, y); zero for domain edges and resting solids */
static void wall_velocity(const or_sim *s, int x, int y, double *ux, double *uy)
{
    *ux = 0.0;
    *uy = 0.0;
    if (!s->wall_u) return;
    if (!wrap(s, &x, &y)) return;
    int64_t k = node_of(s, x, y);
    *ux = s->wall_u[k];
    *uy = s->wall_u[s->n + k];
}

/* ------------------------------------------------------------ streaming --- */

/* Eq. (lbe.str) in pull form: f_i(x) = f_bar_i(x - e_i).  When x - e_i is a wall
 * the population that left x toward it (direction o = opposite of i) comes back:
 *   half-way (q = 1/2): f_i = f_bar_o(x) + mw
 *   q <  1/2: f_i = 2q f_bar_o(x) + (1 - 2q) f_bar_o(x + e_i) + mw
 *   q >= 1/2: f_i = f_bar_o(x) / (2q) + (2q - 1)/(2q) f_bar_i(x) + mw / (2q)
 * (interpolated bounce-back of Bouzidi et al. with the moving-wall term of Lallemand
 * & Luo), mw = 2 w_o rho_w (e_i . u_w) / c_s^2 and rho_w = sum_k f_bar_k(x), the
 * density at x before the last collision.  The paper cites its own wall scheme but
 * does not define it; these standard forms stand in for it.  *mom (may be NULL)
 * receives the momentum this link hands to the wall, -e_i (f_bar_o(x) + f_i). */
static double pull_one(const or_sim *s, const double *A, int x, int y, int i, double mom[2])
{
    const int64_t n = s->n;
    int xs = x - EX[i], ys = y - EY[i];
    if (!is_wall(s, xs, ys)) {
        wrap(s, &xs, &ys);
        return A[i * n + node_of(s, xs, ys)];
    }
    const int o = OPP[i];
    const int64_t k = node_of(s, x, y);
    double rho_w = 0.0;
    for (int m = 0; m < NQ; ++m) rho_w += A[m * n + k];
    double uwx, uwy;
    wall_velocity(s, xs, ys, &uwx, &uwy);
    double mw = 2.0 * WEQ[o] * rho_w * (EX[i] * uwx + EY[i] * uwy) * 3.0;
    double q = s->q ? s->q[(int64_t)(o - 1) * n + k] : 0.5;
    int xb = x + EX[i], yb = y + EY[i];
    if (q < 0.5 && is_wall(s, xb, yb)) q = 0.5; /* no second fluid node: half-way */
    double f;
    if (q < 0.5) {
        wrap(s, &xb, &yb);
        f = 2.0 * q * A[o * n + k] + (1.0 - 2.0 * q) * A[o * n + node_of(s, xb, yb)] + mw;
    } else if (q == 0.5) {
        f = A[o * n + k] + mw;
    } else {
        f = A[o * n + k] / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * A[i * n + k] + mw / (2.0 * q);
    }
    if (mom) {
        mom[0] += -(double)EX[i] * (A[o * n + k] + f);
        mom[1] += -(double)EY[i] * (A[o * n + k] + f);
    }
    return f;
}

/* ------------------------------------------------------------ collision --- */

/* m = M f */
static void to_moments(const double f[NQ], double m[NQ])
{
    for (int k = 0; k < NQ; ++k) {
        double acc = 0.0;
        for (int i = 0; i < NQ; ++i) acc += MM[k][i] * f[i];
        m[k] = acc;
    }
}

/* f = M^-1 m = M^T diag(1/MNORM) m */
static void from_moments(const double m[NQ], double f[NQ])
{
    for (int i = 0; i < NQ; ++i) {
        double acc = 0.0;
        for (int k = 0; k < NQ; ++k) acc += MM[k][i] * (m[k] / MNORM[k]);
        f[i] = acc;
    }
}

/* equilibrium moments of Sec. 2 (c = 1) */
static void equilibrium_moments(double rho, double ux, double uy, double meq[NQ])
{
    double u2 = ux * ux + uy * uy;
    meq[0] = rho;
    meq[1] = -2.0 * rho + 3.0 * rho * u2;
    meq[2] = rho - 3.0 * rho * u2;
    meq[3] = rho * ux;
    meq[4] = -rho * ux;
    meq[5] = rho * uy;
    meq[6] = -rho * uy;
    meq[7] = rho * ux * ux - rho * uy * uy;
    meq[8] = rho * ux * uy;
}

/* discrete force term F_m of Sec. 2 (total force, c = 1) */
static void force_moments(double Fx, double Fy, double ux, double uy, double Fm[NQ])
{
    double Fu = Fx * ux + Fy * uy;
    Fm[0] = 0.0;
    Fm[1] = 6.0 * Fu;
    Fm[2] = -6.0 * Fu;
    Fm[3] = Fx;
    Fm[4] = -Fx;
    Fm[5] = Fy;
    Fm[6] = -Fy;
    Fm[7] = 2.0 * Fx * ux - 2.0 * Fy * uy;
    Fm[8] = Fx * uy + Fy * ux;
}

/* Discrete source term Q_m.  Original (Huang & Wu, Sec. 2):
 *   Q1 = 3(k1+2k2)|F_int|^2/(G psi^2), Q2 = -Q1, Q7 = k1 (F_x^2 - F_y^2)/(G psi^2),
 *   Q8 = k1 F_x F_y/(G psi^2), other entries zero.
 * Improved, Eqs. (qm.improved) and (qm46.improved) with Q2 = -Q1/2 (Sec. 2.2):
 *   Q4 = ((30 eps - 15)/16 F_x^2/(G psi^2) - 3 eps/8 F_y^2/(G psi^2)) u_x
 *   Q6 = ((30 eps - 15)/16 F_y^2/(G psi^2) - 3 eps/8 F_x^2/(G psi^2)) u_y
 * with eps = -8 (k1 + k2).  F is the pairwise force F_int only. */
static void source_moments(const or_params *p, double Fix, double Fiy, double psi, double ux,
                           double uy, double Q[NQ])
{
    double Gpsi2 = p->G * psi * psi;
    double X = Fix * Fix / Gpsi2;
    double Y = Fiy * Fiy / Gpsi2;
    double eps = -8.0 * (p->k1 + p->k2);
    for (int k = 0; k < NQ; ++k) Q[k] = 0.0;
    Q[1] = 3.0 * (p->k1 + 2.0 * p->k2) * (X + Y);
    Q[7] = p->k1 * (Fix * Fix - Fiy * Fiy) / Gpsi2;
    Q[8] = p->k1 * Fix * Fiy / Gpsi2;
    if (p->scheme == 0) {
        Q[2] = -Q[1];
    } else {
        Q[2] = p->q2_original ? -Q[1] : -Q[1] / 2.0;
        Q[4] = ((30.0 * eps - 15.0) / 16.0 * X - 3.0 * eps / 8.0 * Y) * ux;
        Q[6] = ((30.0 * eps - 15.0) / 16.0 * Y - 3.0 * eps / 8.0 * X) * uy;
    }
}

/* relaxation time tau(rho): constant when tau_l == tau_g, otherwise the kinematic
 * viscosity nu = (tau - 1/2)/3 is interpolated linearly in rho between (rho_g, nu_g)
 * and (rho_l, nu_l), clamped outside that interval. */
static double tau_of(const or_params *p, double rho)
{
    if (p->tau_l == p->tau_g) return p->tau_l;
    double nu_l = (p->tau_l - 0.5) / 3.0, nu_g = (p->tau_g - 0.5) / 3.0;
    double w = (rho - p->rho_g) / (p->rho_l - p->rho_g);
    if (w < 0.0) w = 0.0;
    if (w > 1.0) w = 1.0;
    double nu = nu_g + w * (nu_l - nu_g);
    return 3.0 * nu + 0.5;
}

/* Collision of one node: stages 5-8 of the header.  Inputs are the pulled populations,
 * psi(x), S = sum_i w_i psi(x+e_i) e_i (so that F_int = -G psi S) and the external
 * force.  Optional outputs (may be NULL): velocity, m, m_eq, F_m, Q_m. */
void or_collide_node(const or_params *p, const double f[NQ], double psi, double Sx, double Sy,
                     double Fex, double Fey, double fbar[NQ], double uout[2], double mout[NQ],
                     double meqout[NQ], double Fmout[NQ], double Qout[NQ])
{
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < NQ; ++i) {
        rho += f[i];
        jx += EX[i] * f[i];
        jy += EY[i] * f[i];
    }
    double Fix = -p->G * psi * Sx, Fiy = -p->G * psi * Sy; /* Eq. (fint) */
    double Fx = Fix + Fex, Fy = Fiy + Fey;                 /* total force */
    double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho; /* Eq. (rho.rhou) */
    double m[NQ], meq[NQ], Fm[NQ], Q[NQ], s[NQ], mbar[NQ];
    to_moments(f, m);
    equilibrium_moments(rho, ux, uy, meq);
    force_moments(Fx, Fy, ux, uy, Fm);
    source_moments(p, Fix, Fiy, psi, ux, uy, Q);
    double tau = tau_of(p, rho);
    double sp = 1.0 / tau;
    double sq = 1.0 / (0.5 + p->Lambda / (tau - 0.5));
    s[0] = 1.0;
    s[1] = sp;
    s[2] = sp;
    s[3] = 1.0;
    s[4] = sq;
    s[5] = 1.0;
    s[6] = sq;
    s[7] = sp;
    s[8] = sp;
    for (int k = 0; k < NQ; ++k)
        mbar[k] = m[k] + Fm[k] - s[k] * (m[k] - meq[k] + 0.5 * Fm[k]) + s[k] * Q[k]; /* (lbe.col) */
    from_moments(mbar, fbar);
    if (uout) {
        uout[0] = ux;
        uout[1] = uy;
    }
    if (mout) memcpy(mout, m, sizeof m);
    if (meqout) memcpy(meqout, meq, sizeof meq);
    if (Fmout) memcpy(Fmout, Fm, sizeof Fm);
    if (Qout) memcpy(Qout, Q, sizeof Q);
}

/* ------------------------------------------------------------ lifetime ---- */

or_sim *or_create(const or_params *p)
{
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    if (!s) return NULL;
    s->p = *p;
    s->n = (int64_t)p->nx * p->ny;
    s->A = (double *)calloc((size_t)(NQ * s->n), sizeof(double));
    s->B = (double *)calloc((size_t)(NQ * s->n), sizeof(double));
    s->fpull = (double *)calloc((size_t)(NQ * s->n), sizeof(double));
    s->rho = (double *)calloc((size_t)s->n, sizeof(double));
    s->jx = (double *)calloc((size_t)s->n, sizeof(double));
    s->jy = (double *)calloc((size_t)s->n, sizeof(double));
    s->psi = (double *)calloc((size_t)s->n, sizeof(double));
    return s;
}

void or_destroy(or_sim *s)
{
    if (!s) return;
    free(s->A);
    free(s->B);
    free(s->fpull);
    free(s->rho);
    free(s->jx);
    free(s->jy);
    free(s->psi);
    free(s->solid);
    free(s->wall_u);
    free(s->q);
    free(s->fext);
    free(s->wall_rho);
    free(s);
}

static void *dup_or_null(const void *src, size_t bytes)
{
    if (!src) return NULL;
    void *d = malloc(bytes);
    memcpy(d, src, bytes);
    return d;
}

void or_set_geometry(or_sim *s, const uint8_t *solid, const double *wall_u, const double *q,
                     const double *fext)
{
    free(s->solid);
    free(s->wall_u);
    free(s->q);
    free(s->fext);
    s->solid = (uint8_t *)dup_or_null(solid, (size_t)s->n);
    s->wall_u = (double *)dup_or_null(wall_u, (size_t)(2 * s->n) * sizeof(double));
    s->q = (double *)dup_or_null(q, (size_t)(8 * s->n) * sizeof(double));
    s->fext = (double *)dup_or_null(fext, (size_t)(2 * s->n) * sizeof(double));
}

/* Virtual density per solid node (the wettability of each wall, after Benzi et al.'s
 * virtual-density walls that Sec. 3 uses with one value rho_s); NULL restores rho_s for
 * every wall.  Walls beyond a non-periodic edge keep rho_s. */
void or_set_wall_density(or_sim *s, const double *wall_rho)
{
    free(s->wall_rho);
    s->wall_rho = (double *)dup_or_null(wall_rho, (size_t)s->n * sizeof(double));
}

/* Initial state: f_bar = M^-1 m_eq(rho0, u0) at fluid nodes (the paper does not state
 * an initialisation); solid nodes hold the same, unused. */
void or_init(or_sim *s, const double *rho, const double *ux, const double *uy)
{
    for (int64_t k = 0; k < s->n; ++k) {
        double meq[NQ], f[NQ];
        equilibrium_moments(rho[k], ux ? ux[k] : 0.0, uy ? uy[k] : 0.0, meq);
        from_moments(meq, f);
        for (int i = 0; i < NQ; ++i) s->A[i * s->n + k] = f[i];
    }
    s->step = 0;
}

void or_set_state(or_sim *s, const double *A) { memcpy(s->A, A, sizeof(double) * NQ * s->n); }
void or_get_state(const or_sim *s, double *A) { memcpy(A, s->A, sizeof(double) * NQ * s->n); }
int64_t or_step_count(const or_sim *s) { return s->step; }

/* Threads the parallel row loops use (1 without OpenMP); the results do not depend on it. */
#ifdef _OPENMP
#include <omp.h>
int or_threads(void) { return omp_get_max_threads(); }
#else
int or_threads(void) { return 1; }
#endif

/* --------------------------------------------------------------- a step --- */

/* stages 1-3 for every node: pulled populations, rho, j, psi (walls: psi(rho_s)).
 * The wall momentum of each row is kept apart and summed in row order afterwards. */
static void pull_moments_psi(or_sim *s)
{
    const int nx = s->p.nx, ny = s->p.ny;
    const int64_t n = s->n;
    double *row_mom = (double *)calloc((size_t)(2 * ny), sizeof(double));
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t k = node_of(s, x, y);
            if (s->solid && s->solid[k]) {
                const double rs = s->wall_rho ? s->wall_rho[k] : s->p.rho_s;
                s->rho[k] = rs;
                s->jx[k] = s->jy[k] = 0.0;
                s->psi[k] = or_psi(&s->p, rs);
                continue;
            }
            double rho = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < NQ; ++i) {
                double f = pull_one(s, s->A, x, y, i, row_mom + 2 * y);
                s->fpull[i * n + k] = f;
                rho += f;
                jx += EX[i] * f;
                jy += EY[i] * f;
            }
            s->rho[k] = rho;
            s->jx[k] = jx;
            s->jy[k] = jy;
            s->psi[k] = or_psi(&s->p, rho);
        }
    }
    s->drag[0] = 0.0;
    s->drag[1] = 0.0;
    for (int y = 0; y < ny; ++y) {
        s->drag[0] += row_mom[2 * y];
        s->drag[1] += row_mom[2 * y + 1];
    }
    free(row_mom);
}

/* psi of a neighbour: psi(rho_s) beyond a non-periodic edge (virtual density, Sec. 3);
 * a solid node holds the psi of its own virtual density, set by pull_moments_psi */
static double psi_at(const or_sim *s, int x, int y)
{
    if (!wrap(s, &x, &y)) return or_psi(&s->p, s->p.rho_s);
    return s->psi[node_of(s, x, y)];
}

/* S = sum_{i=1..8} w(|e_i|^2) psi(x + e_i) e_i, so that Eq. (fint) reads F_int = -G psi(x) S */
static void stencil_S(const or_sim *s, int x, int y, double *Sx, double *Sy)
{
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < NQ; ++i) {
        double ps = psi_at(s, x + EX[i], y + EY[i]);
        sx += omega_sc(i) * ps * EX[i];
        sy += omega_sc(i) * ps * EY[i];
    }
    *Sx = sx;
    *Sy = sy;
}

static void external_force(const or_sim *s, int64_t k, double rho, double *Fx, double *Fy)
{
    if (s->p.force_mode == 0) {
        *Fx = s->p.Fx;
        *Fy = s->p.Fy;
    } else if (s->p.force_mode == 1) { /* gravity, Sec. 3.3: F = (rho - rho_g) g */
        *Fx = (rho - s->p.rho_g) * s->p.Fx;
        *Fy = (rho - s->p.rho_g) * s->p.Fy;
    } else {
        *Fx = s->fext ? s->fext[k] : 0.0;
        *Fy = s->fext ? s->fext[s->n + k] : 0.0;
    }
}

void or_step(or_sim *s, int64_t nsteps)
{
    const int nx = s->p.nx, ny = s->p.ny;
    const int64_t n = s->n;
    for (int64_t t = 0; t < nsteps; ++t) {
        pull_moments_psi(s);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int64_t k = node_of(s, x, y);
                if (s->solid && s->solid[k]) {
                    for (int i = 0; i < NQ; ++i) s->B[i * n + k] = s->A[i * n + k];
                    continue;
                }
                double f[NQ], fbar[NQ], Sx, Sy, Fex, Fey;
                for (int i = 0; i < NQ; ++i) f[i] = s->fpull[i * n + k];
                stencil_S(s, x, y, &Sx, &Sy);
                external_force(s, k, s->rho[k], &Fex, &Fey);
                or_collide_node(&s->p, f, s->psi[k], Sx, Sy, Fex, Fey, fbar, NULL, NULL, NULL,
                                NULL, NULL);
                for (int i = 0; i < NQ; ++i) s->B[i * n + k] = fbar[i];
            }
        }
        double *tmp = s->A;
        s->A = s->B;
        s->B = tmp;
        s->step += 1;
    }
}

/* Macroscopic fields of the current state (the pre-collision state that the next step
 * pulls): rho, u (with the half-force term), F_int, psi, Q_m (9 planes) and the pulled
 * populations (9 planes).  Any output may be NULL.  Solid nodes report rho_s, u = 0. */
void or_fields(or_sim *s, double *rho, double *ux, double *uy, double *Fix, double *Fiy,
               double *psi, double *Q, double *fpull)
{
    const int nx = s->p.nx, ny = s->p.ny;
    const int64_t n = s->n;
    pull_moments_psi(s);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t k = node_of(s, x, y);
            int solid = s->solid && s->solid[k];
            double f[NQ], fbar[NQ], u[2] = {0.0, 0.0}, Qk[NQ] = {0}, Sx = 0.0, Sy = 0.0;
            if (!solid) {
                double Fex, Fey;
                for (int i = 0; i < NQ; ++i) f[i] = s->fpull[i * n + k];
                stencil_S(s, x, y, &Sx, &Sy);
                external_force(s, k, s->rho[k], &Fex, &Fey);
                or_collide_node(&s->p, f, s->psi[k], Sx, Sy, Fex, Fey, fbar, u, NULL, NULL, NULL,
                                Qk);
            }
            if (rho) rho[k] = s->rho[k];
            if (ux) ux[k] = u[0];
            if (uy) uy[k] = u[1];
            if (Fix) Fix[k] = solid ? 0.0 : -s->p.G * s->psi[k] * Sx;
            if (Fiy) Fiy[k] = solid ? 0.0 : -s->p.G * s->psi[k] * Sy;
            if (psi) psi[k] = s->psi[k];
            for (int i = 0; i < NQ; ++i) {
                if (Q) Q[i * n + k] = Qk[i];
                if (fpull) fpull[i * n + k] = solid ? 0.0 : s->fpull[i * n + k];
            }
        }
    }
}

/* Diagnostics of the current state, all sums over fluid nodes:
 *  out[0] mass sum rho
 *  out[1..2] population momentum sum j (sum_i e_i f_i, without the half force)
 *  out[3..4] total force sum F (F_int + F_ext)
 *  out[5..6] momentum handed to the walls by the streaming that produced this state
 *  out[7] sum over the liquid region (rho > (rho_l + rho_g)/2) of rho u_y,
 *  out[8] sum over the liquid region of rho  (U_c = out[7]/out[8], Sec. 3.3)
 *  out[9] max |u| */
void or_diagnostics(or_sim *s, double out[10])
{
    const int nx = s->p.nx, ny = s->p.ny;
    const int64_t n = s->n;
    pull_moments_psi(s);
    double acc[10] = {0};
    double rho_mid = 0.5 * (s->p.rho_l + s->p.rho_g);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t k = node_of(s, x, y);
            if (s->solid && s->solid[k]) continue;
            double f[NQ], fbar[NQ], u[2], Sx, Sy, Fex, Fey;
            for (int i = 0; i < NQ; ++i) f[i] = s->fpull[i * n + k];
            stencil_S(s, x, y, &Sx, &Sy);
            external_force(s, k, s->rho[k], &Fex, &Fey);
            or_collide_node(&s->p, f, s->psi[k], Sx, Sy, Fex, Fey, fbar, u, NULL, NULL, NULL,
                            NULL);
            double rho = s->rho[k];
            acc[0] += rho;
            acc[1] += s->jx[k];
            acc[2] += s->jy[k];
            acc[3] += -s->p.G * s->psi[k] * Sx + Fex;
            acc[4] += -s->p.G * s->psi[k] * Sy + Fey;
            if (rho > rho_mid) {
                acc[7] += rho * u[1];
                acc[8] += rho;
            }
            double um = sqrt(u[0] * u[0] + u[1] * u[1]);
            if (um > acc[9]) acc[9] = um;
        }
    }
    acc[5] = s->drag[0];
    acc[6] = s->drag[1];
    memcpy(out, acc, sizeof acc);
}

/* The oracle's lattice tables, exported so that tests can check them against the
 * properties the paper and the textbook fix (orthogonality, weights, numbering). */
void or_tables(double M[NQ * NQ], double w[NQ], int ex[NQ], int ey[NQ], int opp[NQ])
{
    for (int k = 0; k < NQ; ++k)
        for (int i = 0; i < NQ; ++i) M[k * NQ + i] = MM[k][i];
    for (int i = 0; i < NQ; ++i) {
        w[i] = WEQ[i];
        ex[i] = EX[i];
        ey[i] = EY[i];
        opp[i] = OPP[i];
    }
}
