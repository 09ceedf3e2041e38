/*
 * pm_oracle.c -- plain FP64 CPU oracle for the screened EFTofDE scalar-field
 * particle-mesh path of arXiv 2604.15434 (PySCo-EFT / ECOSMOG-EFT).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library, and it is deliberately written as straightforward loops
 * over a padded (n+2)^3 array, with no blocking, fusion or reordering beyond
 * what the paper's equations state.  Compile with -ffp-contract=off so that
 * every product and sum is rounded exactly as written.
 *
 * What it computes (paper section / equation in brackets):
 *   - EFT background coefficients alpha_B(a), alpha_M(a), Omega_m(a), G_eff/G,
 *     C2, C4, nu, xi and kappa = C4/(4 E^2 a^4)        [Sec. 2.2, 2.4, 2.5, Eq. chi_scm]
 *   - the discrete chi operator N(chi) = nu*L(chi) - kappa*q2(chi) with the
 *     7-point Laplacian, the three second differences and the three 4h^2
 *     cross differences                                  [Sec. 3.2.1, Method I]
 *   - the local quadratic (Eq. chi_discrete) solved in correction form on
 *     the root that continues the linear solution (Eq. quadratic), with the
 *     discriminant floored in voids                      [Sec. 3.3]
 *   - the same local equation solved as a quadratic in the cell's Laplacian,
 *     with the squared traceless Hessian from the neighbours, and a Newton
 *     update of the cell value (operator splitting)      [Sec. 3.2.2, Method II,
 *                                                          Eq. opsplit]
 *   - red-black Gauss-Seidel sweeps and an FAS multigrid V-cycle
 *                                                        [Sec. 3.4]
 *   - CIC density assignment in 2^40 fixed point, the 5-point gradient of
 *     Psi = Psi_N + (alpha_B - alpha_M) chi, CIC force interpolation and a
 *     kick-drift                                         [Sec. 3.5, Eq. force, Eq. phipsi_mod]
 *
 * Readings where the paper is silent or ambiguous (all are pinned by tests):
 *   R-coef  alpha_B-dot/H = d alpha_B / d ln a = 3 alpha_B Omega_m(a) (optional),
 *           rho_m/(2 H^2 M^2) = (3/2) Omega_m(a) G_eff/G, H-dot/H^2 = -(3/2)Omega_m(a),
 *           Omega_m in the code-unit equations is Omega_m0.
 *   R-root  the root is the one continuous with the linear solution: the
 *           paper's (-Q - sqrt(Q^2-4PR))/(2P) for nu > 0, its mirror for nu < 0.
 *   R-sat   "set the discriminant to a very low value close to zero" is read
 *           as D_eff = max(D, D_floor) with sqrt(D_floor) = eta * 6|nu|/h^2.
 *   R-gauge periodic solvability: N(chi) = f + lambda with <chi> = 0.
 *   R-ops   Method II: the traceless Hessian from Method I's stencils; its discriminant
 *           floored at (eta nu)^2 (Method I's floor in this variable); the paper's
 *           mean subtraction of the target Laplacian is the gauge multiplier lambda.
 *   R-rb    red-black: the 12 edge neighbours share the centre's colour; a
 *           half-sweep reads them from the values at the start of the half-sweep.
 *   R-res   residual: f + lambda - N(chi) in cells with a real root, and
 *           nu*(L_sat - L(chi)) in floored cells, L_sat = 3 nu (1-eta)/(4 kappa).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOCONV 2
#define ORC_ERR_NONFINITE 3

/* ------------------------------------------------------------------ */
/* Background and EFT coefficients (Sec. 2.2 C2/C4, Eq. alpha-a, G_eff/G,
 * Eq. linearised's nu and xi, Eq. chi_scm's kappa).                    */
/* ------------------------------------------------------------------ */
typedef struct {
    double omega_m_a, alpha_B, alpha_M, geff, E2, hdot_over_h2, alphaB_dot_over_h;
    double rho_term, C2, C4, nu, xi, kappa, mu_chi, mu_psi, src;
} orc_coeffs;

void orc_coefficients(double aB0, double aM0, double a, double om0, int include_dot, orc_coeffs* c)
{
    double a3 = a * a * a;
    /* Eq. alpha-a: Omega_m(a) for a flat LCDM background (a_0 = 1). */
    c->omega_m_a = om0 / (om0 + (1.0 - om0) * a3);
    c->alpha_B = aB0 * (1.0 - c->omega_m_a) / (1.0 - om0);
    c->alpha_M = aM0 * (1.0 - c->omega_m_a) / (1.0 - om0);
    /* G_eff/G = Omega_m(a)^(alpha_M0 / (3 (1 - Omega_m0))) (Sec. 2.4). */
    c->geff = pow(c->omega_m_a, aM0 / (3.0 * (1.0 - om0)));
    /* E^2 = H^2/H0^2 for the LCDM background. */
    c->E2 = om0 / a3 + (1.0 - om0);
    /* H-dot/H^2 = d ln H / d ln a = -(3/2) Omega_m(a) for LCDM. */
    c->hdot_over_h2 = -1.5 * c->omega_m_a;
    /* alpha_B-dot / H = d alpha_B/d ln a; d Omega_m/d ln a = -3 Omega_m (1 - Omega_m). */
    c->alphaB_dot_over_h = include_dot ? 3.0 * c->alpha_B * c->omega_m_a : 0.0;
    /* rho_m / (2 H^2 M^2) with M^2 = M_*^2 f, G_eff/G = 1/f. */
    c->rho_term = 1.5 * c->omega_m_a * c->geff;
    /* C2 with alpha_T = 0 (Sec. 2.2). */
    c->C2 = -c->alpha_M + c->alpha_B * (1.0 + c->alpha_M)
          + (1.0 + c->alpha_B) * c->hdot_over_h2 + c->alphaB_dot_over_h + c->rho_term;
    c->C4 = -4.0 * c->alpha_B + 2.0 * c->alpha_M;
    /* Eq. linearised: nu = -C2 + alpha_B (2 alpha_M - alpha_B), xi = alpha_B - alpha_M. */
    c->nu = -c->C2 + c->alpha_B * (2.0 * c->alpha_M - c->alpha_B);
    c->xi = c->alpha_B - c->alpha_M;
    /* Eq. chi_scm: the screening prefactor C4 / (4 E^2 a^4). */
    c->kappa = c->C4 / (4.0 * c->E2 * a3 * a);
    c->mu_chi = c->xi / c->nu;
    c->mu_psi = 1.0 + c->xi * c->xi / c->nu;
    /* Eq. chi_scm rearranged to nu L - kappa q2 = f: f = xi (3/2)(G_eff/G) a Omega_m0 delta. */
    c->src = c->xi * 1.5 * c->geff * a * om0;
}

/* ------------------------------------------------------------------ */
/* Padded-array helpers.  A level of size n is stored with one ghost
 * layer, (n+2)^3 values, x fastest.  Every stencil of Sec. 3.2.1 reaches
 * at most one cell in each direction, so one layer suffices.           */
/* ------------------------------------------------------------------ */
static inline size_t pidx(int i, int j, int k, int n)
{
    size_t m = (size_t)n + 2;
    return ((size_t)(k + 1) * m + (size_t)(j + 1)) * m + (size_t)(i + 1);
}
static inline size_t uidx(int i, int j, int k, int n)
{
    return ((size_t)k * n + (size_t)j) * n + (size_t)i;
}
static inline int wrap(int i, int n) { return (i % n + n) % n; }

static void pad_from(const double* u, int n, double* p)
{
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) p[pidx(i, j, k, n)] = u[uidx(i, j, k, n)];
}
static void unpad_to(const double* p, int n, double* u)
{
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) u[uidx(i, j, k, n)] = p[pidx(i, j, k, n)];
}
/* Fill the ghost layer: periodic wrap (ghost == NULL) or fixed Dirichlet
 * values taken from a padded array of the same size.                   */
static void fill_ghosts(double* p, int n, const double* ghost)
{
    for (int k = -1; k <= n; ++k)
        for (int j = -1; j <= n; ++j)
            for (int i = -1; i <= n; ++i) {
                if (i >= 0 && i < n && j >= 0 && j < n && k >= 0 && k < n) continue;
                size_t d = pidx(i, j, k, n);
                if (ghost) p[d] = ghost[d];
                else p[d] = p[pidx(wrap(i, n), wrap(j, n), wrap(k, n), n)];
            }
}

/* ------------------------------------------------------------------ */
/* The discrete operator at one cell (Sec. 3.2.1).  Returns the pieces of
 * the local quadratic E(c0 + e) = G + Ep e + P e^2 in the centre value.  */
/* ------------------------------------------------------------------ */
typedef struct { double N, L, q2, G, Ep, P, D; } orc_local;

static void local_eval(const double* p, size_t c, int n, double h, double nu, double kap,
                       double rhs, orc_local* o)
{
    size_t sx = 1, sy = (size_t)n + 2, sz = sy * sy;
    double h2 = h * h;
    double c0 = p[c];
    double ax = p[c + sx] + p[c - sx];
    double ay = p[c + sy] + p[c - sy];
    double az = p[c + sz] + p[c - sz];
    /* second differences chi_xx, chi_yy, chi_zz */
    double X = (ax - 2.0 * c0) / h2;
    double Y = (ay - 2.0 * c0) / h2;
    double Z = (az - 2.0 * c0) / h2;
    /* cross differences chi_xy, chi_xz, chi_yz on the 4h^2 stencil */
    double cxy = (p[c + sx + sy] - p[c + sx - sy] - p[c - sx + sy] + p[c - sx - sy]) / (4.0 * h2);
    double cxz = (p[c + sx + sz] - p[c + sx - sz] - p[c - sx + sz] + p[c - sx - sz]) / (4.0 * h2);
    double cyz = (p[c + sy + sz] - p[c + sy - sz] - p[c - sy + sz] + p[c - sy - sz]) / (4.0 * h2);
    o->L = X + Y + Z;
    /* the bracket of Eq. chi_scm, expanded as in Sec. 3.2.1 */
    o->q2 = 2.0 * (X * Y + Y * Z + Z * X) - 2.0 * (cxy * cxy + cxz * cxz + cyz * cyz);
    o->N = nu * o->L - kap * o->q2;
    o->G = o->N - rhs;
    /* dN/dc0 and (1/2) d^2N/dc0^2: the paper's Q and P of Eq. chi_discrete
     * re-centred on the current value c0. */
    o->Ep = (-6.0 * nu + 8.0 * kap * o->L) / h2;
    o->P = -24.0 * kap / (h2 * h2);
    o->D = o->Ep * o->Ep - 4.0 * o->P * o->G;
}

/* Screening weight of a cell from its mask byte k: the cell keeps (8 - k)/8 of the
 * screening term, none for k >= 8.  Coarse FAS levels store in k how many of the cell's 8
 * children were floored or themselves partly unscreened (their mean, in eighths), so the
 * coarse operator varies continuously across the edge of a floored region. */
static double screen_w(const unsigned char* kmask, size_t u)
{
    if (!kmask) return 1.0;
    return kmask[u] >= 8 ? 0.0 : (8.0 - (double)kmask[u]) / 8.0;
}

static double floor_disc(double nu, double h, double eta)
{
    double s = eta * 6.0 * fabs(nu) / (h * h);
    return s * s;
}

/* The local correction e = c_new - c0 (Eq. quadratic, with R-root and R-sat). */
static double local_update(const orc_local* o, double nu, double Df, int* sat)
{
    double sp = (nu >= 0.0) ? -1.0 : 1.0;
    *sat = 0;
    if (o->P == 0.0) return -o->G / o->Ep;
    if (o->D < Df) {
        *sat = 1;
        return (sp * sqrt(Df) - o->Ep) / (2.0 * o->P);
    }
    double sq = sqrt(o->D);
    if (o->Ep * sp > 0.0) return -2.0 * o->G / (o->Ep + sp * sq);
    return (sp * sq - o->Ep) / (2.0 * o->P);
}

/* Residual with R-res: returns r and whether the floored piece was used. */
static double local_residual(const orc_local* o, double nu, double kap, double eta, double Df, int* sat)
{
    *sat = 0;
    if (o->P != 0.0 && o->D < Df) {
        *sat = 1;
        double Lsat = 3.0 * nu * (1.0 - eta) / (4.0 * kap);
        return nu * (Lsat - o->L);
    }
    return -o->G;
}

/* N(u) for a padded array whose ghost layer the caller has filled. */
void orc_apply_N_padded(const double* p, int n, double h, double nu, double kap, double* out)
{
    orc_local o;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                local_eval(p, pidx(i, j, k, n), n, h, nu, kap, 0.0, &o);
                out[uidx(i, j, k, n)] = o.N;
            }
}

/* N(u) on a periodic grid (Sec. 3.2.1). */
void orc_apply_N(const double* u, int n, double h, double nu, double kap, double* out)
{
    size_t m = (size_t)n + 2;
    double* p = (double*)malloc(m * m * m * sizeof(double));
    pad_from(u, n, p);
    fill_ghosts(p, n, NULL);
    orc_apply_N_padded(p, n, h, nu, kap, out);
    free(p);
}

/* ------------------------------------------------------------------ */
/* One red-black sweep (red = (i+j+k) even first), R-rb semantics.
 * kmask (nullable): per cell, the eighths of the screening term switched off
 * (0 keeps it, 8 or more removes it; coarse levels of the FAS cycle).  lam is added to the rhs of the cells
 * that carry the gauge multiplier.  Works on a padded array.            */
/* ------------------------------------------------------------------ */
static void sweep_padded(double* p, double* snap, const double* f, double lam, int n, double h,
                         double nu, double kap, double eta, const unsigned char* kmask,
                         const double* ghost)
{
    size_t m = (size_t)n + 2, tot = m * m * m;
    double Df = floor_disc(nu, h, eta);
    for (int colour = 0; colour < 2; ++colour) {
        fill_ghosts(p, n, ghost);
        memcpy(snap, p, tot * sizeof(double));
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    if (((i + j + k) & 1) != colour) continue;
                    size_t u = uidx(i, j, k, n);
                    double kc = kap * screen_w(kmask, u);
                    orc_local o;
                    int sat;
                    local_eval(snap, pidx(i, j, k, n), n, h, nu, kc, f[u] + lam, &o);
                    p[pidx(i, j, k, n)] = snap[pidx(i, j, k, n)] + local_update(&o, nu, Df, &sat);
                }
    }
    fill_ghosts(p, n, ghost);
}

/* ------------------------------------------------------------------ */
/* Method II, operator splitting (Sec. 3.2.2, Eq. opsplit; w = 1/3).
 * With Method I's second differences X, Y, Z and cross differences, the squared traceless
 * Hessian
 *     T2 = (X - L/3)^2 + (Y - L/3)^2 + (Z - L/3)^2 + 2 (chi_xy^2 + chi_xz^2 + chi_yz^2)
 * needs only the neighbours: X - L/3 = (2 a_x - a_y - a_z) / (3 h^2), a_x the sum of the
 * two x neighbours (the centre cancels), and the cross differences never hold the centre.
 * Since q2 = (2/3) L^2 - T2, the cell's equation nu L - kappa q2 = f + lambda is a
 * quadratic in its Laplacian L:
 *     a L^2 + b L + c = 0,   a = -(2/3) kappa,   b = nu,   c = kappa T2 - (f + lambda).
 * The root continuing the linear solution L = (f + lambda)/nu is taken.  Readings:
 *   - the discriminant floor of R-sat, carried to this variable: the chi-quadratic's
 *     discriminant is (6/h^2)^2 times this one, so D_L is floored at (eta nu)^2, and the
 *     floored root is the vertex-shifted one, L = L_sat;
 *   - the paper's subtraction of the mean of the target Laplacians (periodic solvability)
 *     is the gauge multiplier lambda of R-gauge, as for Method I.
 * The Newton update then moves the centre value so that its discrete Laplacian, linear in
 * the centre with slope -6/h^2, equals the root:  chi += (L_now - L_root) h^2 / 6.       */
/* ------------------------------------------------------------------ */
static double opsplit_update(const double* p, size_t c, int n, double h, double nu, double kap, double rhs,
                             double eta, int* sat)
{
    size_t sx = 1, sy = (size_t)n + 2, sz = sy * sy;
    double h2 = h * h;
    double c0 = p[c];
    double ax = p[c + sx] + p[c - sx];
    double ay = p[c + sy] + p[c - sy];
    double az = p[c + sz] + p[c - sz];
    double Lnow = (ax + ay + az - 6.0 * c0) / h2;
    double Lroot;
    *sat = 0;
    if (kap == 0.0) {
        Lroot = rhs / nu;
    } else {
        double tx = (2.0 * ax - ay - az) / (3.0 * h2);
        double ty = (2.0 * ay - ax - az) / (3.0 * h2);
        double tz = (2.0 * az - ax - ay) / (3.0 * h2);
        double cxy = (p[c + sx + sy] - p[c + sx - sy] - p[c - sx + sy] + p[c - sx - sy]) / (4.0 * h2);
        double cxz = (p[c + sx + sz] - p[c + sx - sz] - p[c - sx + sz] + p[c - sx - sz]) / (4.0 * h2);
        double cyz = (p[c + sy + sz] - p[c + sy - sz] - p[c - sy + sz] + p[c - sy - sz]) / (4.0 * h2);
        double T2 = tx * tx + ty * ty + tz * tz + 2.0 * (cxy * cxy + cxz * cxz + cyz * cyz);
        double a = -2.0 * kap / 3.0, b = nu, cc = kap * T2 - rhs;
        double D = b * b - 4.0 * a * cc;
        double Dfl = eta * nu * eta * nu;
        double sb = nu >= 0.0 ? 1.0 : -1.0;
        if (D < Dfl) {
            *sat = 1;
            Lroot = (-b + sb * sqrt(Dfl)) / (2.0 * a);
        } else {
            Lroot = -2.0 * cc / (b + sb * sqrt(D));
        }
    }
    return c0 + (Lnow - Lroot) * h2 / 6.0;
}

/* One red-black sweep of Method II, with the snapshot semantics of sweep_padded. */
static void sweep_padded_opsplit(double* p, double* snap, const double* f, double lam, int n, double h,
                                 double nu, double kap, double eta, const unsigned char* kmask,
                                 const double* ghost)
{
    size_t m = (size_t)n + 2, tot = m * m * m;
    for (int colour = 0; colour < 2; ++colour) {
        fill_ghosts(p, n, ghost);
        memcpy(snap, p, tot * sizeof(double));
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    if (((i + j + k) & 1) != colour) continue;
                    size_t u = uidx(i, j, k, n);
                    int sat;
                    p[pidx(i, j, k, n)] = opsplit_update(snap, pidx(i, j, k, n), n, h, nu, kap * screen_w(kmask, u),
                                                         f[u] + lam, eta, &sat);
                }
    }
    fill_ghosts(p, n, ghost);
}

/* Residual on a padded array; returns the count of floored cells. */
static long long residual_padded(double* p, const double* f, double lam, int n, double h, double nu,
                                 double kap, double eta, const unsigned char* kmask, const double* ghost,
                                 double* r, unsigned char* satmask)
{
    double Df = floor_disc(nu, h, eta);
    long long nsat = 0;
    fill_ghosts(p, n, ghost);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t u = uidx(i, j, k, n);
                double kc = kap * screen_w(kmask, u);
                orc_local o;
                int sat;
                local_eval(p, pidx(i, j, k, n), n, h, nu, kc, f[u] + lam, &o);
                r[u] = local_residual(&o, nu, kc, eta, Df, &sat);
                if (satmask) satmask[u] = (unsigned char)sat;
                nsat += sat;
            }
    return nsat;
}

/* Public single-operation entry points on periodic unpadded grids. */
void orc_smooth_sweep_opsplit(double* u, const double* f, double lam, int n, double h, double nu, double kap,
                              double eta, const unsigned char* kmask)
{
    size_t m = (size_t)n + 2;
    double* p = (double*)malloc(m * m * m * sizeof(double));
    double* s = (double*)malloc(m * m * m * sizeof(double));
    pad_from(u, n, p);
    sweep_padded_opsplit(p, s, f, lam, n, h, nu, kap, eta, kmask, NULL);
    unpad_to(p, n, u);
    free(p);
    free(s);
}

void orc_smooth_sweep(double* u, const double* f, double lam, int n, double h, double nu, double kap,
                      double eta, const unsigned char* kmask)
{
    size_t m = (size_t)n + 2;
    double* p = (double*)malloc(m * m * m * sizeof(double));
    double* s = (double*)malloc(m * m * m * sizeof(double));
    pad_from(u, n, p);
    sweep_padded(p, s, f, lam, n, h, nu, kap, eta, kmask, NULL);
    unpad_to(p, n, u);
    free(p);
    free(s);
}

long long orc_residual(const double* u, const double* f, double lam, int n, double h, double nu, double kap,
                       double eta, const unsigned char* kmask, double* r, unsigned char* satmask)
{
    size_t m = (size_t)n + 2;
    double* p = (double*)malloc(m * m * m * sizeof(double));
    pad_from(u, n, p);
    long long ns = residual_padded(p, f, lam, n, h, nu, kap, eta, kmask, NULL, r, satmask);
    free(p);
    return ns;
}

/* The exact coarsest-level solve alone on a periodic n^3 grid: u (in: start, out: solution)
 * of the residual pieces of R-res for right-hand side f, with the gauge multiplier and the
 * mean of u kept; kmask as for the sweep (nullable).  Returns the final lambda. */
double orc_coarse_exact(double* u, const double* f, int n, double h, double nu, double kap, double eta,
                        const unsigned char* kmask);

/* Restriction: average of the 8 children (Sec. 3.4 FAS; the paper leaves R open). */
void orc_restrict(const double* fine, int nf, double* coarse)
{
    int nc = nf / 2;
    for (int K = 0; K < nc; ++K)
        for (int J = 0; J < nc; ++J)
            for (int I = 0; I < nc; ++I) {
                double s = 0.0;
                for (int dk = 0; dk < 2; ++dk)
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di)
                            s += fine[uidx(2 * I + di, 2 * J + dj, 2 * K + dk, nf)];
                coarse[uidx(I, J, K, nc)] = 0.125 * s;
            }
}

/* Prolongation of a coarse correction by cell-centred trilinear weights
 * (3/4, 1/4 per axis), added to the fine field.  periodic != 0 wraps the
 * coarse neighbours; otherwise (fixed boundary values) a neighbour outside
 * the grid takes minus its mirror cell, so the correction vanishes on the
 * boundary face. */
void orc_prolong_add(const double* corr, int nc, double* fine, int periodic)
{
    int nf = 2 * nc;
    for (int k = 0; k < nf; ++k)
        for (int j = 0; j < nf; ++j)
            for (int i = 0; i < nf; ++i) {
                int P[3] = {i / 2, j / 2, k / 2};
                int Q[3] = {(i & 1) ? P[0] + 1 : P[0] - 1, (j & 1) ? P[1] + 1 : P[1] - 1,
                            (k & 1) ? P[2] + 1 : P[2] - 1};
                double s = 0.0;
                for (int c = 0; c < 8; ++c) {
                    int ii = (c & 1) ? Q[0] : P[0];
                    int jj = (c & 2) ? Q[1] : P[1];
                    int kk = (c & 4) ? Q[2] : P[2];
                    double w = ((c & 1) ? 0.25 : 0.75) * ((c & 2) ? 0.25 : 0.75) * ((c & 4) ? 0.25 : 0.75);
                    double sgn = 1.0;
                    if (periodic) {
                        ii = wrap(ii, nc); jj = wrap(jj, nc); kk = wrap(kk, nc);
                    } else {
                        if (ii < 0 || ii >= nc) { sgn = -sgn; ii = ii < 0 ? 0 : nc - 1; }
                        if (jj < 0 || jj >= nc) { sgn = -sgn; jj = jj < 0 ? 0 : nc - 1; }
                        if (kk < 0 || kk >= nc) { sgn = -sgn; kk = kk < 0 ? 0 : nc - 1; }
                    }
                    s += sgn * w * corr[uidx(ii, jj, kk, nc)];
                }
                fine[uidx(i, j, k, nf)] += s;
            }
}

/* ------------------------------------------------------------------ */
/* FAS multigrid (Sec. 3.4).                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    double nu, kappa, eta;
    int npre, npost, max_cycles, coarsest_n, coarse_sweeps;
    int dirichlet;              /* 0: periodic with gauge multiplier; 1: fixed ghosts */
    const double* ghosts;       /* Dirichlet: padded ghost arrays of every level, finest first */
    int smoother;               /* 0: Method I (quadratic in the cell value); 1: Method II */
    int coarse_exact;           /* 1: Newton with a dense Jacobian and LU on the coarsest grid */
} orc_mg_params;


typedef struct {
    int cycles;
    double rel_res;
    double lambda;
    long long sat_cells;
    double hist[256];
} orc_mg_info;

typedef struct {
    int n;
    double h;
    double *p, *snap, *f, *r, *ur;
    unsigned char *kmask, *sat;
    const double* ghost;
} level_t;

/* One smoothing sweep of a level with the method the parameters select. */
static void smooth_level(level_t* L, double lam, const orc_mg_params* prm)
{
    if (prm->smoother == 1)
        sweep_padded_opsplit(L->p, L->snap, L->f, lam, L->n, L->h, prm->nu, prm->kappa, prm->eta, L->kmask,
                             L->ghost);
    else
        sweep_padded(L->p, L->snap, L->f, lam, L->n, L->h, prm->nu, prm->kappa, prm->eta, L->kmask, L->ghost);
}

static double sum_arr(const double* a, size_t m)
{
    double s = 0.0;
    for (size_t i = 0; i < m; ++i) s += a[i];
    return s;
}

/* Coarsest solve: sweeps with the gauge multiplier updated after each one. */
static void coarse_solve(level_t* L, const orc_mg_params* prm, int periodic)
{
    size_t m = (size_t)L->n * L->n * L->n;
    double lam = 0.0;
    for (int it = 0; it < prm->coarse_sweeps; ++it) {
        smooth_level(L, lam, prm);
        if (periodic) {
            residual_padded(L->p, L->f, lam, L->n, L->h, prm->nu, prm->kappa, prm->eta, L->kmask, L->ghost,
                            L->r, L->sat);
            double sw = 0.0, sg = sum_arr(L->r, m);
            for (size_t i = 0; i < m; ++i) sw += L->sat[i] ? 0.0 : 1.0;
            if (sw > 0.0) lam -= sg / sw;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Exact coarsest-level solve (Sec. 3.4 FAS; the paper leaves the coarse
 * solve open).  Reading: Newton's method on the whole discrete system of
 * the level, with its Jacobian written out as a dense matrix and solved by
 * LU with partial pivoting.  Unknowns: the m cell values and, on a periodic
 * grid, the gauge multiplier lambda.  Equations: each cell's residual piece
 * of R-res with its sign flipped (N - f - lambda where the discriminant has
 * a real root, nu (L - L_sat) where it is floored) and, on a periodic grid,
 * the mean constraint sum(chi) = its value on entry, scaled by 6|nu|/h^2 so
 * that its row is of the size of the others.  The floored set is taken
 * afresh at every iterate; a backtracking line search on the residual norm
 * keeps each step from increasing it.                                   */
/* ------------------------------------------------------------------ */

/* A x = b for a dense m x m matrix (row-major), by Gaussian elimination with partial
 * pivoting; A is overwritten, b receives x.  Returns 1 on a zero pivot. */
static int dense_solve(double* A, double* b, int m)
{
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int i = k + 1; i < m; ++i)
            if (fabs(A[(size_t)i * m + k]) > fabs(A[(size_t)piv * m + k])) piv = i;
        if (A[(size_t)piv * m + k] == 0.0) return 1;
        if (piv != k) {
            for (int j = 0; j < m; ++j) {
                double t = A[(size_t)k * m + j];
                A[(size_t)k * m + j] = A[(size_t)piv * m + j];
                A[(size_t)piv * m + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < m; ++i) {
            double l = A[(size_t)i * m + k] / A[(size_t)k * m + k];
            if (l == 0.0) continue;
            for (int j = k; j < m; ++j) A[(size_t)i * m + j] -= l * A[(size_t)k * m + j];
            b[i] -= l * b[k];
        }
    }
    for (int k = m - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < m; ++j) s -= A[(size_t)k * m + j] * b[j];
        b[k] = s / A[(size_t)k * m + k];
    }
    return 0;
}

/* Unknown index of cell (i, j, k) of an n^3 level: the wrapped cell on a periodic grid,
 * -1 for a fixed (Dirichlet) ghost. */
static int exact_col(int i, int j, int k, int n, int periodic)
{
    if (periodic) return (int)uidx(wrap(i, n), wrap(j, n), wrap(k, n), n);
    if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n) return -1;
    return (int)uidx(i, j, k, n);
}

/* Residual pieces F (size m + periodic) at the padded iterate p, and with J != NULL the
 * Jacobian dF/d(chi, lambda).  Returns |F|_2. */
static double exact_system(const level_t* L, const orc_mg_params* prm, int periodic, const double* p, double lam,
                           double msum, double* F, double* J)
{
    int n = L->n, m = n * n * n, M = m + (periodic ? 1 : 0);
    double h = L->h, h2 = h * h, Df = floor_disc(prm->nu, h, prm->eta), nu = prm->nu;
    double scale = 6.0 * fabs(nu) / h2;
    if (J) memset(J, 0, (size_t)M * M * sizeof(double));
    double f2 = 0.0;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                int c = (int)uidx(i, j, k, n);
                double kc = prm->kappa * screen_w(L->kmask, (size_t)c);
                orc_local o;
                size_t pc = pidx(i, j, k, n);
                local_eval(p, pc, n, h, nu, kc, L->f[c] + (periodic ? lam : 0.0), &o);
                int fl = (o.P != 0.0 && o.D < Df);
                if (fl) F[c] = nu * (o.L - 3.0 * nu * (1.0 - prm->eta) / (4.0 * kc));
                else F[c] = o.G;
                f2 += F[c] * F[c];
                if (!J) continue;
                double* row = J + (size_t)c * M;
                /* d/d(own and face values) of nu L */
                row[exact_col(i, j, k, n, periodic)] += -6.0 * nu / h2;
                int fi[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
                for (int q = 0; q < 6; ++q) {
                    int d = exact_col(i + fi[q][0], j + fi[q][1], k + fi[q][2], n, periodic);
                    if (d >= 0) row[d] += nu / h2;
                }
                if (fl) continue;
                if (periodic) row[m] = -1.0;
                if (kc == 0.0) continue;
                /* -kappa dq2: q2 = 2(XY + YZ + ZX) - 2(cxy^2 + cxz^2 + cyz^2) */
                size_t sx = 1, sy = (size_t)n + 2, sz = sy * sy;
                double X = (p[pc + sx] + p[pc - sx] - 2.0 * p[pc]) / h2;
                double Y = (p[pc + sy] + p[pc - sy] - 2.0 * p[pc]) / h2;
                double Z = (p[pc + sz] + p[pc - sz] - 2.0 * p[pc]) / h2;
                double cxy = (p[pc + sx + sy] - p[pc + sx - sy] - p[pc - sx + sy] + p[pc - sx - sy]) / (4.0 * h2);
                double cxz = (p[pc + sx + sz] - p[pc + sx - sz] - p[pc - sx + sz] + p[pc - sx - sz]) / (4.0 * h2);
                double cyz = (p[pc + sy + sz] - p[pc + sy - sz] - p[pc - sy + sz] + p[pc - sy - sz]) / (4.0 * h2);
                double dX = 2.0 * (Y + Z), dY = 2.0 * (X + Z), dZ = 2.0 * (X + Y);
                row[exact_col(i, j, k, n, periodic)] -= kc * (-2.0 / h2) * (dX + dY + dZ);
                double dd[3] = {dX, dY, dZ};
                for (int q = 0; q < 6; ++q) {
                    int d = exact_col(i + fi[q][0], j + fi[q][1], k + fi[q][2], n, periodic);
                    if (d >= 0) row[d] -= kc * dd[q / 2] / h2;
                }
                /* cross differences: d(-2 c^2)/dc = -4c, dc/d(corner) = +-1/(4h^2) */
                double cc[3] = {cxy, cxz, cyz};
                int ax[3][2] = {{0, 1}, {0, 2}, {1, 2}};
                for (int q = 0; q < 3; ++q)
                    for (int s1 = -1; s1 <= 1; s1 += 2)
                        for (int s2 = -1; s2 <= 1; s2 += 2) {
                            int o3[3] = {0, 0, 0};
                            o3[ax[q][0]] = s1;
                            o3[ax[q][1]] = s2;
                            int d = exact_col(i + o3[0], j + o3[1], k + o3[2], n, periodic);
                            if (d >= 0) row[d] -= kc * (-4.0 * cc[q]) * (double)(s1 * s2) / (4.0 * h2);
                        }
            }
    if (periodic) {
        double s = 0.0;
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) s += p[pidx(i, j, k, n)];
        F[m] = scale * (s - msum);
        f2 += F[m] * F[m];
        if (J)
            for (int d = 0; d < m; ++d) J[(size_t)m * M + d] = scale;
    }
    return sqrt(f2);
}

static double coarse_exact(level_t* L, const orc_mg_params* prm, int periodic)
{
    int n = L->n, m = n * n * n, M = m + (periodic ? 1 : 0);
    size_t mp = (size_t)(n + 2) * (n + 2) * (n + 2);
    double* J = (double*)malloc((size_t)M * M * sizeof(double));
    double* F = (double*)malloc((size_t)M * sizeof(double));
    double* Ft = (double*)malloc((size_t)M * sizeof(double));
    double* pt = (double*)malloc(mp * sizeof(double));
    fill_ghosts(L->p, n, L->ghost);
    double msum = 0.0, fm = 0.0, fn = 0.0;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) msum += L->p[pidx(i, j, k, n)];
    for (int c = 0; c < m; ++c) fm += L->f[c] / (double)m;
    for (int c = 0; c < m; ++c) fn += (L->f[c] - (periodic ? fm : 0.0)) * (L->f[c] - (periodic ? fm : 0.0));
    fn = sqrt(fn);
    double lam = 0.0;
    double nrm = exact_system(L, prm, periodic, L->p, lam, msum, F, J);
    for (int it = 0; it < 50; ++it) {
        if (nrm <= 1e-14 * fn || nrm == 0.0) break;
        for (int q = 0; q < M; ++q) F[q] = -F[q];
        if (dense_solve(J, F, M)) break;
        double step = 1.0, nt = nrm, lt = lam;
        for (;;) {
            memcpy(pt, L->p, mp * sizeof(double));
            for (int k = 0; k < n; ++k)
                for (int j = 0; j < n; ++j)
                    for (int i = 0; i < n; ++i) pt[pidx(i, j, k, n)] += step * F[uidx(i, j, k, n)];
            fill_ghosts(pt, n, L->ghost);
            lt = periodic ? lam + step * F[m] : 0.0;
            nt = exact_system(L, prm, periodic, pt, lt, msum, Ft, NULL);
            if (nt < (1.0 - 1e-4 * step) * nrm || step < 1e-4) break;
            step *= 0.5;
        }
        if (!(nt < nrm)) break; /* no decrease along the Newton direction: keep the iterate */
        memcpy(L->p, pt, mp * sizeof(double));
        lam = lt;
        nrm = exact_system(L, prm, periodic, L->p, lam, msum, F, J);
    }
    free(J); free(F); free(Ft); free(pt);
    return lam;
}

static void vcycle(level_t* lv, int l, int nlev, double lam, const orc_mg_params* prm, int periodic)
{
    level_t* L = &lv[l];
    if (l == nlev - 1) {
        if (prm->coarse_exact) (void)coarse_exact(L, prm, periodic);
        else coarse_solve(L, prm, periodic);
        return;
    }
    level_t* C = &lv[l + 1];
    size_t m = (size_t)L->n * L->n * L->n, mc = (size_t)C->n * C->n * C->n;
    for (int s = 0; s < prm->npre; ++s)
        smooth_level(L, lam, prm);
    residual_padded(L->p, L->f, lam, L->n, L->h, prm->nu, prm->kappa, prm->eta, L->kmask, L->ghost, L->r, L->sat);
    /* project out the part of the residual the gauge multiplier absorbs */
    if (periodic) {
        double sw = 0.0, sg = sum_arr(L->r, m);
        for (size_t i = 0; i < m; ++i) sw += L->sat[i] ? 0.0 : 1.0;
        double gm = sw > 0.0 ? sg / sw : 0.0;
        for (size_t i = 0; i < m; ++i)
            if (!L->sat[i]) L->r[i] -= gm;
    }
    /* coarse mask: the unscreened fraction of a coarse cell, in eighths, is the mean of
     * its children's (1 for a floored child, whose equation is linear) */
    double* tmp = (double*)malloc(m * sizeof(double));
    for (size_t i = 0; i < m; ++i) tmp[i] = L->sat[i] ? 1.0 : 1.0 - screen_w(L->kmask, i);
    double* tc = (double*)malloc(mc * sizeof(double));
    orc_restrict(tmp, L->n, tc);
    for (size_t i = 0; i < mc; ++i) C->kmask[i] = (unsigned char)lround(tc[i] * 8.0);
    /* FAS: restrict the approximation and build f_H = N_H(R u) + R r */
    unpad_to(L->p, L->n, tmp);
    orc_restrict(tmp, L->n, C->ur);
    double* nh = (double*)malloc(mc * sizeof(double));
    pad_from(C->ur, C->n, C->p);
    fill_ghosts(C->p, C->n, C->ghost);
    {
        orc_local o;
        for (int k = 0; k < C->n; ++k)
            for (int j = 0; j < C->n; ++j)
                for (int i = 0; i < C->n; ++i) {
                    size_t u = uidx(i, j, k, C->n);
                    double kc = prm->kappa * screen_w(C->kmask, u);
                    local_eval(C->p, pidx(i, j, k, C->n), C->n, C->h, prm->nu, kc, 0.0, &o);
                    nh[u] = o.N;
                }
    }
    orc_restrict(L->r, L->n, tc);
    for (size_t i = 0; i < mc; ++i) C->f[i] = nh[i] + tc[i];
    vcycle(lv, l + 1, nlev, 0.0, prm, periodic);
    /* correction chi_h += P(chi_H - R chi_h) */
    unpad_to(C->p, C->n, nh);
    for (size_t i = 0; i < mc; ++i) nh[i] -= C->ur[i];
    unpad_to(L->p, L->n, tmp);
    orc_prolong_add(nh, C->n, tmp, periodic);
    pad_from(tmp, L->n, L->p);
    fill_ghosts(L->p, L->n, L->ghost);
    free(tmp);
    free(tc);
    free(nh);
    for (int s = 0; s < prm->npost; ++s)
        smooth_level(L, lam, prm);
}

double orc_coarse_exact(double* u, const double* f, int n, double h, double nu, double kap, double eta,
                        const unsigned char* kmask)
{
    size_t m = (size_t)n * n * n, mp = (size_t)(n + 2) * (n + 2) * (n + 2);
    level_t L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    L.h = h;
    L.p = (double*)calloc(mp, sizeof(double));
    L.f = (double*)malloc(m * sizeof(double));
    L.kmask = (unsigned char*)kmask;
    memcpy(L.f, f, m * sizeof(double));
    pad_from(u, n, L.p);
    orc_mg_params prm;
    memset(&prm, 0, sizeof(prm));
    prm.nu = nu;
    prm.kappa = kap;
    prm.eta = eta;
    double lam = coarse_exact(&L, &prm, 1);
    unpad_to(L.p, n, u);
    free(L.p);
    free(L.f);
    return lam;
}

/*
 * Solve nu L(chi) - kappa q2(chi) = f (+ lambda) to relative residual tol.
 * chi holds the initial guess on entry and the solution on exit.  Periodic
 * runs re-centre chi to zero mean after every cycle (R-gauge).
 * Returns ORC_OK, ORC_ERR_NOCONV or ORC_ERR_ARG.
 */
int orc_mg_solve(const double* f, int n, const orc_mg_params* prm, double tol, double* chi, orc_mg_info* info)
{
    if (n < 2 || (n & (n - 1)) != 0 || prm->nu == 0.0) return ORC_ERR_ARG;
    int periodic = !prm->dirichlet;
    int nlev = 1;
    while ((n >> (nlev - 1)) > prm->coarsest_n && ((n >> (nlev - 1)) % 2 == 0)) ++nlev;
    level_t* lv = (level_t*)calloc((size_t)nlev, sizeof(level_t));
    size_t goff = 0;
    for (int l = 0; l < nlev; ++l) {
        int nl = n >> l;
        size_t m = (size_t)nl * nl * nl, mp = (size_t)(nl + 2) * (nl + 2) * (nl + 2);
        lv[l].n = nl;
        lv[l].h = 1.0 / (double)nl;
        lv[l].p = (double*)calloc(mp, sizeof(double));
        lv[l].snap = (double*)calloc(mp, sizeof(double));
        lv[l].f = (double*)calloc(m, sizeof(double));
        lv[l].r = (double*)calloc(m, sizeof(double));
        lv[l].ur = (double*)calloc(m, sizeof(double));
        lv[l].kmask = l == 0 ? NULL : (unsigned char*)calloc(m, 1);
        lv[l].sat = (unsigned char*)calloc(m, 1);
        lv[l].ghost = (prm->dirichlet && prm->ghosts) ? prm->ghosts + goff : NULL;
        goff += mp;
    }
    size_t m0 = (size_t)n * n * n;
    memcpy(lv[0].f, f, m0 * sizeof(double));
    pad_from(chi, n, lv[0].p);
    fill_ghosts(lv[0].p, n, lv[0].ghost);
    /* norm of f with its mean removed (periodic) */
    double fm = periodic ? sum_arr(f, m0) / (double)m0 : 0.0, fn = 0.0;
    for (size_t i = 0; i < m0; ++i) fn += (f[i] - fm) * (f[i] - fm);
    fn = sqrt(fn);
    double lam = 0.0, rr = 0.0;
    int status = ORC_ERR_NOCONV, cyc = 0;
    long long nsat = 0;
    for (;;) {
        /* residual, gauge update and stopping test */
        nsat = residual_padded(lv[0].p, lv[0].f, lam, n, lv[0].h, prm->nu, prm->kappa, prm->eta, NULL,
                               lv[0].ghost, lv[0].r, lv[0].sat);
        double r2 = 0.0;
        if (periodic) {
            double sw = 0.0, sg = sum_arr(lv[0].r, m0);
            for (size_t i = 0; i < m0; ++i) sw += lv[0].sat[i] ? 0.0 : 1.0;
            double gm = sw > 0.0 ? sg / sw : 0.0;
            lam -= gm;
            for (size_t i = 0; i < m0; ++i) {
                double g = lv[0].r[i] - (lv[0].sat[i] ? 0.0 : gm);
                r2 += g * g;
            }
        } else {
            for (size_t i = 0; i < m0; ++i) r2 += lv[0].r[i] * lv[0].r[i];
        }
        rr = fn > 0.0 ? sqrt(r2) / fn : sqrt(r2);
        if (!isfinite(rr)) { status = ORC_ERR_NONFINITE; break; }
        if (info && cyc < 256) info->hist[cyc] = rr;
        if (rr <= tol || fn == 0.0) { status = ORC_OK; break; }
        if (cyc >= prm->max_cycles) break;
        vcycle(lv, 0, nlev, lam, prm, periodic);
        ++cyc;
        if (periodic) {
            unpad_to(lv[0].p, n, chi);
            double mu = sum_arr(chi, m0) / (double)m0;
            for (size_t i = 0; i < m0; ++i) chi[i] -= mu;
            pad_from(chi, n, lv[0].p);
        }
    }
    unpad_to(lv[0].p, n, chi);
    if (info) {
        info->cycles = cyc;
        info->rel_res = rr;
        info->lambda = lam;
        info->sat_cells = nsat;
    }
    for (int l = 0; l < nlev; ++l) {
        free(lv[l].p); free(lv[l].snap); free(lv[l].f); free(lv[l].r); free(lv[l].ur);
        free(lv[l].kmask); free(lv[l].sat);
    }
    free(lv);
    return status;
}

/* ------------------------------------------------------------------ */
/* Particle-mesh steps.                                                 */
/* ------------------------------------------------------------------ */

/* CIC weights of one coordinate x in [0,1) on n cells centred at (i+1/2)/n. */
static void cic_1d(double x, int n, int* i0, int* i1, double* w0, double* w1)
{
    double u = x * (double)n;
    double s = u - 0.5;
    double fl = floor(s);
    double d = s - fl;
    int i = (int)fl;
    *i0 = wrap(i, n);
    *i1 = wrap(i + 1, n);
    *w0 = 1.0 - d;
    *w1 = d;
}

/*
 * CIC assignment (Sec. 3.6.2: all runs use CIC) into a 2^40 fixed-point
 * int64 grid.  pos is [3][np] (x, y, z rows) in box units.  Each of the 8
 * weights is (wx*wy)*wz rounded to the nearest integer multiple of 2^-40.
 * Integer sums are order independent, so the grid is exact.
 */
void orc_deposit_cic(const double* pos, long long np, int n, int64_t* acc)
{
    const double scale = 1099511627776.0; /* 2^40 */
    memset(acc, 0, (size_t)n * n * n * sizeof(int64_t));
    for (long long p = 0; p < np; ++p) {
        int ix[2], iy[2], iz[2];
        double wx[2], wy[2], wz[2];
        cic_1d(pos[p], n, &ix[0], &ix[1], &wx[0], &wx[1]);
        cic_1d(pos[np + p], n, &iy[0], &iy[1], &wy[0], &wy[1]);
        cic_1d(pos[2 * np + p], n, &iz[0], &iz[1], &wz[0], &wz[1]);
        for (int c = 0; c < 8; ++c) {
            int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
            double w = (wx[a] * wy[b]) * wz[e];
            int64_t q = (int64_t)llrint(w * scale);
            acc[uidx(ix[a], iy[b], iz[e], n)] += q;
        }
    }
}

/* delta = rho/rho_bar - 1 with rho_bar = np / n^3 particles per cell. */
void orc_density(const int64_t* acc, int n, long long np, double* delta)
{
    const double inv = 1.0 / 1099511627776.0;
    double cells = (double)n * (double)n * (double)n;
    double fac = cells / (double)np;
    for (size_t i = 0; i < (size_t)n * n * n; ++i) delta[i] = ((double)acc[i] * inv) * fac - 1.0;
}

/*
 * Acceleration grid g = -grad Psi with Psi = Psi_N + xi_f * chi
 * (Eq. phipsi_mod; xi_f = alpha_B - alpha_M) and the five-point
 * fourth-order central difference of Sec. 3.5.2 (order 4), or the
 * two-point central difference (order 2).  acc is [3][n^3].
 */
void orc_accel_grid(const double* psiN, const double* chi, double xi_f, int n, int order, double* acc)
{
    double h = 1.0 / (double)n;
    size_t m = (size_t)n * n * n;
    double* psi = (double*)malloc(m * sizeof(double));
    for (size_t i = 0; i < m; ++i) psi[i] = psiN[i] + (chi ? xi_f * chi[i] : 0.0);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t u = uidx(i, j, k, n);
                if (order == 2) {
                    acc[u] = -(psi[uidx(wrap(i + 1, n), j, k, n)] - psi[uidx(wrap(i - 1, n), j, k, n)]) / (2.0 * h);
                    acc[m + u] = -(psi[uidx(i, wrap(j + 1, n), k, n)] - psi[uidx(i, wrap(j - 1, n), k, n)]) / (2.0 * h);
                    acc[2 * m + u] = -(psi[uidx(i, j, wrap(k + 1, n), n)] - psi[uidx(i, j, wrap(k - 1, n), n)]) / (2.0 * h);
                    continue;
                }
                double gx = (-psi[uidx(wrap(i + 2, n), j, k, n)] + 8.0 * psi[uidx(wrap(i + 1, n), j, k, n)]
                             - 8.0 * psi[uidx(wrap(i - 1, n), j, k, n)] + psi[uidx(wrap(i - 2, n), j, k, n)]) / (12.0 * h);
                double gy = (-psi[uidx(i, wrap(j + 2, n), k, n)] + 8.0 * psi[uidx(i, wrap(j + 1, n), k, n)]
                             - 8.0 * psi[uidx(i, wrap(j - 1, n), k, n)] + psi[uidx(i, wrap(j - 2, n), k, n)]) / (12.0 * h);
                double gz = (-psi[uidx(i, j, wrap(k + 2, n), n)] + 8.0 * psi[uidx(i, j, wrap(k + 1, n), n)]
                             - 8.0 * psi[uidx(i, j, wrap(k - 1, n), n)] + psi[uidx(i, j, wrap(k - 2, n), n)]) / (12.0 * h);
                acc[u] = -gx;
                acc[m + u] = -gy;
                acc[2 * m + u] = -gz;
            }
    free(psi);
}

/* CIC interpolation of a [3][n^3] grid to particles with the deposit weights. */
void orc_interp_cic(const double* grid, int n, const double* pos, long long np, double* out)
{
    size_t m = (size_t)n * n * n;
    for (long long p = 0; p < np; ++p) {
        int ix[2], iy[2], iz[2];
        double wx[2], wy[2], wz[2];
        cic_1d(pos[p], n, &ix[0], &ix[1], &wx[0], &wx[1]);
        cic_1d(pos[np + p], n, &iy[0], &iy[1], &wy[0], &wy[1]);
        cic_1d(pos[2 * np + p], n, &iz[0], &iz[1], &wz[0], &wz[1]);
        double s[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 8; ++c) {
            int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
            double w = (wx[a] * wy[b]) * wz[e];
            size_t u = uidx(ix[a], iy[b], iz[e], n);
            for (int d = 0; d < 3; ++d) s[d] += w * grid[d * m + u];
        }
        for (int d = 0; d < 3; ++d) out[d * np + p] = s[d];
    }
}

/* Kick then drift in supercomoving time: v += g dt; x = frac(x + v dt). */
void orc_kick_drift(double* pos, double* vel, const double* acc, long long np, double dt)
{
    for (long long i = 0; i < 3 * np; ++i) {
        vel[i] = vel[i] + acc[i] * dt;
        double x = pos[i] + vel[i] * dt;
        x = x - floor(x);
        if (x >= 1.0) x = 0.0;
        pos[i] = x;
    }
}
