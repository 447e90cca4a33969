/*
 * FP64 CPU oracle for the two-distribution incompressible multiphase lattice Boltzmann scheme
 * (Li, Luo & Gao, "Additional interfacial force in lattice Boltzmann models for incompressible
 * multiphase flows").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct restatement of the
 * scheme that the CUDA library is checked against.  Only the tests, the smoke check and the
 * bench's CPU-baseline leg may load it.  It shares no code, header, table or helper with the
 * CUDA library: the D2Q9 tables, the stencils, the equilibria and the forcing are written out
 * here a second time, directly from the equations.
 *
 * What is computed (one time step, every cell, in the order of the equations):
 *   phi   = sum_a f_a                                        (order parameter)
 *   mu    = theta'(phi) - kappa lap(phi),  theta = beta (phi^2 - phi*^2)^2           (Eq. 1, mu)
 *   rho   = rho_B + c (rho_A - rho_B),  c = (phi + phi*) / (2 phi*)  clamped to [0,1] (Eq. 4)
 *   grad, lap: isotropic central differences over the D2Q9 neighbours            (experiments)
 *   F_s   = -phi grad(mu) (fs_form 0) or mu grad(phi) (fs_form 1),  G = (0, -rho g)  (Eq. 3)
 *   s     = rho' theta_M lap(mu)   = d_t rho + div(rho u) by Eq. 5              (s_form 0)
 *         = (rho^t - rho^{t-1}) + div(rho u)^{t-1}, the mass defect taken directly from the
 *           stored density and flux of the previous step (s_form 1; at t = 0 the initial
 *           fields stand for t-1)
 *   u     = (sum_a e_a gbar_a / cs2 + (F_s + G)/2) / (rho - s/2 [corrected])
 *   p     = sum_a gbar_a + cs2 u.grad(rho) / 2
 *   grad(psi) = grad(p) - cs2 grad(rho),  psi = p - rho cs2                        (Eq. 6-8)
 *   Gamma_a = omega_a(u) = w_a [1 + e.u/cs2 + (e.u)^2/(2 cs2^2) - u^2/(2 cs2)]
 *   g^eq_a = cs2 rho Gamma_a + psi w_a = w_a p + rho cs2 (Gamma_a - w_a)
 *   S_a   = (e_a - u).[ F Gamma_a - (Gamma_a - w_a) grad(psi) ],
 *           F = F_s + G (scheme as first stated) or F_s + G + u s (F_a removed)   (Eq. 8, Eq. 12)
 *   F_a   = -u s, the additional interfacial force (Eq. 12), exported as a field whichever
 *           scheme runs (orc_field ORC_FAX / ORC_FAY; u as above, s by s_form)
 *   gbar_a(x + e_a, t+1) = gbar_a - (gbar_a - g^eq_a)/tau_g + (1 - 1/(2 tau_g)) S_a
 *   f^eq_a (a != 0) = w_a [Gamma_f mu / cs2 + phi (e.u/cs2 + (e.u)^2/(2 cs2^2) - u^2/(2 cs2))],
 *   f^eq_0 = phi - sum_{a != 0} f^eq_a,  Gamma_f = theta_M / (tau_f - 1/2)   (recovers Eq. 2)
 *   f_a(x + e_a, t+1) = f_a - (f_a - f^eq_a)/tau_f + w_a phi div(u)   [convective form]
 *   f_form = 1 (forced order-parameter LBE) instead relaxes f to phi Gamma_a and adds
 *     (1 - 1/(2 tau_f)) (e_a - u).grad(phi) Gamma_a + theta_M lap(mu) Gamma_a:
 *     f_a(x + e_a, t+1) = f_a - (f_a - phi Gamma_a)/tau_f + (1 - 1/(2 tau_f)) (e_a - u).grad(phi) Gamma_a
 *                         + theta_M lap(mu) Gamma_a + w_a phi div(u)   [convective form]
 *     The first moment of the grad(phi) term, cs2 grad(phi), cancels the lattice diffusion
 *     cs2 (tau_f - 1/2) lap(phi) of the phi Gamma_a equilibrium; the mobility enters as the
 *     zeroth-moment source div(theta_M grad mu), applied in full each step.
 *   The moments of f^eq make the f-LBE recover d_t phi + div(phi u) = div(theta_M grad mu);
 *   Eq. 2 is the convective form d_t phi + u.grad(phi) = div(theta_M grad mu).  The two differ
 *   by phi div(u), which the weakly compressible flow does not make zero; the source
 *   w_a phi div(u) (zeroth moment phi div(u), div by the isotropic central differences) turns
 *   the recovered equation into Eq. 2.  ch_conservative = 1 drops it (conservative form).
 * Boundaries: periodic, or a no-slip wall half a cell outside the first/last row (column):
 *   links that would leave through the wall are reversed in place (half-way bounce-back), and
 *   stencils see mirrored ghost values (zero normal gradient of phi, mu and p).
 * Relaxation time of g: tau_g = mu_v / (rho cs2) + 1/2 with the dynamic viscosity
 *   mu_v = c mu_A + (1 - c) mu_B,  mu_X = rho_X cs2 (tau_g_X - 1/2).
 * Initial state: f = f^eq(phi0, mu0, u0), gbar = g^eq(p0, rho0, u0).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
#define BC_PERIODIC 0
#define BC_WALL 1

/* D2Q9: rest, four axis neighbours (E, N, W, S), four diagonals (NE, NW, SW, SE).
 * Weights as printed with the pressure distribution: 4/9, 1/9, 1/36. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

typedef struct {
    double beta, kappa, phi_star, theta_M, tau_f, tau_g_A, tau_g_B, rho_A, rho_B, gravity;
    int bc_x, bc_y, remove_Fa, storage;
    int ch_conservative;    /* 0: convective Cahn-Hilliard (Eq. 2), 1: conservative form */
    int fs_form;            /* 0: F_s = -phi grad(mu), 1: F_s = mu grad(phi) */
    int s_form;             /* 0: s by Eq. 5, 1: s from the stored rho and div(rho u) */
    int f_form;             /* 0: f^eq carrying the mu term, 1: forced order-parameter LBE */
} orc_params;

typedef struct {
    long long step;
    double sum_phi, liquid_area, centroid_x, centroid_y, vel_x, vel_y;
    double spread_radius, max_u, p_liquid, p_gas;
    int finite, pad;
} orc_diag;

typedef struct {
    int nx, ny;
    orc_params P;
    long long step;
    double *f, *g;          /* state at time t: pre-collision populations, [Q][ny][nx] */
    double *fs, *gs;        /* post-collision scratch */
    /* per-cell work fields, [ny][nx] */
    double *phi, *mu, *lap, *rho, *gpx, *gpy, *gmx, *gmy, *lmu;
    double *fsx, *fsy, *gy, *s, *ux, *uy, *p, *dpx, *dpy;
    double *divu, *w1, *w2;  /* div(u) and gradient scratch */
    double *rho_prev, *D_prev, *rux, *ruy;  /* s_form 1: rho and div(rho u) of the last step */
} orc_sim;

static int opposite(int a) {
    for (int b = 0; b < Q; ++b)
        if (EX[b] == -EX[a] && EY[b] == -EY[a]) return b;
    return -1;
}

/* Index of the neighbour i (possibly outside [0,n)) along one axis.  Periodic: wrap.
 * Wall (half a cell outside the edge): mirror, so i=-1 -> 0, i=-2 -> 1, i=n -> n-1. */
static int nb(int i, int n, int bc) {
    if (i >= 0 && i < n) return i;
    if (bc == BC_PERIODIC) {
        i %= n;
        if (i < 0) i += n;
        return i;
    }
    if (i < 0) return -1 - i;
    return 2 * n - 1 - i;
}

/* Isotropic Laplacian: lap(phi) = (2 / cs2) sum_a w_a [phi(x + e_a) - phi(x)]. */
void orc_lap_iso(int nx, int ny, int bcx, int bcy, const double* in, double* out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double acc = 0.0;
            double c = in[(size_t)y * nx + x];
            for (int a = 1; a < Q; ++a) {
                int xn = nb(x + EX[a], nx, bcx), yn = nb(y + EY[a], ny, bcy);
                acc += WT[a] * (in[(size_t)yn * nx + xn] - c);
            }
            out[(size_t)y * nx + x] = 2.0 * acc / CS2;
        }
}

/* Isotropic gradient: grad(phi) = (1 / cs2) sum_a w_a e_a phi(x + e_a). */
void orc_grad_iso(int nx, int ny, int bcx, int bcy, const double* in, double* gx, double* gy) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double ax = 0.0, ay = 0.0;
            for (int a = 1; a < Q; ++a) {
                int xn = nb(x + EX[a], nx, bcx), yn = nb(y + EY[a], ny, bcy);
                double v = in[(size_t)yn * nx + xn];
                ax += WT[a] * EX[a] * v;
                ay += WT[a] * EY[a] * v;
            }
            gx[(size_t)y * nx + x] = ax / CS2;
            gy[(size_t)y * nx + x] = ay / CS2;
        }
}

/* omega_a(u), the second-order polynomial equilibrium weight (pressure distribution). */
static double omega_a(int a, double ux, double uy) {
    double eu = EX[a] * ux + EY[a] * uy;
    double uu = ux * ux + uy * uy;
    return WT[a] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

static double liquid_fraction(const orc_params* P, double phi) {
    double c = (phi + P->phi_star) / (2.0 * P->phi_star);
    if (c < 0.0) c = 0.0;
    if (c > 1.0) c = 1.0;
    return c;
}

static double density(const orc_params* P, double phi) {
    return P->rho_B + liquid_fraction(P, phi) * (P->rho_A - P->rho_B);
}

static double drho_dphi(const orc_params* P) {
    return (P->rho_A - P->rho_B) / (2.0 * P->phi_star);
}

static double tau_g_of(const orc_params* P, double phi) {
    double c = liquid_fraction(P, phi);
    double muA = P->rho_A * CS2 * (P->tau_g_A - 0.5);
    double muB = P->rho_B * CS2 * (P->tau_g_B - 0.5);
    double mv = c * muA + (1.0 - c) * muB;
    return mv / (density(P, phi) * CS2) + 0.5;
}

static double gamma_f(const orc_params* P) {
    return P->theta_M / (P->tau_f - 0.5);
}

/* Per-node equilibria.  Gamma[a] = omega_a(u). */
void orc_node_equilibria(const orc_params* P, double phi, double mu, double rho, double p,
                         double ux, double uy, double* feq, double* geq, double* Gamma) {
    double Gf = gamma_f(P);
    double uu = ux * ux + uy * uy;
    double rest = 0.0;
    for (int a = 0; a < Q; ++a) {
        double Ga = omega_a(a, ux, uy);
        if (Gamma) Gamma[a] = Ga;
        geq[a] = WT[a] * p + rho * CS2 * (Ga - WT[a]);
        if (a > 0) {
            double eu = EX[a] * ux + EY[a] * uy;
            feq[a] = WT[a] * (Gf * mu / CS2 +
                              phi * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));
            rest += feq[a];
        }
    }
    feq[0] = phi - rest;
}

/* Per-node forcing S_a = (e_a - u).[F Gamma_a - (Gamma_a - w_a) grad(psi)]   (Eq. 8, K). */
void orc_node_forcing(double ux, double uy, double Fx, double Fy, double dpsix, double dpsiy,
                      double* S) {
    for (int a = 0; a < Q; ++a) {
        double Ga = omega_a(a, ux, uy);
        double Kx = Fx * Ga - (Ga - WT[a]) * dpsix;
        double Ky = Fy * Ga - (Ga - WT[a]) * dpsiy;
        S[a] = (EX[a] - ux) * Kx + (EY[a] - uy) * Ky;
    }
}

void orc_params_from_sigma_W(double sigma, double W, double phi_star, double* beta,
                             double* kappa) {
    /* Planar equilibrium of Eq. 1 (second form): phi = phi* tanh(2x/W) with
     * W = sqrt(2 kappa / beta) / phi* and sigma = (4/3) sqrt(2 kappa beta) phi*^3. */
    *kappa = 3.0 * sigma * W / (8.0 * phi_star * phi_star);
    *beta = 3.0 * sigma / (4.0 * W * phi_star * phi_star * phi_star * phi_star);
}

double orc_tau_from_nu(double nu) { return nu / CS2 + 0.5; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ simulation object */

static double* alloc_field(size_t n) { return (double*)calloc(n, sizeof(double)); }

void lbm_destroy_ref(orc_sim* s) {
    if (!s) return;
    double** fields[] = {&s->f, &s->g, &s->fs, &s->gs, &s->phi, &s->mu, &s->lap, &s->rho,
                         &s->gpx, &s->gpy, &s->gmx, &s->gmy, &s->lmu, &s->fsx, &s->fsy,
                         &s->gy, &s->s, &s->ux, &s->uy, &s->p, &s->dpx, &s->dpy,
                         &s->divu, &s->w1, &s->w2, &s->rho_prev, &s->D_prev, &s->rux, &s->ruy};
    for (size_t i = 0; i < sizeof(fields) / sizeof(fields[0]); ++i) free(*fields[i]);
    free(s);
}

int lbm_create_ref(int nx, int ny, const orc_params* P, orc_sim** out) {
    if (!out || !P) return -1;
    *out = NULL;
    int min_n = 3;
    if (nx < ((P->bc_x == BC_WALL) ? 4 : min_n) || ny < ((P->bc_y == BC_WALL) ? 4 : min_n))
        return -1;
    if (!(P->tau_f > 0.5 && P->tau_g_A > 0.5 && P->tau_g_B > 0.5)) return -1;
    if (!(P->rho_A > 0 && P->rho_B > 0 && P->kappa > 0 && P->beta > 0 && P->phi_star > 0))
        return -1;
    if (P->theta_M < 0) return -1;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return -2;
    s->nx = nx;
    s->ny = ny;
    s->P = *P;
    size_t N = (size_t)nx * ny;
    s->f = alloc_field(Q * N);
    s->g = alloc_field(Q * N);
    s->fs = alloc_field(Q * N);
    s->gs = alloc_field(Q * N);
    double** fields[] = {&s->phi, &s->mu, &s->lap, &s->rho, &s->gpx, &s->gpy, &s->gmx, &s->gmy,
                         &s->lmu, &s->fsx, &s->fsy, &s->gy, &s->s, &s->ux, &s->uy, &s->p,
                         &s->dpx, &s->dpy, &s->divu, &s->w1, &s->w2, &s->rho_prev, &s->D_prev,
                         &s->rux, &s->ruy};
    int ok = s->f && s->g && s->fs && s->gs;
    for (size_t i = 0; i < sizeof(fields) / sizeof(fields[0]); ++i) {
        *fields[i] = alloc_field(N);
        ok = ok && *fields[i];
    }
    if (!ok) {
        lbm_destroy_ref(s);
        return -2;
    }
    *out = s;
    return 0;
}

/* mu = theta'(phi) - kappa lap(phi), theta'(phi) = 4 beta phi (phi^2 - phi*^2). */
static void chemical_potential(orc_sim* s) {
    const orc_params* P = &s->P;
    size_t N = (size_t)s->nx * s->ny;
    orc_lap_iso(s->nx, s->ny, P->bc_x, P->bc_y, s->phi, s->lap);
    double ps2 = P->phi_star * P->phi_star;
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; ++i) {
        double ph = s->phi[i];
        s->mu[i] = 4.0 * P->beta * ph * (ph * ph - ps2) - P->kappa * s->lap[i];
    }
}

static void store_mass_flux(orc_sim* s);

int lbm_init_fields_ref(orc_sim* s, const double* phi0, const double* ux0, const double* uy0,
                        const double* p0) {
    if (!s || !phi0) return -1;
    const orc_params* P = &s->P;
    size_t N = (size_t)s->nx * s->ny;
    memcpy(s->phi, phi0, N * sizeof(double));
    chemical_potential(s);
    for (size_t i = 0; i < N; ++i) {
        double ux = ux0 ? ux0[i] : 0.0, uy = uy0 ? uy0[i] : 0.0, p = p0 ? p0[i] : 0.0;
        double feq[Q], geq[Q];
        orc_node_equilibria(P, s->phi[i], s->mu[i], density(P, s->phi[i]), p, ux, uy, feq, geq,
                            NULL);
        for (int a = 0; a < Q; ++a) {
            /* f_form 1 relaxes f to phi Gamma_a: start there */
            s->f[a * N + i] = P->f_form ? s->phi[i] * omega_a(a, ux, uy) : feq[a];
            s->g[a * N + i] = geq[a];
        }
        s->rho[i] = density(P, s->phi[i]);
        s->ux[i] = ux;
        s->uy[i] = uy;
    }
    store_mass_flux(s);   /* the initial fields stand for the step before the first */
    s->step = 0;
    return 0;
}

/* Macroscopic fields of the current state (pre-collision populations at time t). */
static void compute_moments(orc_sim* s) {
    const orc_params* P = &s->P;
    int nx = s->nx, ny = s->ny;
    size_t N = (size_t)nx * ny;
    /* order parameter */
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int a = 0; a < Q; ++a) acc += s->f[a * N + i];
        s->phi[i] = acc;
    }
    chemical_potential(s);
    orc_grad_iso(nx, ny, P->bc_x, P->bc_y, s->phi, s->gpx, s->gpy);
    orc_grad_iso(nx, ny, P->bc_x, P->bc_y, s->mu, s->gmx, s->gmy);
    orc_lap_iso(nx, ny, P->bc_x, P->bc_y, s->mu, s->lmu);
    double rp = drho_dphi(P);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; ++i) {
        double ph = s->phi[i];
        double rho = density(P, ph);
        s->rho[i] = rho;
        if (P->fs_form) {
            s->fsx[i] = s->mu[i] * s->gpx[i];
            s->fsy[i] = s->mu[i] * s->gpy[i];
        } else {
            s->fsx[i] = -ph * s->gmx[i];
            s->fsy[i] = -ph * s->gmy[i];
        }
        s->gy[i] = -rho * P->gravity;
        s->s[i] = P->s_form ? (rho - s->rho_prev[i]) + s->D_prev[i] : rp * P->theta_M * s->lmu[i];
        double jx = 0.0, jy = 0.0, m0 = 0.0;
        for (int a = 0; a < Q; ++a) {
            double gv = s->g[a * N + i];
            m0 += gv;
            jx += EX[a] * gv;
            jy += EY[a] * gv;
        }
        double denom = rho - (P->remove_Fa ? 0.5 * s->s[i] : 0.0);
        double ux = (jx / CS2 + 0.5 * s->fsx[i]) / denom;
        double uy = (jy / CS2 + 0.5 * (s->fsy[i] + s->gy[i])) / denom;
        s->ux[i] = ux;
        s->uy[i] = uy;
        s->p[i] = m0 + 0.5 * CS2 * (ux * rp * s->gpx[i] + uy * rp * s->gpy[i]);
    }
}

/* rho_prev = rho, D_prev = div(rho u) (isotropic) of the current moments. */
static void store_mass_flux(orc_sim* s) {
    const orc_params* P = &s->P;
    size_t N = (size_t)s->nx * s->ny;
    for (size_t i = 0; i < N; ++i) {
        s->rux[i] = s->rho[i] * s->ux[i];
        s->ruy[i] = s->rho[i] * s->uy[i];
    }
    orc_grad_iso(s->nx, s->ny, P->bc_x, P->bc_y, s->rux, s->D_prev, s->w1);
    orc_grad_iso(s->nx, s->ny, P->bc_x, P->bc_y, s->ruy, s->w1, s->w2);
    for (size_t i = 0; i < N; ++i) {
        s->D_prev[i] += s->w2[i];
        s->rho_prev[i] = s->rho[i];
    }
}

/* div(u) by the isotropic central differences: d(ux)/dx + d(uy)/dy. */
static void divergence(orc_sim* s) {
    const orc_params* P = &s->P;
    size_t N = (size_t)s->nx * s->ny;
    orc_grad_iso(s->nx, s->ny, P->bc_x, P->bc_y, s->ux, s->divu, s->w1);
    orc_grad_iso(s->nx, s->ny, P->bc_x, P->bc_y, s->uy, s->w1, s->w2);
    for (size_t i = 0; i < N; ++i) s->divu[i] += s->w2[i];
}

/* Post-collision populations of the current state, no streaming. */
static void collide(orc_sim* s) {
    const orc_params* P = &s->P;
    int nx = s->nx, ny = s->ny;
    size_t N = (size_t)nx * ny;
    compute_moments(s);
    orc_grad_iso(nx, ny, P->bc_x, P->bc_y, s->p, s->dpx, s->dpy);
    divergence(s);
    double rp = drho_dphi(P);
    double tf = P->tau_f;
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; ++i) {
        double ph = s->phi[i], rho = s->rho[i], ux = s->ux[i], uy = s->uy[i];
        double dpsix = s->dpx[i] - CS2 * rp * s->gpx[i];
        double dpsiy = s->dpy[i] - CS2 * rp * s->gpy[i];
        double Fx = s->fsx[i];
        double Fy = s->fsy[i] + s->gy[i];
        if (P->remove_Fa) {
            /* -F_a = u [d_t rho + div(rho u)] = u s */
            Fx += ux * s->s[i];
            Fy += uy * s->s[i];
        }
        double feq[Q], geq[Q], S[Q];
        orc_node_equilibria(P, ph, s->mu[i], rho, s->p[i], ux, uy, feq, geq, NULL);
        orc_node_forcing(ux, uy, Fx, Fy, dpsix, dpsiy, S);
        double tg = tau_g_of(P, ph);
        for (int a = 0; a < Q; ++a) {
            double gv = s->g[a * N + i];
            s->gs[a * N + i] = gv - (gv - geq[a]) / tg + (1.0 - 1.0 / (2.0 * tg)) * S[a];
            double fv = s->f[a * N + i];
            double src = P->ch_conservative ? 0.0 : WT[a] * ph * s->divu[i];
            if (P->f_form) {
                /* forced order-parameter LBE: equilibrium phi Gamma_a, forcing (e_a - u).grad(phi)
                   Gamma_a (trapezoidal weight) and the mobility source theta_M lap(mu) Gamma_a */
                double Ga = omega_a(a, ux, uy);
                double ef = (EX[a] - ux) * s->gpx[i] + (EY[a] - uy) * s->gpy[i];
                s->fs[a * N + i] = fv - (fv - ph * Ga) / tf + (1.0 - 1.0 / (2.0 * tf)) * ef * Ga +
                                   P->theta_M * s->lmu[i] * Ga + src;
            } else {
                s->fs[a * N + i] = fv - (fv - feq[a]) / tf + src;
            }
        }
    }
}

/* Streaming of one distribution: out_a(x + e_a) = in_a(x); links leaving through a wall are
 * reversed in place: out_opp(a)(x) = in_a(x). */
void orc_stream(int nx, int ny, int bcx, int bcy, const double* in, double* out) {
    size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int a = 0; a < Q; ++a) {
                int xd = x + EX[a], yd = y + EY[a];
                int hit = 0;
                if (xd < 0 || xd >= nx) {
                    if (bcx == BC_WALL) hit = 1; else xd = nb(xd, nx, bcx);
                }
                if (yd < 0 || yd >= ny) {
                    if (bcy == BC_WALL) hit = 1; else yd = nb(yd, ny, bcy);
                }
                double v = in[a * N + (size_t)y * nx + x];
                if (hit)
                    out[opposite(a) * N + (size_t)y * nx + x] = v;
                else
                    out[a * N + (size_t)yd * nx + xd] = v;
            }
}

int lbm_step_ref(orc_sim* s, int n) {
    if (!s || n < 0) return -1;
    for (int k = 0; k < n; ++k) {
        collide(s);
        if (s->P.s_form) store_mass_flux(s);
        orc_stream(s->nx, s->ny, s->P.bc_x, s->P.bc_y, s->fs, s->f);
        orc_stream(s->nx, s->ny, s->P.bc_x, s->P.bc_y, s->gs, s->g);
        s->step++;
    }
    return 0;
}

int lbm_moments_ref(orc_sim* s, double* phi, double* rho, double* ux, double* uy, double* p) {
    if (!s) return -1;
    compute_moments(s);
    size_t N = (size_t)s->nx * s->ny, B = N * sizeof(double);
    if (phi) memcpy(phi, s->phi, B);
    if (rho) memcpy(rho, s->rho, B);
    if (ux) memcpy(ux, s->ux, B);
    if (uy) memcpy(uy, s->uy, B);
    if (p) memcpy(p, s->p, B);
    return 0;
}

/* Named work fields of the current state (after lbm_moments_ref / a collision). */
enum { ORC_MU = 0, ORC_S = 1, ORC_FSX = 2, ORC_FSY = 3, ORC_DPX = 4, ORC_DPY = 5,
       ORC_GRAD_PHI_X = 6, ORC_GRAD_PHI_Y = 7, ORC_LAP_MU = 8, ORC_TAU_G = 9, ORC_DIVU = 10,
       ORC_FAX = 11, ORC_FAY = 12 };

int orc_field(orc_sim* s, int which, double* out) {
    if (!s || !out) return -1;
    size_t N = (size_t)s->nx * s->ny;
    compute_moments(s);
    orc_grad_iso(s->nx, s->ny, s->P.bc_x, s->P.bc_y, s->p, s->dpx, s->dpy);
    divergence(s);
    const double* src = NULL;
    switch (which) {
        case ORC_MU: src = s->mu; break;
        case ORC_S: src = s->s; break;
        case ORC_FSX: src = s->fsx; break;
        case ORC_FSY: src = s->fsy; break;
        case ORC_DPX: src = s->dpx; break;
        case ORC_DPY: src = s->dpy; break;
        case ORC_GRAD_PHI_X: src = s->gpx; break;
        case ORC_GRAD_PHI_Y: src = s->gpy; break;
        case ORC_LAP_MU: src = s->lmu; break;
        case ORC_DIVU: src = s->divu; break;
        case ORC_TAU_G:
            for (size_t i = 0; i < N; ++i) out[i] = tau_g_of(&s->P, s->phi[i]);
            return 0;
        case ORC_FAX:   /* the additional interfacial force F_a = -u s (Eq. 12), x and y */
            for (size_t i = 0; i < N; ++i) out[i] = -s->ux[i] * s->s[i];
            return 0;
        case ORC_FAY:
            for (size_t i = 0; i < N; ++i) out[i] = -s->uy[i] * s->s[i];
            return 0;
        default: return -1;
    }
    memcpy(out, src, N * sizeof(double));
    return 0;
}

int orc_get_state(orc_sim* s, double* f, double* g) {
    if (!s) return -1;
    size_t B = (size_t)Q * s->nx * s->ny * sizeof(double);
    if (f) memcpy(f, s->f, B);
    if (g) memcpy(g, s->g, B);
    return 0;
}

int orc_set_state(orc_sim* s, const double* f, const double* g) {
    if (!s) return -1;
    size_t B = (size_t)Q * s->nx * s->ny * sizeof(double);
    if (f) memcpy(s->f, f, B);
    if (g) memcpy(s->g, g, B);
    return 0;
}

/* Post-collision populations of the current state (before streaming). */
int orc_collide(orc_sim* s, double* fstar, double* gstar) {
    if (!s) return -1;
    collide(s);
    size_t B = (size_t)Q * s->nx * s->ny * sizeof(double);
    if (fstar) memcpy(fstar, s->fs, B);
    if (gstar) memcpy(gstar, s->gs, B);
    return 0;
}

long long orc_step_count(orc_sim* s) { return s ? s->step : -1; }

/* Diagnostics in FP64, all sums serial in row-major order:
 *   sum_phi; liquid area sum(c); centroid sum(c x)/sum(c); velocity sum(c u)/sum(c);
 *   spread radius = max over rows of sum_x(c) / 2 (half the widest liquid chord);
 *   max |u|; mean p over bulk liquid (phi > 0.9 phi*) and bulk gas (phi < -0.9 phi*). */
int lbm_diagnostics_ref(orc_sim* s, orc_diag* d) {
    if (!s || !d) return -1;
    compute_moments(s);
    const orc_params* P = &s->P;
    int nx = s->nx, ny = s->ny;
    memset(d, 0, sizeof(*d));
    double sc = 0, scx = 0, scy = 0, scu = 0, scv = 0, sphi = 0, umax = 0, chord = 0;
    double pl = 0, pg = 0, nl = 0, ng = 0;
    for (int y = 0; y < ny; ++y) {
        double row = 0.0;
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            double ph = s->phi[i];
            double c = liquid_fraction(P, ph);
            sphi += ph;
            sc += c;
            scx += c * x;
            scy += c * y;
            scu += c * s->ux[i];
            scv += c * s->uy[i];
            row += c;
            double um = sqrt(s->ux[i] * s->ux[i] + s->uy[i] * s->uy[i]);
            if (!(um <= umax)) umax = um; /* NaN propagates */
            if (ph > 0.9 * P->phi_star) { pl += s->p[i]; nl += 1; }
            if (ph < -0.9 * P->phi_star) { pg += s->p[i]; ng += 1; }
        }
        if (row > chord) chord = row;
    }
    d->step = s->step;
    d->sum_phi = sphi;
    d->liquid_area = sc;
    d->centroid_x = sc > 0 ? scx / sc : 0;
    d->centroid_y = sc > 0 ? scy / sc : 0;
    d->vel_x = sc > 0 ? scu / sc : 0;
    d->vel_y = sc > 0 ? scv / sc : 0;
    d->spread_radius = 0.5 * chord;
    d->max_u = umax;
    d->p_liquid = nl > 0 ? pl / nl : 0;
    d->p_gas = ng > 0 ? pg / ng : 0;
    d->finite = isfinite(sphi) && isfinite(umax);
    return 0;
}
