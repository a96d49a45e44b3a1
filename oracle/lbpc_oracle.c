/*
 * lbpc_oracle.c -- plain FP64 CPU oracle of the coupled flow + enthalpy lattice
 * Boltzmann step for 3D solid-liquid phase change (Li & He, Sec. 2.2-2.5).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke() check and the
 * cpu_baseline / reference legs of bench.py.  The CUDA path never calls it and
 * shares nothing with it.
 *
 * One time step, in the paper's order (Eq. 5-7 / 21-25 for g, Eq. 49-56 for f):
 *   1. h = sum_a g_a                                   (Eq. 9, zeroth moment)
 *   2. (T, f_l) from h                                 (Eq. 2, inverted; see invert())
 *   3. rho = sum f, j = sum f e                        (Eq. 56)
 *   4. buoyancy F_b (Eq. 55), solid-phase force, velocity u (Eq. 56)
 *   5. collide f in moment space (Eq. 49) and g (Eq. 6 SRT or Eq. 21 MRT)
 *   6. stream both lattices (Eq. 5 / Eq. 50) and apply the wall rules.
 * Readings of points the paper leaves open are marked READING in the comments.
 */
#include "lbpc_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D3Q7 velocity set, Eq. 3 (c = 1). */
static const int E7[7][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

/* D3Q19 velocity set, Eq. 48, in the printed order. */
static const int E19[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, 1, 0}, {1, -1, 0},  {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1},
    {-1, 0, -1}, {0, 1, 1}, {0, -1, 1},  {0, 1, -1},  {0, -1, -1}};

/* Moment transform of the enthalpy lattice, Eq. 24. */
static const double NMAT[7][7] = {
    {1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0},
    {0, 0, 0, 0, 0, 1, -1},
    {6, -1, -1, -1, -1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1},
    {0, 0, 0, 1, 1, -1, -1}};

/* Moment transform of the flow lattice, Eq. 51, as printed. */
static const double MMAT[19][19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
    {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1}};

struct orc_state {
    int nx, ny, nz;
    long N;
    orc_params p;
    /* derived lattice constants */
    double dT, L, hs, hl, chi, nu, gbeta, U0, H;
    double tau_g, tau_f, sigma[7], lam[19];
    int varchi;             /* per-phase conductivities: rates per node from f_l */
    double Minv[19][19], Ninv[7][7];
    int opp19[19], opp7[7];
    /* state */
    double *f, *g;          /* pre-collision populations */
    double *fpost, *gpost;  /* post-collision scratch */
    double *Tw[6];          /* per-face wall temperature fields */
    double *flux[6];        /* enthalpy entering through each wall link in the last stream */
    long step;
};

static char g_err[256] = "";
static void set_err(const char *m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char *orc_last_error(void) { return g_err; }

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Gauss-Jordan inversion with partial pivoting of an n x n row-major matrix. */
static int invert_matrix(int n, const double *A, double *Ainv) {
    double a[19][38];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            a[i][j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (fabs(a[piv][c]) < 1e-300) return -1;
        if (piv != c)
            for (int j = 0; j < 2 * n; j++) {
                double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t;
            }
        double d = a[c][c];
        for (int j = 0; j < 2 * n; j++) a[c][j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            double m = a[r][c];
            if (m != 0.0)
                for (int j = 0; j < 2 * n; j++) a[r][j] -= m * a[c][j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Ainv[i * n + j] = a[i][j + n];
    return 0;
}

static int find_opposite(const int (*e)[3], int q, int a) {
    for (int b = 0; b < q; b++)
        if (e[b][0] == -e[a][0] && e[b][1] == -e[a][1] && e[b][2] == -e[a][2]) return b;
    return -1;
}

/* Face of the wall crossed by the link that brings population a (velocity e) to a
 * node whose upwind neighbour x - e lies outside, or -1 if the neighbour is inside. */
static int face_of(int ex, int ey, int ez, int x, int y, int z, int nx, int ny, int nz) {
    if (ex == 1 && x == 0) return 0;
    if (ex == -1 && x == nx - 1) return 1;
    if (ey == 1 && y == 0) return 2;
    if (ey == -1 && y == ny - 1) return 3;
    if (ez == 1 && z == 0) return 4;
    if (ez == -1 && z == nz - 1) return 5;
    return -1;
}

static long face_area(const orc_state *s, int face) {
    if (face < 2) return (long)s->ny * s->nz;
    if (face < 4) return (long)s->nx * s->nz;
    return (long)s->nx * s->ny;
}

/* Position of node (x,y,z) inside the field of a face (the two in-plane coordinates). */
static long face_index(const orc_state *s, int face, int x, int y, int z) {
    if (face < 2) return y + (long)s->ny * z;
    if (face < 4) return x + (long)s->nx * z;
    return x + (long)s->nx * y;
}

/* ---- parameter mapping (Eq. 20, 34, 59, 64) ---- */
static int map_params(orc_state *s) {
    const orc_params *p = &s->p;
    if (p->omega_T <= 0.0 || p->omega_T > 1.0 / 3.0) { set_err("omega_T out of (0,1/3]"); return -1; }
    if (p->Cp_s <= 0 || p->Cp_l <= 0 || p->Cp_ref <= 0) { set_err("Cp must be > 0"); return -1; }
    if (p->St <= 0) { set_err("St must be > 0"); return -1; }
    s->dT = p->Th - p->Tm;
    if (s->dT <= 0) { set_err("Th must exceed Tm"); return -1; }
    /* Stefan number Ste = Cp dT / L (Eq. 64) fixes the latent heat. */
    s->L = p->Cp_l * s->dT / p->St;
    s->hs = p->Cp_s * p->Tm;  /* h of solid at T_m (Eq. 2 with f_l = 0, h0 = 0) */
    s->hl = s->hs + s->L;     /* h of liquid at T_m */
    s->H = (double)s->nx;     /* wall-to-wall distance: walls half a cell outside */
    s->nu = 0.0; s->gbeta = 0.0; s->U0 = 0.0;
    s->chi = 0.0;
    if (p->flow_model != ORC_FLOW_NONE) {
        if (p->Ra <= 0 || p->Pr <= 0 || p->Ma <= 0) { set_err("Ra, Pr, Ma must be > 0"); return -1; }
        /* READING: free-fall velocity U0 = sqrt(g beta dT H) = Ma c_s fixes the lattice
         * scales; Ra and Pr (Eq. 64) then give nu, chi and g beta. */
        s->U0 = p->Ma / sqrt(3.0);
        s->nu = s->U0 * s->H * sqrt(p->Pr / p->Ra);
        if (p->nu > 0) s->nu = p->nu;
        s->chi = s->nu / p->Pr;
        s->gbeta = s->U0 * s->U0 / (s->dT * s->H);
    }
    if (p->tau_g > 0) s->chi = (p->tau_g - 0.5) * p->omega_T; /* Eq. 20 */
    s->varchi = p->lambda_s > 0 || p->lambda_l > 0;
    if (s->varchi) {
        /* Per-phase conductivities (Sec. 3.1.2 case (b)).  Eq. 1 diffuses with lambda/rho0
         * and Eq. 33 with chi acting on C_p,ref T, so chi = lambda / (rho0 C_p,ref), rho0 = 1;
         * the relaxation rates then follow per node from f_l (orc_collide_node).  The
         * constants below use the solid value. */
        if (p->lambda_s <= 0 || p->lambda_l <= 0) { set_err("give both lambda_s and lambda_l"); return -1; }
        if (p->flow_model != ORC_FLOW_NONE || p->tau_g > 0) {
            set_err("per-phase conductivities need flow_model NONE and no tau_g"); return -1;
        }
        s->chi = p->lambda_s / p->Cp_ref;
    }
    if (s->chi <= 0) { set_err("thermal diffusivity undefined: give tau_g or the flow groups"); return -1; }
    /* Eq. 20 / Eq. 34: chi = (tau_g - 1/2) omega_T = (1/sigma_chi - 1/2) omega_T */
    s->tau_g = s->chi / p->omega_T + 0.5;
    double sig_chi = 1.0 / s->tau_g;
    for (int k = 0; k < 7; k++) s->sigma[k] = sig_chi;
    s->sigma[0] = 1.0; /* READING: n_0 = n_0^eq = h, so sigma_0 never acts */
    if (p->enth_model == ORC_ENTH_MRT) {
        double s4 = p->sigma4 > 0 ? p->sigma4 : 2.0 - sig_chi; /* Eq. 47 */
        s->sigma[4] = s->sigma[5] = s->sigma[6] = s4;
    } else if (p->enth_model != ORC_ENTH_SRT) { set_err("bad enth_model"); return -1; }
    for (int k = 0; k < 19; k++) s->lam[k] = 0.0;
    s->tau_f = 0.0;
    if (p->flow_model != ORC_FLOW_NONE) {
        /* Eq. 59: nu = (1/s_nu - 1/2)/3 */
        double s_nu = 1.0 / (3.0 * s->nu + 0.5);
        s->tau_f = 1.0 / s_nu;
        double se, seps, sq, spi, st;
        if (p->flow_model == ORC_FLOW_SRT) {
            se = seps = sq = spi = st = s_nu;
        } else {
            /* READING: rates not printed in Eq. 52; defaults are the D3Q19 values of the
             * paper's Ref. [20] (d'Humieres et al. 2002). */
            se = p->s_e > 0 ? p->s_e : 1.19;
            seps = p->s_eps > 0 ? p->s_eps : 1.4;
            sq = p->s_q > 0 ? p->s_q : 1.2;
            spi = p->s_pi > 0 ? p->s_pi : 1.4;
            st = p->s_t > 0 ? p->s_t : 1.98;
        }
        /* Eq. 52 */
        double lam[19] = {0, se, seps, 0, sq, 0, sq, 0, sq, s_nu, spi, s_nu, spi, s_nu, s_nu,
                          s_nu, st, st, st};
        memcpy(s->lam, lam, sizeof lam);
    } else if (p->flow_model != ORC_FLOW_NONE) { set_err("bad flow_model"); return -1; }
    for (int k = 0; k < 7; k++)
        if (!(s->sigma[k] > 0 && s->sigma[k] < 2)) { set_err("enthalpy relaxation rate outside (0,2)"); return -1; }
    for (int k = 0; k < 19; k++)
        if (s->lam[k] < 0 || s->lam[k] >= 2) { set_err("flow relaxation rate outside [0,2)"); return -1; }
    return 0;
}

/* ---- Eq. 2 inverted: h -> (T, f_l) ----
 * READING: h = C_p T + f_l L with h_s = C_p,s T_m, h_l = h_s + L; the solid branch
 * takes h <= h_s, the liquid branch h >= h_l, the mushy zone sits at T_m. */
void orc_invert(const orc_state *s, double h, double *T, double *fl) {
    const orc_params *p = &s->p;
    if (h <= s->hs) {
        *fl = 0.0;
        *T = p->Tm + (h - s->hs) / p->Cp_s;
    } else if (h >= s->hl) {
        *fl = 1.0;
        *T = p->Tm + (h - s->hl) / p->Cp_l;
    } else {
        *fl = (h - s->hs) / s->L;
        *T = p->Tm;
    }
}

/* ---- flow equilibrium moments, Eq. 53 (c = 1) ----
 * READING: element 10 prints "-u_x^2 + 0.5 u_y^2 + u_z^2"; the projection of the
 * second-order equilibrium on row 10 of M gives -u_x^2 + u_y^2/2 + u_z^2/2. */
void orc_flow_meq(double rho, const double *u, double *meq) {
    double ux = u[0], uy = u[1], uz = u[2];
    double u2 = ux * ux + uy * uy + uz * uz;
    meq[0] = rho;
    meq[1] = rho * (-11.0 + 19.0 * u2);
    meq[2] = rho * (3.0 - 11.0 * u2 / 2.0);
    meq[3] = rho * ux;
    meq[4] = rho * (-2.0 * ux / 3.0);
    meq[5] = rho * uy;
    meq[6] = rho * (-2.0 * uy / 3.0);
    meq[7] = rho * uz;
    meq[8] = rho * (-2.0 * uz / 3.0);
    meq[9] = rho * (3.0 * ux * ux - u2);
    meq[10] = rho * (-ux * ux + 0.5 * uy * uy + 0.5 * uz * uz);
    meq[11] = rho * (uy * uy - uz * uz);
    meq[12] = rho * (uz * uz - uy * uy) / 2.0;
    meq[13] = rho * ux * uy;
    meq[14] = rho * uy * uz;
    meq[15] = rho * uz * ux;
    meq[16] = meq[17] = meq[18] = 0.0;
}

/* ---- forcing moments, Eq. 54 (c = 1) ----
 * READING: element 9 prints "2 F_x u_x - 2 F.u"; the projection of the discrete
 * forcing on row 9 of M gives 6 F_x u_x - 2 F.u (element 10 is -1/2 of it as printed). */
void orc_flow_forcing(const double *F, const double *u, double *FF) {
    double Fu = F[0] * u[0] + F[1] * u[1] + F[2] * u[2];
    FF[0] = 0.0;
    FF[1] = 38.0 * Fu;
    FF[2] = -11.0 * Fu;
    FF[3] = F[0];
    FF[4] = -2.0 * F[0] / 3.0;
    FF[5] = F[1];
    FF[6] = -2.0 * F[1] / 3.0;
    FF[7] = F[2];
    FF[8] = -2.0 * F[2] / 3.0;
    FF[9] = 6.0 * F[0] * u[0] - 2.0 * Fu;
    FF[10] = Fu - 3.0 * F[0] * u[0];
    FF[11] = 2.0 * F[1] * u[1] - 2.0 * F[2] * u[2];
    FF[12] = F[2] * u[2] - F[1] * u[1];
    FF[13] = F[0] * u[1] + F[1] * u[0];
    FF[14] = F[1] * u[2] + F[2] * u[1];
    FF[15] = F[0] * u[2] + F[2] * u[0];
    FF[16] = FF[17] = FF[18] = 0.0;
}

static double local_cp(const orc_state *s, double fl) {
    /* READING: local C_p of Eq. 7 / Eq. 25 mixes the phase values by f_l. */
    return fl * s->p.Cp_l + (1.0 - fl) * s->p.Cp_s;
}

/* ---- enthalpy equilibrium, Eq. 7 with weights Eq. 8 and c_sT^2 = omega_T (c = 1) ---- */
void orc_enth_geq(const orc_state *s, double h, double T, double fl, const double *u,
                  double *geq) {
    const double wT = s->p.omega_T, Cref = s->p.Cp_ref, Cp = local_cp(s, fl);
    double w[7];
    w[0] = 1.0 - 3.0 * wT;
    for (int a = 1; a < 7; a++) w[a] = 0.5 * wT;
    const double cs2 = wT;
    geq[0] = h - (1.0 - w[0]) * Cref * T;
    for (int a = 1; a < 7; a++) {
        double eu = u[0] * E7[a][0] + u[1] * E7[a][1] + u[2] * E7[a][2];
        geq[a] = w[a] * Cref * T + eu / cs2 * w[a] * Cp * T;
    }
}

/* ---- enthalpy equilibrium moments, Eq. 25 (c = 1) ---- */
void orc_enth_neq(const orc_state *s, double h, double T, double fl, const double *u,
                  double *neq) {
    const double Cp = local_cp(s, fl);
    neq[0] = h;
    neq[1] = Cp * T * u[0];
    neq[2] = Cp * T * u[1];
    neq[3] = Cp * T * u[2];
    neq[4] = 6.0 * h - 21.0 * s->p.omega_T * s->p.Cp_ref * T;
    neq[5] = 0.0;
    neq[6] = 0.0;
}

double orc_solid_phi(const orc_params *p, double fl) {
    if (p->darcy_A <= 0) return fl;
    const double eps = p->darcy_eps > 0 ? p->darcy_eps : 1e-3;
    const double D = p->darcy_A * (1.0 - fl) * (1.0 - fl) / (fl * fl * fl + eps);
    return 1.0 / (1.0 + 0.5 * D);
}

/* ---- one node: macroscopic quantities and both collisions ----
 * macro (optional, 10 values): h, T, f_l, rho, u[3], F[3]. */
void orc_collide_node(const orc_state *s, const double *f, const double *g, double *fpost,
                      double *gpost, double *macro) {
    const orc_params *p = &s->p;
    /* 1. h = sum g (Eq. 9) */
    double h = 0.0;
    for (int a = 0; a < 7; a++) h += g[a];
    /* 2. Eq. 2 inverted */
    double T, fl;
    orc_invert(s, h, &T, &fl);
    double rho = 0.0, u[3] = {0, 0, 0}, F[3] = {0, 0, 0};
    if (p->flow_model != ORC_FLOW_NONE) {
        /* 3. rho and momentum j (Eq. 56) */
        double j[3] = {0, 0, 0};
        for (int a = 0; a < 19; a++) {
            rho += f[a];
            for (int d = 0; d < 3; d++) j[d] += f[a] * E19[a][d];
        }
        /* 4. buoyancy (Eq. 55, rho_ref = rho_0 = 1, gravity along -z) */
        const double rho0 = 1.0;
        double Fb[3] = {0.0, 0.0, s->gbeta * (T - p->Tref)};
        /* READING: solid-phase force. The flow lives in the liquid and the interface is
         * no-slip; the force -2 (1 - f_l) rho0 u* removes the fraction (1 - f_l) of
         * the velocity u* = (j + F_b/2)/rho0, so u = f_l u* and u = 0 in the solid.
         * The enthalpy-porosity alternative (not in the paper) replaces f_l by phi. */
        const double phi = orc_solid_phi(p, fl);
        double us[3], Fs[3];
        for (int d = 0; d < 3; d++) {
            us[d] = (j[d] + 0.5 * Fb[d]) / rho0;
            Fs[d] = -2.0 * (1.0 - phi) * rho0 * us[d];
            F[d] = Fb[d] + Fs[d];
            u[d] = (j[d] + 0.5 * F[d]) / rho0; /* Eq. 56 */
        }
        /* 5a. MRT collision in moment space, Eq. 49 (delta_t = 1) */
        double m[19], meq[19], FF[19], mp[19];
        for (int k = 0; k < 19; k++) {
            m[k] = 0.0;
            for (int a = 0; a < 19; a++) m[k] += MMAT[k][a] * f[a];
        }
        orc_flow_meq(rho, u, meq);
        orc_flow_forcing(F, u, FF);
        for (int k = 0; k < 19; k++)
            mp[k] = m[k] - s->lam[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s->lam[k]) * FF[k];
        /* Eq. 50: back to velocity space */
        for (int a = 0; a < 19; a++) {
            fpost[a] = 0.0;
            for (int k = 0; k < 19; k++) fpost[a] += s->Minv[a][k] * mp[k];
        }
    }
    /* 5b. enthalpy collision */
    const double *sigma = s->sigma;
    double tau_g = s->tau_g, sigma_n[7];
    if (s->varchi) {
        /* READING: the paper gives no mushy-zone rule for lambda; lambda(f_l) = lambda_s +
         * f_l (lambda_l - lambda_s), then chi = lambda / C_p,ref and Eq. 34 per node */
        const double chi_n = (p->lambda_s + fl * (p->lambda_l - p->lambda_s)) / p->Cp_ref;
        const double sc = 1.0 / (chi_n / p->omega_T + 0.5);
        for (int k = 0; k < 7; k++) sigma_n[k] = sc;
        sigma_n[0] = 1.0;
        sigma_n[4] = sigma_n[5] = sigma_n[6] = p->sigma4 > 0 ? p->sigma4 : 2.0 - sc; /* Eq. 47 */
        sigma = sigma_n;
        tau_g = 1.0 / sc;
    }
    if (p->enth_model == ORC_ENTH_SRT) {
        /* Eq. 5-7: BGK relaxation towards g^eq */
        double geq[7];
        orc_enth_geq(s, h, T, fl, u, geq);
        for (int a = 0; a < 7; a++) gpost[a] = g[a] - (g[a] - geq[a]) / tau_g;
    } else {
        /* Eq. 21-25: relaxation of the moments n = N g */
        double n[7], neq[7], np[7];
        for (int k = 0; k < 7; k++) {
            n[k] = 0.0;
            for (int a = 0; a < 7; a++) n[k] += NMAT[k][a] * g[a];
        }
        orc_enth_neq(s, h, T, fl, u, neq);
        for (int k = 0; k < 7; k++) np[k] = n[k] - sigma[k] * (n[k] - neq[k]);
        for (int a = 0; a < 7; a++) {
            gpost[a] = 0.0;
            for (int k = 0; k < 7; k++) gpost[a] += s->Ninv[a][k] * np[k];
        }
    }
    if (macro) {
        macro[0] = h; macro[1] = T; macro[2] = fl; macro[3] = rho;
        for (int d = 0; d < 3; d++) { macro[4 + d] = u[d]; macro[7 + d] = F[d]; }
    }
}

/* ---- streaming of one node (pull form of Eq. 5 / Eq. 50) with the wall rules ----
 * READING (walls; the paper names no scheme): every wall lies half a cell outside
 * the boundary nodes.  A population whose upwind neighbour x - e lies outside a
 * non-periodic face is rebuilt from the node's own post-collision populations:
 *   flow (no slip, Sec. 3.3):      f_a(x) = f*_abar(x)                  (bounce-back)
 *   enthalpy, adiabatic face:      g_a(x) = g*_abar(x)                  (bounce-back)
 *   enthalpy, isothermal face:     g_a(x) = -g*_abar(x) + omega_T C_p,ref T_w
 * (anti-bounce-back; with u = 0 at the wall only the even part of Eq. 7 remains). */
static void stream_node(const orc_state *s, const double *fpost, const double *gpost,
                        long n, double *fout, double *gout, double *flux_face) {
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const long N = s->N;
    int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
    const int *bc = s->p.bc;
    if (fout) {
        for (int a = 0; a < 19; a++) {
            int ex = E19[a][0], ey = E19[a][1], ez = E19[a][2];
            int xs = x - ex, ys = y - ey, zs = z - ez;
            int out = 0;
            if (xs < 0 || xs >= nx) { if (bc[0] == ORC_PERIODIC) xs = (xs + nx) % nx; else out = 1; }
            if (ys < 0 || ys >= ny) { if (bc[2] == ORC_PERIODIC) ys = (ys + ny) % ny; else out = 1; }
            if (zs < 0 || zs >= nz) { if (bc[4] == ORC_PERIODIC) zs = (zs + nz) % nz; else out = 1; }
            if (out)
                fout[a] = fpost[(long)s->opp19[a] * N + n];
            else
                fout[a] = fpost[(long)a * N + xs + (long)nx * (ys + (long)ny * zs)];
        }
    }
    gout[0] = gpost[n];
    for (int a = 1; a < 7; a++) {
        int ex = E7[a][0], ey = E7[a][1], ez = E7[a][2];
        int face = face_of(ex, ey, ez, x, y, z, nx, ny, nz);
        if (face >= 0 && bc[face] != ORC_PERIODIC) {
            double gb = gpost[(long)s->opp7[a] * N + n];
            if (bc[face] == ORC_ADIABATIC) {
                gout[a] = gb;
            } else {
                double Tw = s->Tw[face][face_index(s, face, x, y, z)];
                gout[a] = -gb + s->p.omega_T * s->p.Cp_ref * Tw;
            }
            if (flux_face) flux_face[face] = gout[a] - gb;
        } else {
            int xs = (x - ex + nx) % nx, ys = (y - ey + ny) % ny, zs = (z - ez + nz) % nz;
            gout[a] = gpost[(long)a * N + xs + (long)nx * (ys + (long)ny * zs)];
        }
    }
}

static void equilibrium_state(orc_state *s, const double *h0) {
    const long N = s->N;
    double feq[19], meq[19], zero[3] = {0, 0, 0};
    orc_flow_meq(1.0, zero, meq);
    for (int a = 0; a < 19; a++) {
        feq[a] = 0.0;
        for (int k = 0; k < 19; k++) feq[a] += s->Minv[a][k] * meq[k];
    }
    for (long n = 0; n < N; n++) {
        double h = h0 ? h0[n] : s->p.h0, T, fl, geq[7];
        orc_invert(s, h, &T, &fl);
        orc_enth_geq(s, h, T, fl, zero, geq);
        for (int a = 0; a < 7; a++) s->g[(long)a * N + n] = geq[a];
        if (s->f)
            for (int a = 0; a < 19; a++) s->f[(long)a * N + n] = feq[a];
    }
    for (int face = 0; face < 6; face++)
        memset(s->flux[face], 0, sizeof(double) * face_area(s, face));
    s->step = 0;
}

orc_state *orc_create(int nx, int ny, int nz, const orc_params *p, int alloc) {
    if (nx < 1 || ny < 1 || nz < 1) { set_err("lattice extents must be >= 1"); return NULL; }
    for (int ax = 0; ax < 3; ax++) {
        int lo = p->bc[2 * ax], hi = p->bc[2 * ax + 1];
        if ((lo == ORC_PERIODIC) != (hi == ORC_PERIODIC)) { set_err("periodic faces must pair"); return NULL; }
        if (lo < 0 || lo > 2 || hi < 0 || hi > 2) { set_err("bad bc code"); return NULL; }
    }
    if (p->flow_model < 0 || p->flow_model > 2) { set_err("bad flow_model"); return NULL; }
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->N = (long)nx * ny * nz;
    s->p = *p;
    if (map_params(s) != 0) { free(s); return NULL; }
    double Mf[361], Mi[361], Nf[49], Ni[49];
    for (int i = 0; i < 19; i++) for (int j = 0; j < 19; j++) Mf[i * 19 + j] = MMAT[i][j];
    for (int i = 0; i < 7; i++) for (int j = 0; j < 7; j++) Nf[i * 7 + j] = NMAT[i][j];
    if (invert_matrix(19, Mf, Mi) || invert_matrix(7, Nf, Ni)) { set_err("singular transform"); free(s); return NULL; }
    for (int i = 0; i < 19; i++) for (int j = 0; j < 19; j++) s->Minv[i][j] = Mi[i * 19 + j];
    for (int i = 0; i < 7; i++) for (int j = 0; j < 7; j++) s->Ninv[i][j] = Ni[i * 7 + j];
    for (int a = 0; a < 19; a++) s->opp19[a] = find_opposite(E19, 19, a);
    for (int a = 0; a < 7; a++) s->opp7[a] = find_opposite(E7, 7, a);
    for (int face = 0; face < 6; face++) {
        long A = face_area(s, face);
        s->Tw[face] = (double *)malloc(sizeof(double) * A);
        s->flux[face] = (double *)calloc(A, sizeof(double));
        for (long i = 0; i < A; i++) s->Tw[face][i] = p->T_wall[face];
    }
    if (alloc) {
        s->g = (double *)malloc(sizeof(double) * 7 * s->N);
        s->gpost = (double *)malloc(sizeof(double) * 7 * s->N);
        if (p->flow_model != ORC_FLOW_NONE) {
            s->f = (double *)malloc(sizeof(double) * 19 * s->N);
            s->fpost = (double *)malloc(sizeof(double) * 19 * s->N);
        }
        equilibrium_state(s, NULL);
    }
    return s;
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free(s->f); free(s->g); free(s->fpost); free(s->gpost);
    for (int face = 0; face < 6; face++) { free(s->Tw[face]); free(s->flux[face]); }
    free(s);
}

int orc_set_initial_h(orc_state *s, const double *h) {
    if (!s->g) { set_err("context has no lattice arrays"); return -1; }
    equilibrium_state(s, h);
    return 0;
}

int orc_set_wall_temperature(orc_state *s, int face, const double *T) {
    if (face < 0 || face > 5) { set_err("bad face"); return -1; }
    memcpy(s->Tw[face], T, sizeof(double) * face_area(s, face));
    return 0;
}

int orc_set_distributions(orc_state *s, const double *f, const double *g) {
    if (!s->g) { set_err("context has no lattice arrays"); return -1; }
    memcpy(s->g, g, sizeof(double) * 7 * s->N);
    if (s->f && f) memcpy(s->f, f, sizeof(double) * 19 * s->N);
    return 0;
}

void orc_step(orc_state *s, int nsteps) {
    const long N = s->N;
    const int flow = s->p.flow_model != ORC_FLOW_NONE;
    for (int it = 0; it < nsteps; it++) {
        /* steps 1-5: per-node macroscopics and collision */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; n++) {
            double f[19], g[7], fp[19], gp[7];
            for (int a = 0; a < 7; a++) g[a] = s->g[(long)a * N + n];
            if (flow)
                for (int a = 0; a < 19; a++) f[a] = s->f[(long)a * N + n];
            orc_collide_node(s, f, g, fp, gp, NULL);
            for (int a = 0; a < 7; a++) s->gpost[(long)a * N + n] = gp[a];
            if (flow)
                for (int a = 0; a < 19; a++) s->fpost[(long)a * N + n] = fp[a];
        }
        /* step 6: streaming with the wall rules */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; n++) {
            double fo[19], go[7], fl[6];
            for (int k = 0; k < 6; k++) fl[k] = NAN;
            stream_node(s, s->fpost, s->gpost, n, flow ? fo : NULL, go, fl);
            for (int a = 0; a < 7; a++) s->g[(long)a * N + n] = go[a];
            if (flow)
                for (int a = 0; a < 19; a++) s->f[(long)a * N + n] = fo[a];
            int x = (int)(n % s->nx), y = (int)((n / s->nx) % s->ny), z = (int)(n / ((long)s->nx * s->ny));
            for (int face = 0; face < 6; face++)
                if (!isnan(fl[face])) s->flux[face][face_index(s, face, x, y, z)] = fl[face];
        }
        s->step++;
    }
}

void orc_fields(const orc_state *s, double *T, double *fl, double *h, double *rho, double *u) {
    const long N = s->N;
    const int flow = s->p.flow_model != ORC_FLOW_NONE;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double f[19], g[7], fp[19], gp[7], mac[10];
        for (int a = 0; a < 7; a++) g[a] = s->g[(long)a * N + n];
        if (flow)
            for (int a = 0; a < 19; a++) f[a] = s->f[(long)a * N + n];
        orc_collide_node(s, f, g, fp, gp, mac);
        if (h) h[n] = mac[0];
        if (T) T[n] = mac[1];
        if (fl) fl[n] = mac[2];
        if (rho) rho[n] = mac[3];
        if (u) for (int d = 0; d < 3; d++) u[(long)d * N + n] = mac[4 + d];
    }
}

void orc_distributions(const orc_state *s, double *f, double *g) {
    if (g) memcpy(g, s->g, sizeof(double) * 7 * s->N);
    if (f && s->f) memcpy(f, s->f, sizeof(double) * 19 * s->N);
}

void orc_wall_flux(const orc_state *s, int face, double *q) {
    memcpy(q, s->flux[face], sizeof(double) * face_area(s, face));
}

long orc_step_count(const orc_state *s) { return s->step; }

void orc_lattice(const orc_state *s, double *out) {
    out[ORC_L_CHI] = s->chi;
    out[ORC_L_NU] = s->nu;
    out[ORC_L_GBETA] = s->gbeta;
    out[ORC_L_SIGMA_CHI] = s->sigma[1];
    out[ORC_L_SIGMA4] = s->sigma[4];
    out[ORC_L_S_NU] = s->lam[9];
    out[ORC_L_LATENT] = s->L;
    out[ORC_L_HS] = s->hs;
    out[ORC_L_HL] = s->hl;
    out[ORC_L_TAU_G] = s->tau_g;
    out[ORC_L_TAU_F] = s->tau_f;
    out[ORC_L_S_E] = s->lam[1];
    out[ORC_L_S_EPS] = s->lam[2];
    out[ORC_L_S_Q] = s->lam[4];
    out[ORC_L_S_PI] = s->lam[10];
    out[ORC_L_S_T] = s->lam[16];
    out[ORC_L_U0] = s->U0;
}

/* Diagnostics of the current state (Sec. 3.2.2 / 3.3 quantities), FP64.
 * READING (3D form of Eq. 65): Nu = H / (chi C_p,ref dT) times the wall average of
 * the enthalpy entering per step through the -x wall links.  Nu_fd uses the
 * one-sided difference (T_w - T(0)) / (1/2).  FRONT_MEAN is the melted volume per
 * unit wall area; FRONT_MID is the first f_l = 1/2 crossing along x on the lines
 * y = ny/2, z in {nz/4, nz/2, 3nz/4}, measured from the wall at x = -1/2. */
void orc_diagnostics(const orc_state *s, double *out) {
    const long N = s->N;
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    double *T = (double *)malloc(sizeof(double) * N), *fl = (double *)malloc(sizeof(double) * N);
    double *h = (double *)malloc(sizeof(double) * N), *rho = (double *)malloc(sizeof(double) * N);
    orc_fields(s, T, fl, h, rho, NULL);
    double sfl = 0, sh = 0, srho = 0, nan = 0;
    for (long n = 0; n < N; n++) {
        sfl += fl[n]; sh += h[n]; srho += rho[n];
        if (!isfinite(h[n]) || !isfinite(rho[n])) nan += 1;
    }
    double A = (double)ny * nz;
    double q = 0, dtw = 0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++) {
            long fi = y + (long)ny * z;
            q += s->flux[0][fi];
            dtw += (s->Tw[0][fi] - T[(long)nx * (y + (long)ny * z)]) / 0.5;
        }
    double scale = s->H / (s->chi * s->p.Cp_ref * s->dT);
    double front_mid = 0;
    int zs[3] = {nz / 4, nz / 2, (3 * nz) / 4}, yl = ny / 2;
    for (int k = 0; k < 3; k++) {
        double xc = nx; /* no crossing: fully melted line */
        for (int x = 0; x < nx; x++) {
            double v = fl[x + (long)nx * (yl + (long)ny * zs[k])];
            if (v < 0.5) {
                if (x == 0) { xc = -0.5; break; }
                double vp = fl[x - 1 + (long)nx * (yl + (long)ny * zs[k])];
                xc = (x - 1) + (vp - 0.5) / (vp - v);
                break;
            }
        }
        front_mid += (xc + 0.5) / 3.0;
    }
    out[ORC_D_LIQUID_VOL] = sfl;
    out[ORC_D_NU_HOT] = scale * q / A;
    out[ORC_D_FRONT_MEAN] = sfl / A;
    out[ORC_D_SUM_H] = sh;
    out[ORC_D_SUM_RHO] = s->p.flow_model != ORC_FLOW_NONE ? srho : 0.0;
    out[ORC_D_STEP] = (double)s->step;
    out[ORC_D_NU_FD] = s->H / s->dT * dtw / A;
    out[ORC_D_FRONT_MID] = front_mid;
    out[ORC_D_NAN] = nan;
    free(T); free(fl); free(h); free(rho);
}

void orc_update_sampled(const orc_state *s, const double *f, const double *g, long ns,
                        const long *idx, double *fo, double *go) {
    const long N = s->N;
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const int flow = s->p.flow_model != ORC_FLOW_NONE;
    const int *bc = s->p.bc;
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < ns; k++) {
        long n = idx[k];
        int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
        double fn[19], gn[7], fp[19], gp[7];
        /* collide node m and return its post-collision populations */
#define COLLIDE_AT(m)                                                                   \
    do {                                                                                \
        for (int b = 0; b < 7; b++) gn[b] = g[(long)b * N + (m)];                       \
        if (flow) for (int b = 0; b < 19; b++) fn[b] = f[(long)b * N + (m)];            \
        orc_collide_node(s, fn, gn, fp, gp, NULL);                                      \
    } while (0)
        if (flow) {
            for (int a = 0; a < 19; a++) {
                int xs = x - E19[a][0], ys = y - E19[a][1], zs = z - E19[a][2], out = 0;
                if (xs < 0 || xs >= nx) { if (bc[0] == ORC_PERIODIC) xs = (xs + nx) % nx; else out = 1; }
                if (ys < 0 || ys >= ny) { if (bc[2] == ORC_PERIODIC) ys = (ys + ny) % ny; else out = 1; }
                if (zs < 0 || zs >= nz) { if (bc[4] == ORC_PERIODIC) zs = (zs + nz) % nz; else out = 1; }
                if (out) { COLLIDE_AT(n); fo[k * 19 + a] = fp[s->opp19[a]]; }
                else { COLLIDE_AT(xs + (long)nx * (ys + (long)ny * zs)); fo[k * 19 + a] = fp[a]; }
            }
        }
        COLLIDE_AT(n);
        go[k * 7] = gp[0];
        for (int a = 1; a < 7; a++) {
            int ex = E7[a][0], ey = E7[a][1], ez = E7[a][2];
            int face = face_of(ex, ey, ez, x, y, z, nx, ny, nz);
            if (face >= 0 && bc[face] != ORC_PERIODIC) {
                COLLIDE_AT(n);
                double gb = gp[s->opp7[a]];
                if (bc[face] == ORC_ADIABATIC) go[k * 7 + a] = gb;
                else go[k * 7 + a] = -gb + s->p.omega_T * s->p.Cp_ref * s->Tw[face][face_index(s, face, x, y, z)];
            } else {
                int xs = (x - ex + nx) % nx, ys = (y - ey + ny) % ny, zs = (z - ez + nz) % nz;
                COLLIDE_AT(xs + (long)nx * (ys + (long)ny * zs));
                go[k * 7 + a] = gp[a];
            }
        }
#undef COLLIDE_AT
    }
}

void orc_tables(double *M, double *Minv, double *N, double *Ninv, int *e19, int *e7) {
    double Mi[361], Ni[49], Mf[361], Nf[49];
    for (int i = 0; i < 19; i++) for (int j = 0; j < 19; j++) Mf[i * 19 + j] = MMAT[i][j];
    for (int i = 0; i < 7; i++) for (int j = 0; j < 7; j++) Nf[i * 7 + j] = NMAT[i][j];
    invert_matrix(19, Mf, Mi);
    invert_matrix(7, Nf, Ni);
    if (M) memcpy(M, Mf, sizeof Mf);
    if (Minv) memcpy(Minv, Mi, sizeof Mi);
    if (N) memcpy(N, Nf, sizeof Nf);
    if (Ninv) memcpy(Ninv, Ni, sizeof Ni);
    if (e19) for (int a = 0; a < 19; a++) for (int d = 0; d < 3; d++) e19[a * 3 + d] = E19[a][d];
    if (e7) for (int a = 0; a < 7; a++) for (int d = 0; d < 3; d++) e7[a * 3 + d] = E7[a][d];
}

/* ---- read-only views for lbpc_oracle_adjoint.c ---- */
int orc__dims(const orc_state *s, int *nx, int *ny, int *nz) {
    *nx = s->nx; *ny = s->ny; *nz = s->nz;
    return 0;
}
const orc_params *orc__params(const orc_state *s) { return &s->p; }
void orc__lattice_raw(const orc_state *s, double *L, double *hs, double *gbeta, double *sigma,
                      double *lam, const double **Minv, const double **Ninv, const int **opp19,
                      const int **opp7, const double *const **Tw) {
    *L = s->L; *hs = s->hs; *gbeta = s->gbeta;
    memcpy(sigma, s->sigma, sizeof s->sigma);
    memcpy(lam, s->lam, sizeof s->lam);
    *Minv = &s->Minv[0][0]; *Ninv = &s->Ninv[0][0];
    *opp19 = s->opp19; *opp7 = s->opp7;
    *Tw = (const double *const *)s->Tw;
}
double *orc__pop(orc_state *s, int which) { return which == 0 ? s->f : s->g; }
