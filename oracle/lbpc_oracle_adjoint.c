/*
 * lbpc_oracle_adjoint.c -- FP64 CPU reference adjoint of the coupled step (oracle part).
 *
 * TEST INFRASTRUCTURE ONLY (see lbpc_oracle.h).
 *
 * Objective: J = sum over nodes of f_l(h_N), the liquid volume after N steps from the
 * state held when orc_adjoint is called (that state is a fixed input).  Gradients with
 * respect to the per-node temperature field of one isothermal face and to the Stefan
 * number St (which enters only through L = C_p,l dT / St).
 *
 * Method: the whole forward trajectory is kept (tiny lattices only).  Going backwards,
 * the transposed stream moves each adjoint population to the post-collision slot it
 * was streamed from (bounce-back: the node's own opposite slot; anti-bounce-back: the
 * same with a minus sign, plus omega_T C_p,ref times the adjoint into dJ/dT_w).  The
 * transposed collision of every node uses the node's exact Jacobian, obtained by
 * complex-step differentiation (Im C(s + i eps e_k) / eps, eps = 1e-30) of a
 * complex-valued restatement of the collision of lbpc_oracle.c (Eq. 2, 7, 21-25,
 * 49-56).  Branches of the Eq. 2 inversion are taken on the real part: the derivative
 * is that of the branch the forward took.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbpc_oracle.h"

typedef double complex cplx;

/* Read-only views of oracle state needed here (kept in sync with lbpc_oracle.c). */
int orc__dims(const orc_state *s, int *nx, int *ny, int *nz);
const orc_params *orc__params(const orc_state *s);
void orc__lattice_raw(const orc_state *s, double *L, double *hs, double *gbeta, double *sigma,
                      double *lam, const double **Minv, const double **Ninv, const int **opp19,
                      const int **opp7, const double *const **Tw);
double *orc__pop(orc_state *s, int which); /* 0: f, 1: g */

static const int E7c[7][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const int E19c[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, 1, 0}, {1, -1, 0},  {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1},
    {-1, 0, -1}, {0, 1, 1}, {0, -1, 1},  {0, 1, -1},  {0, -1, -1}};

/* Complex restatement of the node collision (same equations and order as
 * orc_collide_node); L is complex so that dC/dL comes out of the same evaluation. */
static void collide_cs(const orc_state *s, const cplx *f, const cplx *g, cplx L, cplx *fp,
                       cplx *gp) {
    const orc_params *p = orc__params(s);
    double Lr, hs, gbeta, sigma[7], lam[19];
    const double *Minv, *Ninv;
    const int *o19, *o7;
    const double *const *Tw;
    orc__lattice_raw(s, &Lr, &hs, &gbeta, sigma, lam, &Minv, &Ninv, &o19, &o7, &Tw);
    (void)Lr;
    static const double M[19][19] = {
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
    static const double N[7][7] = {
        {1, 1, 1, 1, 1, 1, 1},   {0, 1, -1, 0, 0, 0, 0},     {0, 0, 0, 1, -1, 0, 0},
        {0, 0, 0, 0, 0, 1, -1},  {6, -1, -1, -1, -1, -1, -1}, {0, 2, 2, -1, -1, -1, -1},
        {0, 0, 0, 1, 1, -1, -1}};
    /* h and Eq. 2 inverted (branch from the real part) */
    cplx h = 0;
    for (int a = 0; a < 7; a++) h += g[a];
    cplx T, fl;
    const double hr = creal(h);
    if (hr <= hs) { fl = 0; T = p->Tm + (h - hs) / p->Cp_s; }
    else if (hr >= hs + creal(L)) { fl = 1; T = p->Tm + (h - (hs + L)) / p->Cp_l; }
    else { fl = (h - hs) / L; T = p->Tm; }
    cplx u[3] = {0, 0, 0};
    if (p->flow_model != ORC_FLOW_NONE) {
        cplx rho = 0, j[3] = {0, 0, 0};
        for (int a = 0; a < 19; a++) {
            rho += f[a];
            for (int d = 0; d < 3; d++) j[d] += f[a] * E19c[a][d];
        }
        cplx Fb[3] = {0, 0, gbeta * (T - p->Tref)}, F[3];
        cplx phi = fl;  /* orc_solid_phi, in complex arithmetic */
        if (p->darcy_A > 0) {
            const double eps = p->darcy_eps > 0 ? p->darcy_eps : 1e-3;
            const cplx D = p->darcy_A * (1.0 - fl) * (1.0 - fl) / (fl * fl * fl + eps);
            phi = 1.0 / (1.0 + 0.5 * D);
        }
        for (int d = 0; d < 3; d++) {
            cplx us = j[d] + 0.5 * Fb[d];
            F[d] = Fb[d] - 2.0 * (1.0 - phi) * us;
            u[d] = j[d] + 0.5 * F[d];
        }
        cplx ux = u[0], uy = u[1], uz = u[2], u2 = ux * ux + uy * uy + uz * uz;
        cplx meq[19] = {rho, rho * (-11.0 + 19.0 * u2), rho * (3.0 - 11.0 * u2 / 2.0),
                        rho * ux, rho * (-2.0 * ux / 3.0), rho * uy, rho * (-2.0 * uy / 3.0),
                        rho * uz, rho * (-2.0 * uz / 3.0), rho * (3.0 * ux * ux - u2),
                        rho * (-ux * ux + 0.5 * uy * uy + 0.5 * uz * uz), rho * (uy * uy - uz * uz),
                        rho * (uz * uz - uy * uy) / 2.0, rho * ux * uy, rho * uy * uz, rho * uz * ux,
                        0, 0, 0};
        cplx Fu = F[0] * ux + F[1] * uy + F[2] * uz;
        cplx FF[19] = {0, 38.0 * Fu, -11.0 * Fu, F[0], -2.0 * F[0] / 3.0, F[1], -2.0 * F[1] / 3.0,
                       F[2], -2.0 * F[2] / 3.0, 6.0 * F[0] * ux - 2.0 * Fu, Fu - 3.0 * F[0] * ux,
                       2.0 * F[1] * uy - 2.0 * F[2] * uz, F[2] * uz - F[1] * uy,
                       F[0] * uy + F[1] * ux, F[1] * uz + F[2] * uy, F[0] * uz + F[2] * ux, 0, 0, 0};
        cplx mp[19];
        for (int k = 0; k < 19; k++) {
            cplx m = 0;
            for (int a = 0; a < 19; a++) m += M[k][a] * f[a];
            mp[k] = m - lam[k] * (m - meq[k]) + (1.0 - 0.5 * lam[k]) * FF[k];
        }
        for (int a = 0; a < 19; a++) {
            fp[a] = 0;
            for (int k = 0; k < 19; k++) fp[a] += Minv[a * 19 + k] * mp[k];
        }
    }
    const double wT = p->omega_T, Cref = p->Cp_ref;
    cplx Cp = fl * p->Cp_l + (1.0 - fl) * p->Cp_s;
    if (p->enth_model == ORC_ENTH_SRT) {
        const double tau = 1.0 / sigma[1];
        cplx geq[7];
        geq[0] = h - (3.0 * wT) * Cref * T;
        for (int a = 1; a < 7; a++) {
            cplx eu = u[0] * E7c[a][0] + u[1] * E7c[a][1] + u[2] * E7c[a][2];
            geq[a] = 0.5 * wT * Cref * T + eu / wT * (0.5 * wT) * Cp * T;
        }
        for (int a = 0; a < 7; a++) gp[a] = g[a] - (g[a] - geq[a]) / tau;
    } else {
        cplx n[7], neq[7] = {h, Cp * T * u[0], Cp * T * u[1], Cp * T * u[2],
                             6.0 * h - 21.0 * wT * Cref * T, 0, 0};
        for (int k = 0; k < 7; k++) {
            n[k] = 0;
            for (int a = 0; a < 7; a++) n[k] += N[k][a] * g[a];
            n[k] = n[k] - sigma[k] * (n[k] - neq[k]);
        }
        for (int a = 0; a < 7; a++) {
            gp[a] = 0;
            for (int k = 0; k < 7; k++) gp[a] += Ninv[a * 7 + k] * n[k];
        }
    }
}

/* Jacobian of the node collision: J[o][i] = d out_o / d in_i with in/out ordered
 * (f_0..f_18, g_0..g_6), and dL[o] = d out_o / dL.  nin = 26 with flow, 7 without. */
void orc_collide_jacobian(const orc_state *s, const double *f, const double *g, double *J,
                          double *dL) {
    const orc_params *p = orc__params(s);
    double Lr, hs, gbeta, sigma[7], lam[19];
    const double *Minv, *Ninv;
    const int *o19, *o7;
    const double *const *Tw;
    orc__lattice_raw(s, &Lr, &hs, &gbeta, sigma, lam, &Minv, &Ninv, &o19, &o7, &Tw);
    const int flow = p->flow_model != ORC_FLOW_NONE;
    const int nf = flow ? 19 : 0, n = nf + 7;
    const double eps = 1e-30;
    cplx fc[19], gc[7], fp[19], gp[7];
    for (int k = 0; k <= n; k++) { /* k == n: perturb L */
        for (int a = 0; a < 19; a++) fc[a] = flow ? f[a] : 0.0;
        for (int a = 0; a < 7; a++) gc[a] = g[a];
        cplx L = Lr;
        if (k < nf) fc[k] += I * eps;
        else if (k < n) gc[k - nf] += I * eps;
        else L += I * eps;
        collide_cs(s, fc, gc, L, fp, gp);
        for (int o = 0; o < n; o++) {
            cplx v = o < nf ? fp[o] : gp[o - nf];
            double d = cimag(v) / eps;
            if (k < n) J[o * n + k] = d;
            else dL[o] = d;
        }
    }
}

/* d f_l / dh and d f_l / dL of Eq. 2 inverted at h (branch of the forward). */
static void dfl(const orc_state *s, double h, double *dh, double *dLv) {
    double Lr, hs, gbeta, sigma[7], lam[19];
    const double *Minv, *Ninv;
    const int *o19, *o7;
    const double *const *Tw;
    orc__lattice_raw(s, &Lr, &hs, &gbeta, sigma, lam, &Minv, &Ninv, &o19, &o7, &Tw);
    if (h <= hs || h >= hs + Lr) { *dh = 0; *dLv = 0; }
    else { *dh = 1.0 / Lr; *dLv = -(h - hs) / (Lr * Lr); }
}

static int face_of_c(int ex, int ey, int ez, int x, int y, int z, int nx, int ny, int nz) {
    if (ex == 1 && x == 0) return 0;
    if (ex == -1 && x == nx - 1) return 1;
    if (ey == 1 && y == 0) return 2;
    if (ey == -1 && y == ny - 1) return 3;
    if (ez == 1 && z == 0) return 4;
    if (ez == -1 && z == nz - 1) return 5;
    return -1;
}

static long face_index_c(int face, int x, int y, int z, int nx, int ny) {
    if (face < 2) return y + (long)ny * z;
    if (face < 4) return x + (long)nx * z;
    return x + (long)nx * y;
}

int orc_adjoint(orc_state *s, int nsteps, int wface, double *J_out, double *dJ_dTw,
                double *dJ_dSt) {
    int nx, ny, nz;
    orc__dims(s, &nx, &ny, &nz);
    const long NN = (long)nx * ny * nz;
    const orc_params *p = orc__params(s);
    /* the node Jacobians below use the constant relaxation rates */
    if (p->lambda_s > 0 || p->lambda_l > 0) return -1;
    const int flow = p->flow_model != ORC_FLOW_NONE;
    const int nf = flow ? 19 : 0, nv = nf + 7;
    double Lr, hs, gbeta, sigma[7], lam[19];
    const double *Minv, *Ninv;
    const int *o19, *o7;
    const double *const *Tw;
    orc__lattice_raw(s, &Lr, &hs, &gbeta, sigma, lam, &Minv, &Ninv, &o19, &o7, &Tw);
    /* forward, keeping every pre-collision state (node-major: state[t][n][v]) */
    double *traj = (double *)malloc(sizeof(double) * (size_t)(nsteps + 1) * NN * nv);
    if (!traj) return -1;
    for (int t = 0; t <= nsteps; t++) {
        double *f = orc__pop(s, 0), *g = orc__pop(s, 1);
        for (long n = 0; n < NN; n++) {
            double *dst = traj + ((size_t)t * NN + n) * nv;
            for (int a = 0; a < nf; a++) dst[a] = f[(long)a * NN + n];
            for (int a = 0; a < 7; a++) dst[nf + a] = g[(long)a * NN + n];
        }
        if (t < nsteps) orc_step(s, 1);
    }
    /* seed: J = sum f_l(h_N) */
    double *lam_pre = (double *)calloc((size_t)NN * nv, sizeof(double));
    double *lam_post = (double *)calloc((size_t)NN * nv, sizeof(double));
    double J = 0.0, dJdL = 0.0;
    for (long n = 0; n < NN; n++) {
        const double *st = traj + ((size_t)nsteps * NN + n) * nv;
        double h = 0;
        for (int a = 0; a < 7; a++) h += st[nf + a];
        double T, fl, dh, dLv;
        orc_invert(s, h, &T, &fl);
        J += fl;
        dfl(s, h, &dh, &dLv);
        for (int a = 0; a < 7; a++) lam_pre[n * nv + nf + a] = dh;
        dJdL += dLv;
    }
    long wA = wface < 2 ? (long)ny * nz : (wface < 4 ? (long)nx * nz : (long)nx * ny);
    for (long i = 0; i < wA; i++) dJ_dTw[i] = 0.0;
    const double wTC = p->omega_T * p->Cp_ref;
    double *Jac = (double *)malloc(sizeof(double) * nv * nv), dL[26];
    for (int t = nsteps - 1; t >= 0; t--) {
        /* transposed stream: adjoint of the post-collision state at t */
        for (long n = 0; n < NN; n++) {
            int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
            for (int a = 0; a < nf; a++) {
                int xd = x + E19c[a][0], yd = y + E19c[a][1], zd = z + E19c[a][2], out = 0;
                if (xd < 0 || xd >= nx) { if (p->bc[0] == ORC_PERIODIC) xd = (xd + nx) % nx; else out = 1; }
                if (yd < 0 || yd >= ny) { if (p->bc[2] == ORC_PERIODIC) yd = (yd + ny) % ny; else out = 1; }
                if (zd < 0 || zd >= nz) { if (p->bc[4] == ORC_PERIODIC) zd = (zd + nz) % nz; else out = 1; }
                lam_post[n * nv + a] = out ? lam_pre[n * nv + o19[a]]
                                           : lam_pre[(xd + (long)nx * (yd + (long)ny * zd)) * nv + a];
            }
            lam_post[n * nv + nf] = lam_pre[n * nv + nf];
            for (int a = 1; a < 7; a++) {
                /* post-collision g*_a(n) feeds node n + e_a, or (wall) the node's own abar */
                int ab = o7[a];
                int face = face_of_c(E7c[ab][0], E7c[ab][1], E7c[ab][2], x, y, z, nx, ny, nz);
                if (face >= 0 && p->bc[face] != ORC_PERIODIC) {
                    double la = lam_pre[n * nv + nf + ab];
                    if (p->bc[face] == ORC_ISOTHERMAL) {
                        lam_post[n * nv + nf + a] = -la;
                        if (face == wface) dJ_dTw[face_index_c(face, x, y, z, nx, ny)] += wTC * la;
                    } else {
                        lam_post[n * nv + nf + a] = la;
                    }
                } else {
                    int xd = (x + E7c[a][0] + nx) % nx, yd = (y + E7c[a][1] + ny) % ny,
                        zd = (z + E7c[a][2] + nz) % nz;
                    lam_post[n * nv + nf + a] =
                        lam_pre[(xd + (long)nx * (yd + (long)ny * zd)) * nv + nf + a];
                }
            }
        }
        /* transposed collision with the Jacobian of the state at t */
        for (long n = 0; n < NN; n++) {
            const double *st = traj + ((size_t)t * NN + n) * nv;
            double fz[19] = {0};
            if (flow) memcpy(fz, st, sizeof(double) * 19);
            orc_collide_jacobian(s, fz, st + nf, Jac, dL);
            for (int i = 0; i < nv; i++) {
                double acc = 0.0;
                for (int o = 0; o < nv; o++) acc += Jac[o * nv + i] * lam_post[n * nv + o];
                lam_pre[n * nv + i] = acc;
            }
            for (int o = 0; o < nv; o++) dJdL += dL[o] * lam_post[n * nv + o];
        }
    }
    *J_out = J;
    /* L = C_p,l dT / St */
    const double dT = p->Th - p->Tm;
    *dJ_dSt = dJdL * (-p->Cp_l * dT / (p->St * p->St));
    free(Jac);
    free(lam_pre);
    free(lam_post);
    free(traj);
    return 0;
}
