/*
 * lbpc_oracle.h -- plain FP64 CPU oracle of the coupled flow + enthalpy lattice
 * Boltzmann step for 3D solid-liquid phase change (Li & He, "Three-dimensional
 * lattice Boltzmann models for solid-liquid phase change", Sec. 2.2-2.5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the package's smoke() check and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path; the CUDA path never
 * calls it.  Every function follows the paper's equations in the paper's order
 * with dense 19x19 / 7x7 moment transforms, no fusion and no blocking.
 *
 * Layout: node index n = x + nx*(y + ny*z); population a of node n at a*N + n.
 * The held state is the PRE-collision state (f, g) at the current time.
 */
#ifndef LBPC_ORACLE_H
#define LBPC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_ISOTHERMAL = 1, ORC_ADIABATIC = 2 };
enum { ORC_FLOW_NONE = 0, ORC_FLOW_MRT = 1, ORC_FLOW_SRT = 2 };
enum { ORC_ENTH_MRT = 1, ORC_ENTH_SRT = 2 };

/* Physical inputs and overrides (same meaning as the library's parameter block). */
typedef struct orc_params {
    int flow_model;        /* ORC_FLOW_* */
    int enth_model;        /* ORC_ENTH_* */
    int bc[6];             /* faces -x,+x,-y,+y,-z,+z */
    double T_wall[6];      /* uniform wall temperature of ISOTHERMAL faces */
    double Ra, Pr, St, Ma; /* Eq. 64 groups and the free-fall Mach number */
    double Th, Tm, Tref;   /* hot wall / melting / buoyancy reference temperature */
    double Cp_s, Cp_l, Cp_ref, omega_T;
    double tau_g;          /* > 0: SRT relaxation time of g, overrides the Pr mapping */
    double nu;             /* > 0: lattice viscosity, overrides the Ra/Pr mapping */
    double s_e, s_eps, s_q, s_pi, s_t; /* flow non-hydrodynamic rates (<= 0: default) */
    double sigma4;         /* <= 0: sigma4 = sigma5 = sigma6 = 2 - sigma_chi (Eq. 47) */
    double h0;             /* uniform initial enthalpy */
    double lambda_s, lambda_l; /* both > 0: per-phase conductivities (Eq. 1), conduction only */
    double darcy_A, darcy_eps; /* darcy_A > 0: enthalpy-porosity solid drag instead of the
                                  liquid-fraction closure (darcy_eps <= 0: 1e-3) */
} orc_params;

/* Velocity factor of the solid-phase closure: u = phi u*, F_s = -2 (1 - phi) rho0 u*.
 * phi = f_l (the liquid-fraction closure), or, with darcy_A > 0, the drag F_s = -D rho0 u
 * with D = A (1 - f_l)^2 / (f_l^3 + eps) solved together with u = u* + F_s / (2 rho0):
 * phi = 1 / (1 + D / 2). */
double orc_solid_phi(const orc_params *p, double fl);

typedef struct orc_state orc_state;

/* Derived lattice constants, indices of orc_lattice(). */
enum {
    ORC_L_CHI = 0, ORC_L_NU, ORC_L_GBETA, ORC_L_SIGMA_CHI, ORC_L_SIGMA4, ORC_L_S_NU,
    ORC_L_LATENT, ORC_L_HS, ORC_L_HL, ORC_L_TAU_G, ORC_L_TAU_F, ORC_L_S_E, ORC_L_S_EPS,
    ORC_L_S_Q, ORC_L_S_PI, ORC_L_S_T, ORC_L_U0, ORC_L_COUNT
};

/* Diagnostics, indices of orc_diagnostics(). */
enum {
    ORC_D_LIQUID_VOL = 0, ORC_D_NU_HOT, ORC_D_FRONT_MEAN, ORC_D_SUM_H, ORC_D_SUM_RHO,
    ORC_D_STEP, ORC_D_NU_FD, ORC_D_FRONT_MID, ORC_D_NAN, ORC_D_COUNT
};

/* alloc = 0 creates a constants-only context (no lattice arrays) for the node-level
 * functions and for orc_update_sampled.  Returns NULL on invalid input. */
orc_state *orc_create(int nx, int ny, int nz, const orc_params *p, int alloc);
void orc_destroy(orc_state *s);
const char *orc_last_error(void);
void orc_set_threads(int n);
int orc_threads(void);

int orc_set_initial_h(orc_state *s, const double *h);           /* N values, resets t = 0 */
int orc_set_wall_temperature(orc_state *s, int face, const double *T); /* face-area field */
int orc_set_distributions(orc_state *s, const double *f, const double *g); /* 19N, 7N */
void orc_step(orc_state *s, int nsteps);
void orc_fields(const orc_state *s, double *T, double *fl, double *h, double *rho, double *u);
void orc_distributions(const orc_state *s, double *f, double *g);
void orc_diagnostics(const orc_state *s, double *out);
void orc_lattice(const orc_state *s, double *out);
void orc_wall_flux(const orc_state *s, int face, double *q);
long orc_step_count(const orc_state *s);

/* One-step update of selected nodes from a full pre-collision state (f: 19N, g: 7N)
 * of the context's lattice; writes the new pre-collision populations of each
 * selected node to fo[k*19 + a] and go[k*7 + a]. */
void orc_update_sampled(const orc_state *s, const double *f, const double *g, long ns,
                        const long *idx, double *fo, double *go);

/* Tables and node-level operations, exposed for the pinning tests. */
void orc_tables(double *M, double *Minv, double *N, double *Ninv, int *e19, int *e7);
void orc_invert(const orc_state *s, double h, double *T, double *fl);
void orc_flow_meq(double rho, const double *u, double *meq);
void orc_flow_forcing(const double *F, const double *u, double *FF);
void orc_enth_geq(const orc_state *s, double h, double T, double fl, const double *u,
                  double *geq);
void orc_enth_neq(const orc_state *s, double h, double T, double fl, const double *u,
                  double *neq);
void orc_collide_node(const orc_state *s, const double *f, const double *g, double *fpost,
                      double *gpost, double *macro);

/* Reference adjoint (lbpc_oracle_adjoint.c).  Runs nsteps forward from the current
 * state (advancing it), returns J = sum f_l(h_N), dJ/dT_w for the wall field of `face`
 * (face-area values) and dJ/dSt.  The state at the call is held fixed. */
int orc_adjoint(orc_state *s, int nsteps, int face, double *J, double *dJ_dTw, double *dJ_dSt);
/* Exact Jacobian of the node collision by complex step: J[o*n + i], n = 26 with flow
 * (f_0..18, g_0..6) or 7 without; dL[o] = d out_o / dL. */
void orc_collide_jacobian(const orc_state *s, const double *f, const double *g, double *J,
                          double *dL);

#ifdef __cplusplus
}
#endif
#endif
