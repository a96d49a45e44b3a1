/*
 * lbpc.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for 3D solid-liquid
 * phase change after Li & He, "Three-dimensional lattice Boltzmann models for
 * solid-liquid phase change" (enthalpy-based D3Q7 SRT / MRT model, Sec. 2.2-2.4,
 * coupled with the D3Q19 MRT flow model of Sec. 2.5).
 *
 * One time step over every lattice node (the hot path) is:
 *   pull-stream f (19 populations, Eq. 50) and g (Eq. 5) with the wall rules;
 *   h = h' + sum_{a>=1} g_a (Eq. 9), inverted to (T, f_l) (Eq. 2);
 *   rho, momentum, Boussinesq buoyancy (Eq. 55-56) and the liquid-fraction solid force;
 *   D3Q19 MRT collision with forcing (Eq. 49, 51-54);
 *   D3Q7 enthalpy collision, MRT (Eq. 21-25, 47) or SRT (Eq. 6-8);
 *   store of f*, g*_1..6 and the FP64 rest channel h' = h - sum_{a>=1} g*_a.
 *
 * Conventions for every call:
 *  - Lattice extents nx, ny, nz >= 1, nx*ny*nz < 2^31.  Node n = x + nx*(y + ny*z).
 *  - Fields are structure-of-arrays in node order; u is three planes (u_x, u_y, u_z).
 *  - Walls lie half a cell outside the boundary nodes: the -x wall at x = -1/2.
 *  - "host" pointers are ordinary CPU memory and are read or written before the call
 *    returns; "device" pointers are CUDA global memory of the handle's device and are
 *    accessed in stream order on the handle's stream.  The caller owns all memory.
 *  - The library never allocates device memory: all of it is carved out of the
 *    caller's workspace.  A handle is not thread-safe.
 *  - Every call returns an lbpc_status; lbpc_last_error() gives the message.
 */
#ifndef LBPC_H
#define LBPC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBPC_ABI_VERSION 3

typedef enum lbpc_status {
    LBPC_OK = 0,
    LBPC_ERR_PARAM = -1,     /* invalid argument or parameter block */
    LBPC_ERR_WORKSPACE = -2, /* workspace missing, misaligned or too small */
    LBPC_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    LBPC_ERR_DIVERGED = -4,  /* a non-finite h or rho appeared (state stays readable) */
    LBPC_ERR_STATE = -5      /* the call is not allowed in the handle's current state */
} lbpc_status;

/* face order of bc[] / T_wall[] / per-face fields: -x, +x, -y, +y, -z, +z */
enum { LBPC_PERIODIC = 0, LBPC_ISOTHERMAL = 1, LBPC_ADIABATIC = 2 };
enum { LBPC_FLOW_NONE = 0, LBPC_FLOW_MRT = 1, LBPC_FLOW_SRT = 2 };
enum { LBPC_ENTH_MRT = 1, LBPC_ENTH_SRT = 2 };
/* storage precision of the populations; collision runs in FP64 for LBPC_FP64 and in
 * FP32 registers otherwise; h', the H -> (T, f_l) inversion and reductions are FP64.
 * FP16S / BF16S store f - w_a and g_a - (omega_T/2) Cp_ref Tref in 16 bits (116 B per
 * node update); the _G32 modes store f that way and g in FP32 (140 B), which keeps the
 * enthalpy populations and the wall fluxes they carry at FP32 resolution. */
enum { LBPC_FP64 = 0, LBPC_FP32 = 1, LBPC_FP16S = 2, LBPC_BF16S = 3, LBPC_FP16S_G32 = 4,
       LBPC_BF16S_G32 = 5 };
enum { LBPC_PULL = 0, LBPC_AA = 1 };

/*
 * Parameter block (physical inputs; the lattice mapping is done by lbpc_create).
 *  flow_model  LBPC_FLOW_NONE: conduction only (u = 0, no flow lattice);
 *              LBPC_FLOW_MRT: Eq. 49 with the rates of Eq. 52;
 *              LBPC_FLOW_SRT: Eq. 49 with every non-conserved rate = 1/tau_f.
 *  enth_model  LBPC_ENTH_MRT (Eq. 21-25) or LBPC_ENTH_SRT (Eq. 6-7).
 *  bc[6]       LBPC_PERIODIC (both faces of an axis), LBPC_ISOTHERMAL (anti-bounce-back
 *              of g at T_wall), LBPC_ADIABATIC (bounce-back of g).  Every non-periodic
 *              face is a no-slip wall for f (bounce-back).
 *  Ra, Pr, St, Ma   Eq. 64 groups; Ma = U0 / c_s with U0 = sqrt(g beta dT H), H = nx.
 *              The mapping: nu = U0 H sqrt(Pr/Ra), chi = nu/Pr, g beta = U0^2/(dT H),
 *              s_nu from Eq. 59, sigma_chi from Eq. 34, L = Cp_l (Th - Tm) / St.
 *  Th, Tm, Tref  hot-wall, melting and buoyancy-reference temperatures (Eq. 55).
 *  Cp_s, Cp_l, Cp_ref, omega_T  specific heats of Eq. 2/7 and the D3Q7 weight constant
 *              (Eq. 8; c_sT^2 = omega_T).
 *  tau_g > 0   overrides the diffusivity: chi = (tau_g - 1/2) omega_T (Eq. 20).
 *  nu > 0      overrides the lattice viscosity.
 *  s_e, s_eps, s_q, s_pi, s_t  flow rates of Eq. 52 (<= 0: 1.19, 1.4, 1.2, 1.4, 1.98).
 *  sigma4 > 0  sets sigma_4 = sigma_5 = sigma_6; <= 0 uses 2 - sigma_chi (Eq. 47).
 *  h0          uniform initial enthalpy (lbpc_set_initial_h overrides per node).
 *  report_every > 0  record diagnostics every so many steps (lbpc_get_history) and check
 *              for divergence at the end of lbpc_step; 0 disables both.
 *  lambda_s, lambda_l  both > 0: per-phase thermal conductivities (Eq. 1, rho0 = 1; Sec.
 *              3.1.2 case (b)), conduction only (flow_model NONE, no tau_g).  The
 *              enthalpy rates then follow per node from f_l: chi = lambda(f_l) / C_p,ref
 *              with lambda(f_l) = lambda_s + f_l (lambda_l - lambda_s) (the paper gives no
 *              mushy-zone rule), sigma_chi from Eq. 34, sigma_4..6 as set above.  The
 *              adjoint refuses this mode (LBPC_ERR_STATE).  Both 0: one conductivity.
 *  darcy_A > 0 replaces the liquid-fraction solid closure (u = f_l u*, F_s = -2 (1 - f_l)
 *              rho0 u*) by an enthalpy-porosity drag F_s = -D rho0 u with D = darcy_A
 *              (1 - f_l)^2 / (f_l^3 + darcy_eps) (darcy_eps <= 0: 1e-3), solved together
 *              with u = u* + F_s / 2: u = phi u*, phi = 1 / (1 + D/2).  Not in the paper (a
 *              common alternative closure); the adjoint differentiates it.  0: the paper's.
 */
typedef struct lbpc_params {
    int flow_model;
    int enth_model;
    int precision;
    int streaming;
    int bc[6];
    double T_wall[6];
    double Ra, Pr, St, Ma;
    double Th, Tm, Tref;
    double Cp_s, Cp_l, Cp_ref, omega_T;
    double tau_g;
    double nu;
    double s_e, s_eps, s_q, s_pi, s_t;
    double sigma4;
    double h0;
    int report_every;
    double lambda_s, lambda_l;
    double darcy_A, darcy_eps;
} lbpc_params;

typedef struct lbpc_handle lbpc_handle;

/* Field selection bits of lbpc_get_fields*. */
enum { LBPC_FIELD_T = 1, LBPC_FIELD_FL = 2, LBPC_FIELD_H = 4, LBPC_FIELD_RHO = 8,
       LBPC_FIELD_U = 16 };

/* Scalar diagnostics (FP64), indices into lbpc_get_scalars / lbpc_get_history rows.
 *  LIQUID_VOL  sum of f_l over the lattice (liquid volume, Sec. 3.2.2 / 3.3);
 *  NU_HOT      Nusselt number of the -x wall, 3D form of Eq. 65: H/(chi Cp_ref dT) times
 *              the wall-averaged enthalpy entering per step through the wall links;
 *  FRONT_MEAN  liquid volume per unit -x wall area (melt depth);
 *  SUM_H, SUM_RHO  total enthalpy and mass;  STEP  time step of the state;
 *  NU_FD       Eq. 65 with the one-sided difference (T_w - T(x=0)) / (1/2);
 *  FRONT_MID   mean first f_l = 1/2 crossing along x on y = ny/2, z = nz/4, nz/2, 3nz/4;
 *  NAN         number of nodes with non-finite h or rho. */
enum { LBPC_S_LIQUID_VOL = 0, LBPC_S_NU_HOT, LBPC_S_FRONT_MEAN, LBPC_S_SUM_H, LBPC_S_SUM_RHO,
       LBPC_S_STEP, LBPC_S_NU_FD, LBPC_S_FRONT_MID, LBPC_S_NAN, LBPC_S_COUNT };

/* Derived lattice constants, indices into lbpc_get_lattice. */
enum { LBPC_L_CHI = 0, LBPC_L_NU, LBPC_L_GBETA, LBPC_L_SIGMA_CHI, LBPC_L_SIGMA4, LBPC_L_S_NU,
       LBPC_L_LATENT, LBPC_L_HS, LBPC_L_HL, LBPC_L_TAU_G, LBPC_L_TAU_F, LBPC_L_S_E,
       LBPC_L_S_EPS, LBPC_L_S_Q, LBPC_L_S_PI, LBPC_L_S_T, LBPC_L_U0, LBPC_L_COUNT };

/* sizeof(lbpc_params) as compiled into the library (binding layout check). */
size_t lbpc_params_size(void);
int lbpc_abi_version(void);

/* Bytes of device workspace lbpc_create needs for this lattice and parameter block
 * (0 if the parameters are invalid).  Per node: 2 x (19 + 6) populations (pull) or
 * 1 x (19 + 6) (AA) in the storage precision, 8 B of h', 8 B of field staging. */
size_t lbpc_workspace_bytes(int nx, int ny, int nz, const lbpc_params *p);

/* Validate p, map it to lattice units, carve the state out of dev_ws (device, 256-byte
 * aligned, >= lbpc_workspace_bytes) and initialise the equilibrium state at uniform
 * h0 and uniform wall temperatures.  cuda_stream is a cudaStream_t (NULL: legacy
 * default stream) used for every later launch.  On success *out owns no memory but
 * the handle itself; dev_ws must outlive it.  Sizes: nx ny nz < 2^31 nodes, ny and nz
 * <= 65535 (grid limits).  Errors: LBPC_ERR_PARAM (before any CUDA call),
 * LBPC_ERR_WORKSPACE, LBPC_ERR_CUDA. */
lbpc_status lbpc_create(int nx, int ny, int nz, const lbpc_params *p, void *dev_ws,
                        size_t ws_bytes, void *cuda_stream, lbpc_handle **out);

/* Host-only: the derived lattice constants lbpc_create would use (out: n >= LBPC_L_COUNT
 * doubles).  No CUDA call; LBPC_ERR_PARAM for an invalid parameter block. */
lbpc_status lbpc_lattice_constants(int nx, int ny, int nz, const lbpc_params *p, double *out,
                                   int n);

/* Reset to t = 0: f = f^eq(rho = 1, u = 0), g = g^eq(h, T(h), 0) (Eq. 7) from h
 * (host, N values; NULL = uniform p->h0). */
lbpc_status lbpc_set_initial_h(lbpc_handle *h, const double *h_host);

/* Per-node temperature of an ISOTHERMAL face (host, face-area values: y + ny z for
 * -x/+x, x + nx z for -y/+y, x + nx y for -z/+z).  Takes effect from the next step;
 * the current populations are kept. */
lbpc_status lbpc_set_wall_temperature(lbpc_handle *h, int face, const double *T_host);

/* Advance n >= 0 time steps on the handle's stream (asynchronous unless report_every
 * > 0 and the call passes a diagnostics point, in which case the call waits for the stream
 * and returns LBPC_ERR_DIVERGED if the last diagnostics it recorded saw a non-finite
 * value).  LBPC_ERR_STATE after divergence. */
lbpc_status lbpc_step(lbpc_handle *h, int n);

/* Macroscopic fields of the current state (after the last stream, Eq. 2 / Eq. 56),
 * FP64, N values each (u: 3N).  Any pointer may be NULL; mask selects LBPC_FIELD_*.
 * _dev: device pointers, stream-ordered.  Host variant: synchronous. */
lbpc_status lbpc_get_fields(lbpc_handle *h, unsigned mask, double *T, double *fl, double *hh,
                            double *rho, double *u);
lbpc_status lbpc_get_fields_dev(lbpc_handle *h, double *T, double *fl, double *hh, double *rho,
                                double *u);

/* Scalar diagnostics of the current state (host, n >= LBPC_S_COUNT doubles). Synchronous. */
lbpc_status lbpc_get_scalars(lbpc_handle *h, double *out, int n);

/* Rows recorded every report_every steps since the last reset (host, max_rows x
 * LBPC_S_COUNT doubles, row-major); *rows receives the number of rows written.  The
 * device keeps the most recent LBPC_HISTORY_ROWS rows. */
#define LBPC_HISTORY_ROWS 4096
lbpc_status lbpc_get_history(lbpc_handle *h, double *out, int max_rows, int *rows);

/* Pre-collision populations of the current state in FP64 (device): f (19 x N, absent
 * when flow_model = NONE: may be NULL) and g (7 x N, g_0 = h').  _set_ loads such a
 * state (t unchanged); the state is then rounded to the storage precision. */
lbpc_status lbpc_get_distributions_dev(lbpc_handle *h, double *f, double *g);
lbpc_status lbpc_set_distributions_dev(lbpc_handle *h, const double *f, const double *g);

/* Derived lattice constants (host, n >= LBPC_L_COUNT doubles). */
lbpc_status lbpc_get_lattice(const lbpc_handle *h, double *out, int n);

/* Checkpoint of the full state (populations, h', wall fields, step) in host memory:
 * lbpc_state_bytes() bytes; lbpc_load requires a handle of the same shape, precision
 * and streaming.  Synchronous. */
size_t lbpc_state_bytes(const lbpc_handle *h);
lbpc_status lbpc_save(lbpc_handle *h, void *host_buf, size_t bytes);
lbpc_status lbpc_load(lbpc_handle *h, const void *host_buf, size_t bytes);

/*
 * Adjoint (hand-written reverse mode of the coupled step; not in the paper, which has
 * no gradients).  Objective J = sum over nodes of f_l(h_N), the liquid volume after
 * nsteps steps from the state held when lbpc_adjoint_forward is called; that state is a
 * fixed input.  Gradients: dJ/dT_w of the per-node temperature field of one isothermal
 * face (face-area values, layout of lbpc_set_wall_temperature) and dJ/dSt, where St
 * enters through L = C_p,l (Th - Tm) / St (Eq. 2, 64).  Derivatives at the kinks of the
 * Eq. 2 inversion are those of the branch the forward took.
 *
 * Memory stays bounded by checkpointing: the forward saves the state at the start of
 * every ckpt_every-step segment but the last and writes the per-step macroscopic tape
 * (h - h_s, rho and j in the compute precision: 20 B per node and step in FP32)
 * over the last segment; the backward sweeps that tape backwards, then for each earlier
 * segment recomputes it from its checkpoint writing the tape (in the checkpoint slots: the
 * handle's own state is not touched), and sweeps it backwards.  The adjoint populations
 * are kept in the compute precision;
 * the parameter gradients accumulate in FP64.  Pull streaming only (LBPC_ERR_STATE
 * otherwise).  dev_ws: device, 256-byte aligned, >= lbpc_adjoint_workspace_bytes().
 *
 * lbpc_adjoint_forward advances the handle by nsteps and returns J (host);
 * lbpc_adjoint_backward (no stepping in between) returns the gradients (host) and leaves
 * the handle at the final state; lbpc_adjoint does both.
 */
size_t lbpc_adjoint_workspace_bytes(const lbpc_handle *h, int nsteps, int ckpt_every);
lbpc_status lbpc_adjoint_forward(lbpc_handle *h, int nsteps, int ckpt_every, void *dev_ws,
                                 size_t ws_bytes, double *J_host);
lbpc_status lbpc_adjoint_backward(lbpc_handle *h, int face, double *dJ_dTw_host,
                                  double *dJ_dSt_host);
lbpc_status lbpc_adjoint(lbpc_handle *h, int nsteps, int ckpt_every, void *dev_ws, size_t ws_bytes,
                         int face, double *J_host, double *dJ_dTw_host, double *dJ_dSt_host);

/*
 * lbpc_get_scalars_noalloc: the LBPC_S_* diagnostics of the current state, like
 * lbpc_get_scalars, for callers that cannot allocate device memory at that point (a
 * device whose free memory is owned by a pool, code that must not call cudaMalloc or
 * cudaFree because they may synchronise the device, a memory budget fixed before the
 * run).  The paper has no counterpart; this is an interface convenience.
 *
 * out_dev: device buffer of LBPC_S_COUNT doubles, written in stream order on the
 * handle's stream; the call does not wait for the result.  The block partial sums live
 * in a static device array of about 152 KB that the library holds on every device that
 * loads it, until the process exits; no memory is allocated.  The first call on a device
 * looks the array's address up (cudaGetSymbolAddress) and caches it, so make that first
 * call before any stream capture.  All calls share the array: calls whose executions
 * overlap on the GPU (other streams, other handles, other threads) race on it and must
 * be serialised by the caller.  LBPC_ERR_PARAM if nx > LBPC_NOALLOC_MAX_NX or out_dev is
 * NULL.
 */
#define LBPC_NOALLOC_MAX_NX 4096
lbpc_status lbpc_get_scalars_noalloc(lbpc_handle *h, double *out_dev);

long long lbpc_step_count(const lbpc_handle *h);
/* Number of kernels this handle has launched since it was created. */
long long lbpc_launch_count(const lbpc_handle *h);
const char *lbpc_last_error(const lbpc_handle *h); /* NULL handle: last create error */
void lbpc_destroy(lbpc_handle *h);

#ifdef __cplusplus
}
#endif
#endif
