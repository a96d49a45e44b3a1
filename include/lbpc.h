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
 * FP32 registers otherwise.  h' and the reductions are FP64 in every mode, h - h_s is
 * formed in FP64, and the H -> (T, f_l) inversion of Eq. 2 reports FP64 fields; the FP32
 * collision inverts h - h_s rounded once to nearest (within half an FP32 ulp of the FP64
 * inversion).  Every mode but FP64 stores the flow populations as deviations f - w_a:
 * FP32 as such with g in FP32 (216 B per node update); FP16S / BF16S in 16 bits together
 * with g_a - (omega_T/2) Cp_ref Tref (116 B); the _G32 modes store f in 16 bits and g in
 * FP32 (140 B), which keeps the enthalpy populations and the wall fluxes they carry at
 * FP32 resolution. */
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
 *              for divergence at the diagnostics points; 0: no history, and every
 *              lbpc_step call checks g and h' for non-finite values once, at its end.
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

/* sizeof(lbpc_params) as compiled into the library, and the ABI version (binding layout
 * checks).  Passage: none (interface only; the paper has no software interface). */
size_t lbpc_params_size(void);
int lbpc_abi_version(void);

/* Bytes of device workspace lbpc_create needs for this lattice and parameter block
 * (0 if the parameters are invalid).  Per node: 2 x (19 + 6) populations (pull) or
 * 1 x (19 + 6) (AA) in the storage precision, 8 B of h', 8 B of field staging; per face
 * node: 8 B of wall temperature.
 * Passage: the state of the two lattices, D3Q19 (Eq. 48) and D3Q7 (Eq. 3); the sizing
 * itself has no counterpart in the paper.  No CUDA call. */
size_t lbpc_workspace_bytes(int nx, int ny, int nz, const lbpc_params *p);

/* Validate p, map it to lattice units, carve the state out of dev_ws (device, 256-byte
 * aligned, >= lbpc_workspace_bytes) and initialise the equilibrium state at uniform
 * h0 and uniform wall temperatures.  Passages: the mapping of Eq. 20 / 34 (diffusivity
 * and sigma_chi), Eq. 59 (viscosity and s_nu), Eq. 64 (Ra, Pr, St), Eq. 2 (h_s, L) and
 * Eq. 47 (sigma_4..6); the initial state f^eq (Eq. 53 at rho = 1, u = 0) and g^eq of
 * Eq. 7; the cavity set-up of Sec. 3.3.  cuda_stream is a cudaStream_t (NULL: legacy
 * default stream) used for every later launch.  On success *out owns no memory but
 * the handle itself; dev_ws must outlive it.  Sizes: nx ny nz < 2^31 nodes, ny and nz
 * <= 65535 (grid limits).  Errors: LBPC_ERR_PARAM (before any CUDA call),
 * LBPC_ERR_WORKSPACE, LBPC_ERR_CUDA. */
lbpc_status lbpc_create(int nx, int ny, int nz, const lbpc_params *p, void *dev_ws,
                        size_t ws_bytes, void *cuda_stream, lbpc_handle **out);

/* Host-only: the derived lattice constants lbpc_create would use (out: n >= LBPC_L_COUNT
 * doubles).  No CUDA call; LBPC_ERR_PARAM for an invalid parameter block.  Passages: Eq.
 * 20, 34, 47, 52, 59, 64 and Eq. 2 (the constants listed in LBPC_L_*). */
lbpc_status lbpc_lattice_constants(int nx, int ny, int nz, const lbpc_params *p, double *out,
                                   int n);

/* Reset to t = 0: f = f^eq(rho = 1, u = 0), g = g^eq(h, T(h), 0) (Eq. 7) from h
 * (host, N values; NULL = uniform p->h0).  Passages: Eq. 7 and Eq. 2 (T(h)); the initial
 * conditions of Sec. 3.1-3.3 (a uniform or perturbed enthalpy field).  Synchronous;
 * LBPC_ERR_CUDA if a copy or launch fails. */
lbpc_status lbpc_set_initial_h(lbpc_handle *h, const double *h_host);

/* Per-node temperature of an ISOTHERMAL face (host, face-area values: y + ny z for
 * -x/+x, x + nx z for -y/+y, x + nx y for -z/+z).  Takes effect from the next step;
 * the current populations are kept.  Passage: the isothermal walls of Sec. 3.1-3.3
 * (T_h, T_1 held at a face); the per-node field is the adjoint's control and has no
 * counterpart in the paper.  LBPC_ERR_PARAM for a bad face or a NULL field. */
lbpc_status lbpc_set_wall_temperature(lbpc_handle *h, int face, const double *T_host);

/* Advance n >= 0 time steps on the handle's stream.  Passages: one step is the pull
 * form of Eq. 5 (enthalpy, collision Eq. 6 SRT or Eq. 21-25 MRT with Eq. 47) and of Eq.
 * 50 (flow, collision Eq. 49 with Eq. 51-54), coupled through Eq. 2, Eq. 55 and Eq. 56,
 * with the walls of Sec. 3.1-3.3.  Divergence checks: with report_every > 0 the call is
 * asynchronous unless it passes a diagnostics point; then it waits for the stream and
 * returns LBPC_ERR_DIVERGED if the last diagnostics it recorded saw a non-finite h or rho.
 * With report_every = 0 every call with n > 0 ends with one read of the stored g
 * populations and the FP64 rest channel h' (6 g values + 8 B per node; a non-finite f
 * reaches g within one step), waits for the stream and returns LBPC_ERR_DIVERGED if a
 * value there is not finite.  LBPC_ERR_STATE
 * after divergence, until lbpc_set_initial_h, lbpc_set_distributions_dev or lbpc_load. */
lbpc_status lbpc_step(lbpc_handle *h, int n);

/* Macroscopic fields of the current state (after the last stream), FP64, N values each
 * (u: 3N).  Passages: h = sum_a g_a (Eq. 9), T and f_l by the FP64 inversion of Eq. 2,
 * rho and u of Eq. 56 with the buoyancy of Eq. 55 and the solid closure.  Any pointer may
 * be NULL; mask selects LBPC_FIELD_*.  _dev: device pointers, stream-ordered.  Host
 * variant: synchronous (stages through the workspace).  LBPC_ERR_CUDA on a failed copy. */
lbpc_status lbpc_get_fields(lbpc_handle *h, unsigned mask, double *T, double *fl, double *hh,
                            double *rho, double *u);
lbpc_status lbpc_get_fields_dev(lbpc_handle *h, double *T, double *fl, double *hh, double *rho,
                                double *u);

/* Scalar diagnostics of the current state (host, n >= LBPC_S_COUNT doubles), FP64
 * reductions in a fixed order.  Passages: the Nusselt number of Eq. 65 (3D form, see
 * LBPC_S_NU_HOT), the liquid fraction and melt-front position reported in Sec. 3.2.2 and
 * Sec. 3.3; total enthalpy and mass are the conserved sums of Eq. 9 and Eq. 56 (rho).
 * Synchronous.  LBPC_ERR_PARAM if n < LBPC_S_COUNT. */
lbpc_status lbpc_get_scalars(lbpc_handle *h, double *out, int n);

/* Rows recorded every report_every steps since the last reset (host, max_rows x
 * LBPC_S_COUNT doubles, row-major); *rows receives the number of rows written.  The
 * device keeps the most recent LBPC_HISTORY_ROWS rows.  Passage: the time histories of
 * liquid fraction and Nusselt number of Sec. 3.2.2 / 3.3 (scalars as lbpc_get_scalars).
 * Synchronous. */
#define LBPC_HISTORY_ROWS 4096
lbpc_status lbpc_get_history(lbpc_handle *h, double *out, int max_rows, int *rows);

/* Pre-collision populations of the current state in FP64 (device): f (19 x N, absent
 * when flow_model = NONE: may be NULL) and g (7 x N, g_0 = h').  _set_ loads such a
 * state (t unchanged); the state is then rounded to the storage precision.  Passage: the
 * populations f_a of Eq. 48-50 and g_a of Eq. 3-5 (D3Q19 / D3Q7 velocity order of the
 * paper).  Stream-ordered; _set_ clears a divergence. */
lbpc_status lbpc_get_distributions_dev(lbpc_handle *h, double *f, double *g);
lbpc_status lbpc_set_distributions_dev(lbpc_handle *h, const double *f, const double *g);

/* Derived lattice constants of the handle (host, n >= LBPC_L_COUNT doubles).  Passages:
 * as lbpc_lattice_constants. */
lbpc_status lbpc_get_lattice(const lbpc_handle *h, double *out, int n);

/* Checkpoint of the full state (populations, h', wall fields, step) in host memory:
 * lbpc_state_bytes() bytes; lbpc_load requires a handle of the same shape, precision
 * and streaming (LBPC_ERR_PARAM otherwise, or for a short buffer or a bad header).
 * Synchronous.  Passage: none (checkpoint/restart has no counterpart in the paper). */
size_t lbpc_state_bytes(const lbpc_handle *h);
lbpc_status lbpc_save(lbpc_handle *h, void *host_buf, size_t bytes);
lbpc_status lbpc_load(lbpc_handle *h, const void *host_buf, size_t bytes);

/*
 * Adjoint (hand-written reverse mode of the coupled step; not in the paper, which has
 * no gradients: it differentiates the step defined by Eq. 2, 5, 21-25, 49-56).  Objective J = sum over nodes of f_l(h_N), the liquid volume after
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
 * are kept in the compute precision; the parameter gradients are summed per warp in the
 * compute precision and accumulated in FP64.  Pull streaming only (LBPC_ERR_STATE
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

/* Time steps of the current state; kernels this handle has launched since it was created
 * (every launch on its stream, diagnostics and checks included); the message of the last
 * failed call (NULL handle: of the last failed lbpc_create); release of the handle (the
 * workspace stays the caller's).  Passage: none (bookkeeping of the interface). */
long long lbpc_step_count(const lbpc_handle *h);
long long lbpc_launch_count(const lbpc_handle *h);
const char *lbpc_last_error(const lbpc_handle *h);
void lbpc_destroy(lbpc_handle *h);

#ifdef __cplusplus
}
#endif
#endif
