// lbpc_host.h -- validation of the parameter block and its mapping to lattice units
// (Eq. 20, 34, 52, 59, 64), and the kernel argument block built from it.
#pragma once

#include <cmath>
#include <cstring>
#include <string>

#include "lbpc.h"
#include "lbpc_internal.h"

namespace lbpc {

struct Derived {
    double dT, L, hs, hl, H, chi, nu, gbeta, U0;
    double tau_g, sigma_chi, sigma4, tau_f, s_nu, s_e, s_eps, s_q, s_pi, s_t;
};

inline bool validate_and_map(int nx, int ny, int nz, const lbpc_params* p, Derived& d, std::string& e) {
    if (!p) { e = "null parameter block"; return false; }
    if (nx < 1 || ny < 1 || nz < 1) { e = "lattice extents must be >= 1"; return false; }
    if ((long long)nx * ny * nz >= (1LL << 31)) { e = "lattice exceeds 2^31 - 1 nodes"; return false; }
    // the kernels map z to gridDim.z and y to gridDim.y (at most 65535 blocks each)
    if (ny > 65535 || nz > 65535) { e = "ny and nz must be <= 65535"; return false; }
    if (p->flow_model < LBPC_FLOW_NONE || p->flow_model > LBPC_FLOW_SRT) { e = "flow_model must be 0, 1 or 2"; return false; }
    if (p->enth_model != LBPC_ENTH_MRT && p->enth_model != LBPC_ENTH_SRT) { e = "enth_model must be 1 or 2"; return false; }
    if (p->precision < LBPC_FP64 || p->precision > LBPC_BF16S_G32) { e = "precision must be 0..5"; return false; }
    if (p->streaming != LBPC_PULL && p->streaming != LBPC_AA) { e = "streaming must be 0 or 1"; return false; }
    for (int f = 0; f < 6; f++)
        if (p->bc[f] < LBPC_PERIODIC || p->bc[f] > LBPC_ADIABATIC) { e = "bc codes must be 0..2"; return false; }
    for (int ax = 0; ax < 3; ax++)
        if ((p->bc[2 * ax] == LBPC_PERIODIC) != (p->bc[2 * ax + 1] == LBPC_PERIODIC)) {
            e = "periodic faces must come in pairs"; return false;
        }
    if (p->report_every < 0) { e = "report_every must be >= 0"; return false; }
    if (!(p->omega_T > 0.0 && p->omega_T <= 1.0 / 3.0)) { e = "omega_T must lie in (0, 1/3]"; return false; }
    if (!(p->Cp_s > 0 && p->Cp_l > 0 && p->Cp_ref > 0)) { e = "specific heats must be > 0"; return false; }
    if (!(p->St > 0)) { e = "St must be > 0"; return false; }
    if (!(p->darcy_A >= 0) || !(p->darcy_A < 1e300) || !(p->darcy_eps < 1e300)) {
        e = "darcy_A must be >= 0 and finite"; return false;
    }
    d.dT = p->Th - p->Tm;
    if (!(d.dT > 0)) { e = "Th must exceed Tm"; return false; }
    // Stefan number (Eq. 64) fixes the latent heat; Eq. 2 with h0 = 0 gives h_s and h_l.
    d.L = p->Cp_l * d.dT / p->St;
    d.hs = p->Cp_s * p->Tm;
    d.hl = d.hs + d.L;
    d.H = (double)nx;
    d.chi = d.nu = d.gbeta = d.U0 = 0.0;
    if (p->flow_model != LBPC_FLOW_NONE) {
        if (!(p->Ra > 0 && p->Pr > 0)) { e = "Ra and Pr must be > 0"; return false; }
        if (!(p->Ma > 0 && p->Ma < 1)) { e = "Ma must lie in (0, 1)"; return false; }
        // free-fall velocity U0 = sqrt(g beta dT H) = Ma c_s, c_s^2 = 1/3
        d.U0 = p->Ma / std::sqrt(3.0);
        d.nu = p->nu > 0 ? p->nu : d.U0 * d.H * std::sqrt(p->Pr / p->Ra);
        d.chi = d.nu / p->Pr;
        d.gbeta = d.U0 * d.U0 / (d.dT * d.H);
    }
    if (p->tau_g > 0) {
        if (!(p->tau_g > 0.5)) { e = "tau_g must exceed 1/2"; return false; }
        d.chi = (p->tau_g - 0.5) * p->omega_T;  // Eq. 20
    }
    const bool varchi = p->lambda_s > 0 || p->lambda_l > 0;
    if (varchi) {
        // per-phase conductivities (Sec. 3.1.2 case (b)): chi = lambda / (rho0 C_p,ref) per
        // node; the constants use the solid value
        if (!(p->lambda_s > 0 && p->lambda_l > 0)) { e = "give both lambda_s and lambda_l"; return false; }
        if (p->flow_model != LBPC_FLOW_NONE || p->tau_g > 0) {
            e = "per-phase conductivities need flow_model NONE and no tau_g"; return false;
        }
        d.chi = p->lambda_s / p->Cp_ref;
    }
    if (!(d.chi > 0)) { e = "no thermal diffusivity: give tau_g > 1/2 or a flow model"; return false; }
    d.tau_g = d.chi / p->omega_T + 0.5;  // Eq. 20 / Eq. 34 solved for the relaxation time
    d.sigma_chi = 1.0 / d.tau_g;
    d.sigma4 = p->enth_model == LBPC_ENTH_MRT ? (p->sigma4 > 0 ? p->sigma4 : 2.0 - d.sigma_chi)
                                              : d.sigma_chi;  // Eq. 47
    d.tau_f = d.s_nu = d.s_e = d.s_eps = d.s_q = d.s_pi = d.s_t = 0.0;
    if (p->flow_model != LBPC_FLOW_NONE) {
        d.s_nu = 1.0 / (3.0 * d.nu + 0.5);  // Eq. 59
        d.tau_f = 1.0 / d.s_nu;
        if (p->flow_model == LBPC_FLOW_SRT) {
            d.s_e = d.s_eps = d.s_q = d.s_pi = d.s_t = d.s_nu;
        } else {
            d.s_e = p->s_e > 0 ? p->s_e : 1.19;
            d.s_eps = p->s_eps > 0 ? p->s_eps : 1.4;
            d.s_q = p->s_q > 0 ? p->s_q : 1.2;
            d.s_pi = p->s_pi > 0 ? p->s_pi : 1.4;
            d.s_t = p->s_t > 0 ? p->s_t : 1.98;
        }
        const double r[6] = {d.s_nu, d.s_e, d.s_eps, d.s_q, d.s_pi, d.s_t};
        for (double v : r)
            if (!(v > 0 && v < 2)) { e = "flow relaxation rate outside (0, 2)"; return false; }
    }
    if (!(d.sigma_chi > 0 && d.sigma_chi < 2) || !(d.sigma4 > 0 && d.sigma4 < 2)) {
        e = "enthalpy relaxation rate outside (0, 2)"; return false;
    }
    return true;
}

template <class C>
inline void fill_coef(Coef<C>& c, const lbpc_params& p, const Derived& d) {
    c.Tm = (C)p.Tm;
    c.Cps = (C)p.Cp_s;
    c.Cpl = (C)p.Cp_l;
    c.Cps_inv = (C)(1.0 / p.Cp_s);
    c.Cpl_inv = (C)(1.0 / p.Cp_l);
    c.L = (C)d.L;
    c.L_inv = (C)(1.0 / d.L);
    c.Tref = (C)p.Tref;
    c.gbeta = (C)d.gbeta;
    c.wa_cref = (C)(0.5 * p.omega_T * p.Cp_ref);
    c.wT_cref = (C)(p.omega_T * p.Cp_ref);
    c.sig_chi = (C)d.sigma_chi;
    c.sig4 = c.sig5 = c.sig6 = (C)d.sigma4;
    c.s_e = (C)d.s_e;
    c.s_eps = (C)d.s_eps;
    c.s_q = (C)d.s_q;
    c.s_nu = (C)d.s_nu;
    c.s_pi = (C)d.s_pi;
    c.s_t = (C)d.s_t;
    // every mode but FP64 stores (and collides) the deviations f - w_a of the flow
    // populations from their rest weights: in FP32 too, this keeps the rounding of the
    // stored values and of the moment sums (rho - 1 instead of rho) relative to the
    // deviations, not to O(1) populations.  16-bit g is stored as g_a - (omega_T / 2) Cp_ref
    // Tref (16-bit range); FP32 g is not shifted: near T_m = 0, where most of a melting
    // domain sits, the unshifted values keep their full relative precision
    const bool shifted = p.precision != LBPC_FP64;
    const bool gshifted = p.precision == LBPC_FP16S || p.precision == LBPC_BF16S;
    c.fshift0 = (C)(shifted ? 1.0 / 3.0 : 0.0);
    c.fshift1 = (C)(shifted ? 1.0 / 18.0 : 0.0);
    c.fshift2 = (C)(shifted ? 1.0 / 36.0 : 0.0);
    c.gshift = (C)(gshifted ? 0.5 * p.omega_T * p.Cp_ref * p.Tref : 0.0);
    // row 0 of M (Eq. 51) applied to the rest weights (1/3, 1/18 x 6, 1/36 x 12)
    c.frho = (C)(shifted ? 1.0 : 0.0);
    // Eq. 52-54 with the row norms |row k|^2 of Eq. 51 (2394, 252, 40, 36, 72, 12, 24, 4, 8);
    // rows 1 and 2 carry the factor 19 of m1 - m1eq and the FF prefactors 38 and -11
    c.r_e = (C)(-19.0 * d.s_e / 2394.0);
    c.c_e = (C)(38.0 * (1.0 - 0.5 * d.s_e) / 2394.0);
    c.r_eps = (C)(-d.s_eps / 252.0);
    c.c_eps = (C)(-11.0 * (1.0 - 0.5 * d.s_eps) / 252.0);
    c.r_q = (C)(-d.s_q / 40.0);
    c.c_q = (C)(-(2.0 / 3.0) * (1.0 - 0.5 * d.s_q) / 40.0);
    c.r_nu9 = (C)(-d.s_nu / 36.0);
    c.c_nu9 = (C)((1.0 - 0.5 * d.s_nu) / 36.0);
    c.r_pi10 = (C)(-d.s_pi / 72.0);
    c.c_pi10 = (C)(-0.5 * (1.0 - 0.5 * d.s_pi) / 72.0);
    c.r_nu11 = (C)(-d.s_nu / 12.0);
    c.c_nu11 = (C)((1.0 - 0.5 * d.s_nu) / 12.0);
    c.r_pi12 = (C)(-d.s_pi / 24.0);
    c.c_pi12 = (C)(-0.5 * (1.0 - 0.5 * d.s_pi) / 24.0);
    c.r_nu13 = (C)(-d.s_nu / 4.0);
    c.c_nu13 = (C)((1.0 - 0.5 * d.s_nu) / 4.0);
    c.r_t = (C)(-d.s_t / 8.0);
    c.k_e = (C)(19.0 * (1.0 - d.s_e) / 2394.0);
    c.k_eps = (C)((1.0 - d.s_eps) / 252.0);
    c.k_q = (C)((1.0 - d.s_q) / 40.0);
    c.k_nu9 = (C)((1.0 - d.s_nu) / 36.0);
    c.k_pi10 = (C)((1.0 - d.s_pi) / 72.0);
    c.k_nu11 = (C)((1.0 - d.s_nu) / 12.0);
    c.k_pi12 = (C)((1.0 - d.s_pi) / 24.0);
    c.k_nu13 = (C)((1.0 - d.s_nu) / 4.0);
    c.k_t = (C)((1.0 - d.s_t) / 8.0);
    c.sig4_6 = (C)(d.sigma4 / 6.0);  // sig4 = sig5 = sig6 (Eq. 47)
    c.sig5_6 = (C)(d.sigma4 / 6.0);
    c.sig6_4 = (C)(d.sigma4 / 4.0);
    c.hchi = (C)(0.5 * d.sigma_chi);
    c.dCp = (C)(p.Cp_l - p.Cp_s);
    // per-phase conductivities: 1/sigma_chi = chi_a + chi_b f_l (Eq. 34 with chi =
    // lambda(f_l) / C_p,ref); sigma_4 = s4_a + s4_b sigma_chi (2 - sigma_chi under Eq. 47,
    // sigma_chi for SRT, or the fixed value)
    c.varchi = p.lambda_s > 0 || p.lambda_l > 0;
    c.chi_a = (C)(0.5 + p.lambda_s / (p.omega_T * p.Cp_ref));
    c.chi_b = (C)((p.lambda_l - p.lambda_s) / (p.omega_T * p.Cp_ref));
    const bool srt = p.enth_model == LBPC_ENTH_SRT;
    c.s4_a = (C)(srt ? 0.0 : (p.sigma4 > 0 ? p.sigma4 : 2.0));
    c.s4_b = (C)(srt ? 1.0 : (p.sigma4 > 0 ? 0.0 : -1.0));
    c.j_s_e = (C)(d.s_e / 2394.0);
    c.j_h_e = (C)((1.0 - 0.5 * d.s_e) / 2394.0);
    c.j_s_eps = (C)(d.s_eps / 252.0);
    c.j_h_eps = (C)((1.0 - 0.5 * d.s_eps) / 252.0);
    c.j_s_q = (C)(d.s_q / 40.0);
    c.j_h_q = (C)((1.0 - 0.5 * d.s_q) / 40.0);
    c.j_s_nu9 = (C)(d.s_nu / 36.0);
    c.j_h_nu9 = (C)((1.0 - 0.5 * d.s_nu) / 36.0);
    c.j_s_pi10 = (C)(d.s_pi / 72.0);
    c.j_h_pi10 = (C)((1.0 - 0.5 * d.s_pi) / 72.0);
    c.j_s_nu11 = (C)(d.s_nu / 12.0);
    c.j_h_nu11 = (C)((1.0 - 0.5 * d.s_nu) / 12.0);
    c.j_s_pi12 = (C)(d.s_pi / 24.0);
    c.j_h_pi12 = (C)((1.0 - 0.5 * d.s_pi) / 24.0);
    c.j_s_nu13 = (C)(d.s_nu / 4.0);
    c.j_h_nu13 = (C)((1.0 - 0.5 * d.s_nu) / 4.0);
    c.j_k_e = (C)((1.0 - d.s_e) / 2394.0);
    c.j_k_eps = (C)((1.0 - d.s_eps) / 252.0);
    c.j_k_q = (C)((1.0 - d.s_q) / 40.0);
    c.j_k_nu9 = (C)((1.0 - d.s_nu) / 36.0);
    c.j_k_pi10 = (C)((1.0 - d.s_pi) / 72.0);
    c.j_k_nu11 = (C)((1.0 - d.s_nu) / 12.0);
    c.j_k_pi12 = (C)((1.0 - d.s_pi) / 24.0);
    c.j_k_nu13 = (C)((1.0 - d.s_nu) / 4.0);
    c.j_k_t = (C)((1.0 - d.s_t) / 8.0);
    c.darcy = p.darcy_A > 0;
    c.darcy_A = (C)p.darcy_A;
    c.darcy_eps = (C)(p.darcy_eps > 0 ? p.darcy_eps : 1e-3);
    c.gshift2 = (C)(gshifted ? p.omega_T * p.Cp_ref * p.Tref : 0.0);
}

// Kernel argument block of a validated parameter block; Tw[f] are the device (or host,
// for host-side evaluation) wall temperature fields of the six faces.
inline void fill_args(Args& a, int nx, int ny, int nz, const lbpc_params& p, const Derived& d,
                      double* const Tw[6]) {
    std::memset(&a, 0, sizeof a);
    a.nx = nx; a.ny = ny; a.nz = nz; a.N = nx * ny * nz;
    for (int ax = 0; ax < 3; ax++) a.per[ax] = p.bc[2 * ax] == LBPC_PERIODIC;
    for (int f = 0; f < 6; f++) {
        a.wall[f] = p.bc[f] != LBPC_PERIODIC;
        a.wall_iso[f] = p.bc[f] == LBPC_ISOTHERMAL;
        a.Tw[f] = Tw[f];
    }
    a.flow = p.flow_model != LBPC_FLOW_NONE;
    a.hs = d.hs;
    a.L = d.L;
    fill_coef(a.cf, p, d);
    fill_coef(a.cd, p, d);
}

}  // namespace lbpc
