// lbpc_internal.h -- structures shared by the host side of the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "lbpc.h"

namespace lbpc {

// Per-run constants in one compute precision C (float for the 32/16-bit storage modes,
// double for FP64 storage), so kernels never convert constants at run time.
template <class C>
struct Coef {
    C Tm, Cps, Cpl, Cps_inv, Cpl_inv, L, L_inv, Tref, gbeta;
    C wa_cref;  // (omega_T / 2) Cp_ref: weight times Cp_ref of the six moving g populations
    C wT_cref;  // omega_T Cp_ref: anti-bounce-back source per unit wall temperature
    C sig_chi, sig4, sig5, sig6;           // D3Q7 rates (Eq. 23, 47)
    C s_e, s_eps, s_q, s_nu, s_pi, s_t;    // D3Q19 rates (Eq. 52)
    C fshift0, fshift1, fshift2;           // storage shifts of f: rest / axis / diagonal weight
    C gshift;                              // storage shift of g_1..6
    C frho;  // moment 0 of the f shifts (1 when shifted, else 0); moments 1 and 2 (-11, 3)
             // cancel against the rest-state equilibrium moments and need no constant
    // D3Q19 relaxation with the row norms folded in: d_k = r_k (m_k - meq_k) + c_k FF_k,
    // r_k = -s_k / |row k|^2, c_k = (1 - s_k / 2) (FF_k prefactor) / |row k|^2
    C r_e, c_e, r_eps, c_eps, r_q, c_q, r_nu9, c_nu9, r_pi10, c_pi10, r_nu11, c_nu11, r_pi12,
        c_pi12, r_nu13, c_nu13, r_t;
    // f* rebuilt from its moments: k_k = (1 - s_k) / |row k|^2 (row 1: times 19)
    C k_e, k_eps, k_q, k_nu9, k_pi10, k_nu11, k_pi12, k_nu13, k_t;
    // D3Q7 relaxation: sig4 / 6, sig5 / 6, sig6 / 4, sig_chi / 2; Cp_l - Cp_s; 2 gshift
    C sig4_6, sig5_6, sig6_4, hchi, dCp, gshift2;
    // per-phase conductivities (conduction only): rates per node from f_l
    int varchi;
    C chi_a, chi_b, s4_a, s4_b;
    // enthalpy-porosity solid drag D = darcy_A (1 - f_l)^2 / (f_l^3 + darcy_eps)
    int darcy;
    C darcy_A, darcy_eps;
    // adjoint of the D3Q19 relaxation: j_s_k = s_k / |row k|^2, j_h_k = (1 - s_k/2) / |row
    // k|^2, j_k_k = (1 - s_k) / |row k|^2 (row 16-18: s_t)
    C j_s_e, j_h_e, j_s_eps, j_h_eps, j_s_q, j_h_q, j_s_nu9, j_h_nu9, j_s_pi10, j_h_pi10,
        j_s_nu11, j_h_nu11, j_s_pi12, j_h_pi12, j_s_nu13, j_h_nu13;
    C j_k_e, j_k_eps, j_k_q, j_k_nu9, j_k_pi10, j_k_nu11, j_k_pi12, j_k_nu13, j_k_t;
};

struct Args {
    int nx, ny, nz, N;   // N = nx*ny*nz < 2^31
    int per[3];          // periodic axes
    int wall_iso[6];     // face is an isothermal wall (anti-bounce-back of g)
    int wall[6];         // face is a wall (not periodic)
    const double* Tw[6]; // per-face wall temperature fields (device)
    int flow;            // flow lattice present
    double hs, L;        // FP64 copies for the enthalpy inversion
    Coef<float> cf;
    Coef<double> cd;
};

// How populations are laid out in memory for a gather.
enum Layout : int {
    LAYOUT_PULL = 0,      // two-lattice pull: slot a at node x holds f*_a(x) of the last step
    LAYOUT_AA_NATURAL = 1,// AA after an even number of steps: slot a at x holds f_a(x)
    LAYOUT_AA_SWAPPED = 2 // AA after an odd number of steps: slot abar at x holds f*_a(x)
};

// Step kernel flavours.
enum StepKind : int { STEP_PULL = 0, STEP_AA_EVEN = 1, STEP_AA_ODD = 2 };

struct MacroOut {
    double *T, *fl, *h, *rho, *ux, *uy, *uz;  // any may be null
    double* partial;   // [RED_BLOCKS][NRED] block partial sums (null: no reductions)
    double* lines;     // [3][nx] f_l on the three front lines (null: skip)
};

constexpr int NRED = 6;  // sum f_l, sum h, sum rho, wall flux -x, FD gradient -x, nan count
constexpr int RED_BLOCKS = 1216;  // 8 x 152 SMs
constexpr int RED_THREADS = 256;

struct Launchers {
    void (*step)(const Args&, StepKind, const void* fs, void* fd, const void* gs, void* gd,
                 double* hp, cudaStream_t);
    void (*macro)(const Args&, Layout, const void* f, const void* g, const double* hp,
                  const MacroOut&, cudaStream_t);
    // write populations from a pre-collision state Q (f: 19N FP64 or null = rest
    // equilibrium; g: 7N FP64 or null = equilibrium of h0) into `layout`, then h'.
    void (*init)(const Args&, Layout, const double* Qf, const double* Qg, const double* h0,
                 void* f, void* g, double* hp, cudaStream_t);
    // pre-collision populations in FP64 (f: 19N or null, g: 7N)
    void (*dist)(const Args&, Layout, const void* f, const void* g, const double* hp,
                 double* Qf, double* Qg, cudaStream_t);
    // adjoint: pull step that also writes the macroscopic tape (e: N doubles; rho, j:
    // 4N compute-precision values), seed of lambda at the final state, one reverse step
    void (*step_tape)(const Args&, const void* fs, void* fd, const void* gs, void* gd,
                      double* hp, void* tape_e, void* tape_m, cudaStream_t);
    void (*adj_seed)(const Args&, const void* gs, const double* hp, void* lam, double* Lpart,
                     double* Jpart, cudaStream_t);
    void (*adj_reverse)(const Args&, const void* lin, void* lout, const void* tape_e,
                        const void* tape_m, int wface, double* gtw, double* Lpart, cudaStream_t);
    // divergence check: *flag = 1 if a stored g population or h' is not finite (the flag
    // is not cleared here)
    void (*check)(const Args&, const void* g, const double* hp, int* flag, cudaStream_t);
    size_t f_bytes;        // bytes of one stored f value
    size_t g_bytes;        // bytes of one stored g value
    size_t compute_bytes;  // bytes of one compute-precision value (adjoint, tape)
};

// node grid of the per-node kernels (blocks of 128 threads along x, then y)
inline dim3 node_block_dims(int nx) {
    const int bx = nx >= 128 ? 128 : (nx > 32 ? 64 : 32);
    return dim3(bx, 128 / bx, 1);
}
// The adjoint's dJ/dL partials: one slot per warp of every block of the per-node grid
// (blocks of 128 threads), so the reverse sweep reduces within warps only.
constexpr int ADJ_WARPS_PER_BLOCK = 4;
inline int node_grid_blocks(int nx, int ny, int nz) {
    const dim3 b = node_block_dims(nx);
    return ((nx + b.x - 1) / b.x) * ((ny + b.y - 1) / b.y) * nz;
}

const Launchers& launchers_f64();
const Launchers& launchers_f32();
const Launchers& launchers_f16();
const Launchers& launchers_bf16();
const Launchers& launchers_f16g32();
const Launchers& launchers_bf16g32();

// Second stage of the diagnostics, one block on stream s: fixed-order sums of the
// RED_BLOCKS x NRED block partials and the LBPC_S_* scalars into result[LBPC_S_COUNT]
// (and into hist_row when it is not null).  lines: the three front lines of nx values.
cudaError_t finalize_reduction(const double* partial, const double* lines, int nx, double area,
                               double nu_scale, double fd_scale, double step, int flow, int iso0,
                               double* result, double* hist_row, cudaStream_t s);

}  // namespace lbpc

// Read-only view of a handle for lbpc_noalloc.cu (the handle's layout stays private to
// lbpc_api.cu).  view() also makes the handle's device current; count_launches() adds n
// to the handle's launch count.
namespace lbpc_noalloc_access {
struct View {
    const lbpc::Launchers* L;
    const lbpc::Args* args;
    lbpc::Layout layout;
    const void* f;
    const void* g;
    const double* hp;
    int nx, ny, nz, device, flow, iso0;
    double nu_scale, fd_scale, step;
    cudaStream_t stream;
};
lbpc_status view(lbpc_handle* h, View* v);
void set_error(lbpc_handle* h, const char* msg);
void count_launches(lbpc_handle* h, int n);
}  // namespace lbpc_noalloc_access
