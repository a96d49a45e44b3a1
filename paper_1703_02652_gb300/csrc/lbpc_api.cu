// lbpc_api.cu -- host side of the C ABI declared in include/lbpc.h.
//
// Parameter validation and the mapping of the physical groups to lattice units
// (Eq. 20, 34, 52, 59, 64), carving of the caller's device workspace, the time loop and
// the diagnostics.  All device memory belongs to the caller; nothing here allocates it.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbpc.h"
#include "lbpc_host.h"
#include "lbpc_internal.h"

using namespace lbpc;

namespace {

// Byte offsets of every buffer inside the workspace.
struct WsLayout {
    size_t f[2], g[2], hp, tw[6], partial, lines, result, hist, stage, flag, total;
};

constexpr size_t kAlign = 256;
constexpr uint32_t kStateMagic = 0x4c425043u;  // "LBPC"

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// bytes of one stored f / g value of a storage mode
size_t f_store_bytes(int precision) {
    return precision == LBPC_FP64 ? 8 : (precision == LBPC_FP32 ? 4 : 2);
}
size_t g_store_bytes(int precision) {
    return precision == LBPC_FP64 ? 8 : (precision == LBPC_FP16S || precision == LBPC_BF16S ? 2 : 4);
}

long face_area(int nx, int ny, int nz, int face) {
    return face < 2 ? (long)ny * nz : (face < 4 ? (long)nx * nz : (long)nx * ny);
}

WsLayout ws_layout(int nx, int ny, int nz, const lbpc_params* p) {
    WsLayout w{};
    const size_t N = (size_t)nx * ny * nz, Sf = f_store_bytes(p->precision),
                 Sg = g_store_bytes(p->precision);
    const bool flow = p->flow_model != LBPC_FLOW_NONE;
    const int nlat = p->streaming == LBPC_PULL ? 2 : 1;
    size_t off = 0;
    for (int i = 0; i < 2; i++) {
        w.f[i] = off;
        if (flow && i < nlat) off = align_up(off + 19 * N * Sf);
    }
    for (int i = 0; i < 2; i++) {
        w.g[i] = off;
        if (i < nlat) off = align_up(off + 6 * N * Sg);
    }
    w.hp = off; off = align_up(off + 8 * N);
    for (int f = 0; f < 6; f++) { w.tw[f] = off; off = align_up(off + 8 * face_area(nx, ny, nz, f)); }
    w.partial = off; off = align_up(off + 8 * (size_t)RED_BLOCKS * NRED);
    w.lines = off; off = align_up(off + 8 * 3 * (size_t)nx);
    w.result = off; off = align_up(off + 8 * LBPC_S_COUNT);
    w.hist = off; off = align_up(off + 8 * (size_t)LBPC_HISTORY_ROWS * LBPC_S_COUNT);
    w.stage = off; off = align_up(off + 8 * N);
    w.flag = off; off = align_up(off + sizeof(int));
    w.total = off;
    return w;
}

// Fixed-order sum of n partials into out[0] (one block).
__global__ void __launch_bounds__(256) k_sum(const double* __restrict__ p, int n, double* out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += p[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_fill(double* p, double v, int n) {
    // 64-bit index: i + stride may pass 2^31 - 1 for n near the 2^31 - 1 node limit
    for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Deterministic second stage of the diagnostics: fixed-order sums of the block
// partials, then the scalars of the header's LBPC_S_* list.
__global__ void __launch_bounds__(256)
k_finalize(const double* __restrict__ partial, const double* __restrict__ lines, int nx,
           double area, double nu_scale, double fd_scale, double step, int flow, int iso0,
           double* __restrict__ result, double* __restrict__ hist_row) {
    __shared__ double sh[256][NRED];
    double acc[NRED] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < RED_BLOCKS; b += blockDim.x)
        for (int k = 0; k < NRED; k++) acc[k] += partial[b * NRED + k];
    for (int k = 0; k < NRED; k++) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < NRED; k++) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double front = 0.0;
    for (int l = 0; l < 3; l++) {
        const double* v = lines + (size_t)l * nx;
        double xc = nx;  // no crossing: the whole line is liquid
        for (int x = 0; x < nx; x++) {
            if (v[x] < 0.5) {
                xc = x == 0 ? -0.5 : (x - 1) + (v[x - 1] - 0.5) / (v[x - 1] - v[x]);
                break;
            }
        }
        front += (xc + 0.5) / 3.0;
    }
    double r[LBPC_S_COUNT];
    r[LBPC_S_LIQUID_VOL] = sh[0][0];
    r[LBPC_S_NU_HOT] = iso0 ? nu_scale * sh[0][3] / area : 0.0;
    r[LBPC_S_FRONT_MEAN] = sh[0][0] / area;
    r[LBPC_S_SUM_H] = sh[0][1];
    r[LBPC_S_SUM_RHO] = flow ? sh[0][2] : 0.0;
    r[LBPC_S_STEP] = step;
    r[LBPC_S_NU_FD] = fd_scale * sh[0][4] / area;
    r[LBPC_S_FRONT_MID] = front;
    r[LBPC_S_NAN] = sh[0][5];
    for (int k = 0; k < LBPC_S_COUNT; k++) {
        result[k] = r[k];
        if (hist_row) hist_row[k] = r[k];
    }
}

}  // namespace

cudaError_t lbpc::finalize_reduction(const double* partial, const double* lines, int nx,
                                     double area, double nu_scale, double fd_scale, double step,
                                     int flow, int iso0, double* result, double* hist_row,
                                     cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(partial, lines, nx, area, nu_scale, fd_scale, step, flow, iso0,
                                 result, hist_row);
    return cudaGetLastError();
}

struct lbpc_handle {
    int nx, ny, nz, N;
    int device;
    lbpc_params p;
    Derived d;
    cudaStream_t stream;
    const Launchers* L;
    char* ws;
    size_t ws_bytes;
    WsLayout lay;
    void *f[2], *g[2];
    double *hp, *tw[6], *partial, *lines, *result, *hist, *stage;
    int* flag;
    int cur;
    long long step;
    long long hist_count;
    long long launches;
    bool diverged;
    struct Adjoint {
        bool ready = false;
        char* ws = nullptr;
        int nsteps = 0, k = 0, nseg = 0;
        long long end_step = 0;
        size_t ckpt_bytes = 0, off_f = 0, off_g = 0, off_hp = 0;
        char* ckpt = nullptr;
        void* tape_e = nullptr;
        void* tape_m = nullptr;
        void* lam[2] = {nullptr, nullptr};
        double *gtw = nullptr, *Lpart = nullptr, *Jpart = nullptr, *red = nullptr;
        int nblocks = 0;
    } adj;
    Args args;
    std::string err;
};

static std::string g_create_err;

#define LBPC_CK(h, call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
            return LBPC_ERR_CUDA;                                                        \
        }                                                                                \
    } while (0)

namespace {

lbpc_status fail(lbpc_handle* h, lbpc_status s, const char* msg) {
    h->err = msg;
    return s;
}

lbpc_status set_device(lbpc_handle* h) {
    int cur = -1;
    LBPC_CK(h, cudaGetDevice(&cur));
    if (cur != h->device) LBPC_CK(h, cudaSetDevice(h->device));
    return LBPC_OK;
}

Layout current_layout(const lbpc_handle* h) {
    if (h->p.streaming == LBPC_PULL) return LAYOUT_PULL;
    return (h->step % 2 == 0) ? LAYOUT_AA_NATURAL : LAYOUT_AA_SWAPPED;
}

const void* cur_f(const lbpc_handle* h) { return h->p.streaming == LBPC_PULL ? h->f[h->cur] : h->f[0]; }
const void* cur_g(const lbpc_handle* h) { return h->p.streaming == LBPC_PULL ? h->g[h->cur] : h->g[0]; }

// Reduction pass + finalize on the stream; result lands in h->result (and a history row).
lbpc_status diagnostics(lbpc_handle* h, bool record) {
    MacroOut o{};
    o.partial = h->partial;
    o.lines = h->lines;
    h->L->macro(h->args, current_layout(h), cur_f(h), cur_g(h), h->hp, o, h->stream);
    h->launches += 2;  // reduction pass + finalize
    double* row = nullptr;
    if (record) {
        row = h->hist + (size_t)(h->hist_count % LBPC_HISTORY_ROWS) * LBPC_S_COUNT;
        h->hist_count++;
    }
    const double area = (double)h->ny * h->nz;
    const double nu_scale = h->d.H / (h->d.chi * h->p.Cp_ref * h->d.dT);
    const double fd_scale = h->d.H / h->d.dT;
    LBPC_CK(h, finalize_reduction(h->partial, h->lines, h->nx, area, nu_scale, fd_scale,
                                  (double)h->step, h->p.flow_model != LBPC_FLOW_NONE,
                                  h->p.bc[0] == LBPC_ISOTHERMAL, h->result, row, h->stream));
    return LBPC_OK;
}

lbpc_status init_state(lbpc_handle* h, const double* Qf, const double* Qg, const double* h0) {
    void* f = h->p.streaming == LBPC_PULL ? h->f[h->cur] : h->f[0];
    void* g = h->p.streaming == LBPC_PULL ? h->g[h->cur] : h->g[0];
    const Layout lay = h->p.streaming == LBPC_PULL ? LAYOUT_PULL : LAYOUT_AA_NATURAL;
    h->L->init(h->args, lay, Qf, Qg, h0, f, g, h->hp, h->stream);
    h->launches += 2;
    LBPC_CK(h, cudaGetLastError());
    return LBPC_OK;
}

lbpc_status reset_from_h(lbpc_handle* h, const double* h_host) {
    if (h_host) {
        LBPC_CK(h, cudaMemcpyAsync(h->stage, h_host, sizeof(double) * h->N, cudaMemcpyHostToDevice,
                                   h->stream));
    } else {
        k_fill<<<256, 256, 0, h->stream>>>(h->stage, h->p.h0, h->N);
        h->launches++;
        LBPC_CK(h, cudaGetLastError());
    }
    h->cur = 0;
    h->step = 0;
    h->hist_count = 0;
    h->diverged = false;
    // no diagnostics recorded yet (the workspace comes uninitialised from the caller)
    LBPC_CK(h, cudaMemsetAsync(h->result, 0, sizeof(double) * LBPC_S_COUNT, h->stream));
    lbpc_status s = init_state(h, nullptr, nullptr, h->stage);
    if (s != LBPC_OK) return s;
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    return LBPC_OK;
}

}  // namespace

extern "C" {

size_t lbpc_params_size(void) { return sizeof(lbpc_params); }
int lbpc_abi_version(void) { return LBPC_ABI_VERSION; }

size_t lbpc_workspace_bytes(int nx, int ny, int nz, const lbpc_params* p) {
    Derived d;
    std::string e;
    if (!validate_and_map(nx, ny, nz, p, d, e)) return 0;
    return ws_layout(nx, ny, nz, p).total;
}

lbpc_status lbpc_create(int nx, int ny, int nz, const lbpc_params* p, void* dev_ws, size_t ws_bytes,
                        void* cuda_stream, lbpc_handle** out) {
    if (!out) { g_create_err = "null output handle pointer"; return LBPC_ERR_PARAM; }
    *out = nullptr;
    Derived d;
    std::string e;
    if (!validate_and_map(nx, ny, nz, p, d, e)) { g_create_err = e; return LBPC_ERR_PARAM; }
    const WsLayout lay = ws_layout(nx, ny, nz, p);
    if (!dev_ws) { g_create_err = "null workspace"; return LBPC_ERR_WORKSPACE; }
    if (((uintptr_t)dev_ws) % kAlign != 0) { g_create_err = "workspace not 256-byte aligned"; return LBPC_ERR_WORKSPACE; }
    if (ws_bytes < lay.total) { g_create_err = "workspace smaller than lbpc_workspace_bytes()"; return LBPC_ERR_WORKSPACE; }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, dev_ws) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        g_create_err = "workspace is not CUDA device memory";
        return LBPC_ERR_WORKSPACE;
    }
    lbpc_handle* h = new (std::nothrow) lbpc_handle();
    if (!h) { g_create_err = "out of host memory"; return LBPC_ERR_PARAM; }
    h->nx = nx; h->ny = ny; h->nz = nz; h->N = nx * ny * nz;
    h->device = attr.device;
    h->p = *p;
    h->d = d;
    h->stream = (cudaStream_t)cuda_stream;
    switch (p->precision) {
        case LBPC_FP64: h->L = &launchers_f64(); break;
        case LBPC_FP32: h->L = &launchers_f32(); break;
        case LBPC_FP16S: h->L = &launchers_f16(); break;
        case LBPC_BF16S: h->L = &launchers_bf16(); break;
        case LBPC_FP16S_G32: h->L = &launchers_f16g32(); break;
        default: h->L = &launchers_bf16g32(); break;
    }
    h->ws = (char*)dev_ws;
    h->ws_bytes = ws_bytes;
    h->lay = lay;
    const bool flow = p->flow_model != LBPC_FLOW_NONE;
    for (int i = 0; i < 2; i++) {
        h->f[i] = flow ? h->ws + lay.f[i] : nullptr;
        h->g[i] = h->ws + lay.g[i];
    }
    if (p->streaming == LBPC_AA) { h->f[1] = h->f[0]; h->g[1] = h->g[0]; }
    h->hp = (double*)(h->ws + lay.hp);
    for (int f = 0; f < 6; f++) h->tw[f] = (double*)(h->ws + lay.tw[f]);
    h->partial = (double*)(h->ws + lay.partial);
    h->lines = (double*)(h->ws + lay.lines);
    h->result = (double*)(h->ws + lay.result);
    h->hist = (double*)(h->ws + lay.hist);
    h->stage = (double*)(h->ws + lay.stage);
    h->flag = (int*)(h->ws + lay.flag);

    fill_args(h->args, nx, ny, nz, *p, d, h->tw);

    lbpc_status s = set_device(h);
    if (s == LBPC_OK) {
        for (int f = 0; f < 6 && s == LBPC_OK; f++) {
            std::vector<double> tw(face_area(nx, ny, nz, f), p->T_wall[f]);
            if (cudaMemcpy(h->tw[f], tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
                h->err = "cudaMemcpy of the wall temperature failed";
                s = LBPC_ERR_CUDA;
            }
        }
    }
    if (s == LBPC_OK) s = reset_from_h(h, nullptr);
    if (s != LBPC_OK) {
        g_create_err = h->err;
        delete h;
        return s;
    }
    *out = h;
    return LBPC_OK;
}

lbpc_status lbpc_set_initial_h(lbpc_handle* h, const double* h_host) {
    if (!h) return LBPC_ERR_PARAM;
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    return reset_from_h(h, h_host);
}

lbpc_status lbpc_set_wall_temperature(lbpc_handle* h, int face, const double* T_host) {
    if (!h) return LBPC_ERR_PARAM;
    if (face < 0 || face > 5 || !T_host) return fail(h, LBPC_ERR_PARAM, "bad face or null field");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    LBPC_CK(h, cudaMemcpy(h->tw[face], T_host, sizeof(double) * face_area(h->nx, h->ny, h->nz, face),
                          cudaMemcpyHostToDevice));
    return LBPC_OK;
}

lbpc_status lbpc_step(lbpc_handle* h, int n) {
    if (!h) return LBPC_ERR_PARAM;
    if (n < 0) return fail(h, LBPC_ERR_PARAM, "negative step count");
    if (h->diverged) return fail(h, LBPC_ERR_STATE, "state diverged; reset it before stepping");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    const int rep = h->p.report_every;
    bool recorded = false;  // diagnostics taken during this call
    for (int i = 0; i < n; i++) {
        if (h->p.streaming == LBPC_PULL) {
            h->L->step(h->args, STEP_PULL, h->f[h->cur], h->f[1 - h->cur], h->g[h->cur],
                       h->g[1 - h->cur], h->hp, h->stream);
            h->cur = 1 - h->cur;
        } else {
            const StepKind k = (h->step % 2 == 0) ? STEP_AA_EVEN : STEP_AA_ODD;
            h->L->step(h->args, k, h->f[0], h->f[0], h->g[0], h->g[0], h->hp, h->stream);
        }
        h->step++;
        h->launches++;
        if (rep > 0 && h->step % rep == 0) {
            s = diagnostics(h, true);
            if (s != LBPC_OK) return s;
            recorded = true;
        }
    }
    LBPC_CK(h, cudaGetLastError());
    double nan = 0.0;
    if (recorded) {
        LBPC_CK(h, cudaMemcpyAsync(&nan, h->result + LBPC_S_NAN, sizeof(double),
                                   cudaMemcpyDeviceToHost, h->stream));
        LBPC_CK(h, cudaStreamSynchronize(h->stream));
    } else if (rep == 0 && n > 0) {
        // no diagnostics in this mode: check the stored g populations and the FP64 rest
        // channel after the call's last step (a non-finite f reaches g within one step)
        int bad = 0;
        LBPC_CK(h, cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
        h->L->check(h->args, cur_g(h), h->hp, h->flag, h->stream);
        h->launches++;
        LBPC_CK(h, cudaGetLastError());
        LBPC_CK(h, cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        LBPC_CK(h, cudaStreamSynchronize(h->stream));
        nan = bad;
    }
    if (nan != 0.0) {
        h->diverged = true;
        return fail(h, LBPC_ERR_DIVERGED, "non-finite enthalpy or density");
    }
    return LBPC_OK;
}

lbpc_status lbpc_get_fields_dev(lbpc_handle* h, double* T, double* fl, double* hh, double* rho,
                                double* u) {
    if (!h) return LBPC_ERR_PARAM;
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    MacroOut o{};
    o.T = T; o.fl = fl; o.h = hh; o.rho = rho;
    if (u) { o.ux = u; o.uy = u + h->N; o.uz = u + 2 * (size_t)h->N; }
    h->L->macro(h->args, current_layout(h), cur_f(h), cur_g(h), h->hp, o, h->stream);
    h->launches++;
    LBPC_CK(h, cudaGetLastError());
    return LBPC_OK;
}

lbpc_status lbpc_get_fields(lbpc_handle* h, unsigned mask, double* T, double* fl, double* hh,
                            double* rho, double* u) {
    if (!h) return LBPC_ERR_PARAM;
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    double* dst[7] = {(mask & LBPC_FIELD_T) ? T : nullptr, (mask & LBPC_FIELD_FL) ? fl : nullptr,
                      (mask & LBPC_FIELD_H) ? hh : nullptr, (mask & LBPC_FIELD_RHO) ? rho : nullptr,
                      (mask & LBPC_FIELD_U) && u ? u : nullptr,
                      (mask & LBPC_FIELD_U) && u ? u + h->N : nullptr,
                      (mask & LBPC_FIELD_U) && u ? u + 2 * (size_t)h->N : nullptr};
    for (int k = 0; k < 7; k++) {
        if (!dst[k]) continue;
        MacroOut o{};
        double** slot[7] = {&o.T, &o.fl, &o.h, &o.rho, &o.ux, &o.uy, &o.uz};
        *slot[k] = h->stage;
        h->L->macro(h->args, current_layout(h), cur_f(h), cur_g(h), h->hp, o, h->stream);
        h->launches++;
        LBPC_CK(h, cudaGetLastError());
        LBPC_CK(h, cudaMemcpyAsync(dst[k], h->stage, sizeof(double) * h->N, cudaMemcpyDeviceToHost,
                                   h->stream));
        LBPC_CK(h, cudaStreamSynchronize(h->stream));
    }
    return LBPC_OK;
}

lbpc_status lbpc_get_scalars(lbpc_handle* h, double* out, int n) {
    if (!h) return LBPC_ERR_PARAM;
    if (!out || n < LBPC_S_COUNT) return fail(h, LBPC_ERR_PARAM, "output needs LBPC_S_COUNT doubles");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    s = diagnostics(h, false);
    if (s != LBPC_OK) return s;
    LBPC_CK(h, cudaMemcpyAsync(out, h->result, sizeof(double) * LBPC_S_COUNT, cudaMemcpyDeviceToHost,
                               h->stream));
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    return LBPC_OK;
}

lbpc_status lbpc_get_history(lbpc_handle* h, double* out, int max_rows, int* rows) {
    if (!h) return LBPC_ERR_PARAM;
    if (!rows || (max_rows > 0 && !out)) return fail(h, LBPC_ERR_PARAM, "null output");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    const long long avail = h->hist_count < LBPC_HISTORY_ROWS ? h->hist_count : LBPC_HISTORY_ROWS;
    const long long take = avail < max_rows ? avail : max_rows;
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    for (long long r = 0; r < take; r++) {  // oldest first among the kept rows
        const long long idx = (h->hist_count - avail + r) % LBPC_HISTORY_ROWS;
        LBPC_CK(h, cudaMemcpy(out + r * LBPC_S_COUNT, h->hist + idx * LBPC_S_COUNT,
                              sizeof(double) * LBPC_S_COUNT, cudaMemcpyDeviceToHost));
    }
    *rows = (int)take;
    return LBPC_OK;
}

lbpc_status lbpc_get_distributions_dev(lbpc_handle* h, double* f, double* g) {
    if (!h) return LBPC_ERR_PARAM;
    if (!g) return fail(h, LBPC_ERR_PARAM, "g output is required");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    h->L->dist(h->args, current_layout(h), cur_f(h), cur_g(h), h->hp, f, g, h->stream);
    h->launches++;
    LBPC_CK(h, cudaGetLastError());
    return LBPC_OK;
}

lbpc_status lbpc_set_distributions_dev(lbpc_handle* h, const double* f, const double* g) {
    if (!h) return LBPC_ERR_PARAM;
    if (!g) return fail(h, LBPC_ERR_PARAM, "g input is required");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    if (h->p.streaming == LBPC_AA && h->step % 2 != 0)
        return fail(h, LBPC_ERR_STATE, "AA streaming: load a state only after an even step count");
    s = init_state(h, h->p.flow_model != LBPC_FLOW_NONE ? f : nullptr, g, nullptr);
    if (s != LBPC_OK) return s;
    h->diverged = false;
    return LBPC_OK;
}

static void lattice_out(const Derived& d, double* out) {
    out[LBPC_L_CHI] = d.chi;
    out[LBPC_L_NU] = d.nu;
    out[LBPC_L_GBETA] = d.gbeta;
    out[LBPC_L_SIGMA_CHI] = d.sigma_chi;
    out[LBPC_L_SIGMA4] = d.sigma4;
    out[LBPC_L_S_NU] = d.s_nu;
    out[LBPC_L_LATENT] = d.L;
    out[LBPC_L_HS] = d.hs;
    out[LBPC_L_HL] = d.hl;
    out[LBPC_L_TAU_G] = d.tau_g;
    out[LBPC_L_TAU_F] = d.tau_f;
    out[LBPC_L_S_E] = d.s_e;
    out[LBPC_L_S_EPS] = d.s_eps;
    out[LBPC_L_S_Q] = d.s_q;
    out[LBPC_L_S_PI] = d.s_pi;
    out[LBPC_L_S_T] = d.s_t;
    out[LBPC_L_U0] = d.U0;
}

lbpc_status lbpc_get_lattice(const lbpc_handle* h, double* out, int n) {
    if (!h || !out || n < LBPC_L_COUNT) return LBPC_ERR_PARAM;
    lattice_out(h->d, out);
    return LBPC_OK;
}

lbpc_status lbpc_lattice_constants(int nx, int ny, int nz, const lbpc_params* p, double* out,
                                   int n) {
    if (!out || n < LBPC_L_COUNT) { g_create_err = "output needs LBPC_L_COUNT doubles"; return LBPC_ERR_PARAM; }
    Derived d;
    if (!validate_and_map(nx, ny, nz, p, d, g_create_err)) return LBPC_ERR_PARAM;
    lattice_out(d, out);
    return LBPC_OK;
}

namespace {
struct StateHeader {
    uint32_t magic, version;
    int32_t nx, ny, nz, precision, streaming, flow;
    int64_t step;
};

size_t state_pop_bytes(const lbpc_handle* h, size_t* fb, size_t* gb) {
    const size_t N = (size_t)h->N;
    *fb = h->p.flow_model != LBPC_FLOW_NONE ? 19 * N * h->L->f_bytes : 0;
    *gb = 6 * N * h->L->g_bytes;
    size_t tw = 0;
    for (int f = 0; f < 6; f++) tw += 8 * face_area(h->nx, h->ny, h->nz, f);
    return sizeof(StateHeader) + *fb + *gb + 8 * N + tw;
}
}  // namespace

size_t lbpc_state_bytes(const lbpc_handle* h) {
    if (!h) return 0;
    size_t fb, gb;
    return state_pop_bytes(h, &fb, &gb);
}

lbpc_status lbpc_save(lbpc_handle* h, void* host_buf, size_t bytes) {
    if (!h) return LBPC_ERR_PARAM;
    size_t fb, gb;
    const size_t need = state_pop_bytes(h, &fb, &gb);
    if (!host_buf || bytes < need) return fail(h, LBPC_ERR_PARAM, "buffer smaller than lbpc_state_bytes()");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    StateHeader hd{kStateMagic, 1, h->nx, h->ny, h->nz, h->p.precision, h->p.streaming,
                   h->p.flow_model != LBPC_FLOW_NONE, h->step};
    char* o = (char*)host_buf;
    std::memcpy(o, &hd, sizeof hd);
    o += sizeof hd;
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    if (fb) { LBPC_CK(h, cudaMemcpy(o, cur_f(h), fb, cudaMemcpyDeviceToHost)); o += fb; }
    LBPC_CK(h, cudaMemcpy(o, cur_g(h), gb, cudaMemcpyDeviceToHost)); o += gb;
    LBPC_CK(h, cudaMemcpy(o, h->hp, 8 * (size_t)h->N, cudaMemcpyDeviceToHost)); o += 8 * (size_t)h->N;
    for (int f = 0; f < 6; f++) {
        const size_t b = 8 * face_area(h->nx, h->ny, h->nz, f);
        LBPC_CK(h, cudaMemcpy(o, h->tw[f], b, cudaMemcpyDeviceToHost));
        o += b;
    }
    return LBPC_OK;
}

lbpc_status lbpc_load(lbpc_handle* h, const void* host_buf, size_t bytes) {
    if (!h) return LBPC_ERR_PARAM;
    size_t fb, gb;
    const size_t need = state_pop_bytes(h, &fb, &gb);
    if (!host_buf || bytes < need) return fail(h, LBPC_ERR_PARAM, "buffer smaller than lbpc_state_bytes()");
    StateHeader hd;
    std::memcpy(&hd, host_buf, sizeof hd);
    if (hd.magic != kStateMagic || hd.version != 1 || hd.nx != h->nx || hd.ny != h->ny ||
        hd.nz != h->nz || hd.precision != h->p.precision || hd.streaming != h->p.streaming ||
        hd.flow != (h->p.flow_model != LBPC_FLOW_NONE))
        return fail(h, LBPC_ERR_PARAM, "checkpoint does not match this handle");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    const char* o = (const char*)host_buf + sizeof hd;
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    if (fb) { LBPC_CK(h, cudaMemcpy((void*)cur_f(h), o, fb, cudaMemcpyHostToDevice)); o += fb; }
    LBPC_CK(h, cudaMemcpy((void*)cur_g(h), o, gb, cudaMemcpyHostToDevice)); o += gb;
    LBPC_CK(h, cudaMemcpy(h->hp, o, 8 * (size_t)h->N, cudaMemcpyHostToDevice)); o += 8 * (size_t)h->N;
    for (int f = 0; f < 6; f++) {
        const size_t b = 8 * face_area(h->nx, h->ny, h->nz, f);
        LBPC_CK(h, cudaMemcpy(h->tw[f], o, b, cudaMemcpyHostToDevice));
        o += b;
    }
    h->step = hd.step;
    h->hist_count = 0;
    h->diverged = false;
    return LBPC_OK;
}

long long lbpc_step_count(const lbpc_handle* h) { return h ? h->step : -1; }

long long lbpc_launch_count(const lbpc_handle* h) { return h ? h->launches : -1; }

const char* lbpc_last_error(const lbpc_handle* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

void lbpc_destroy(lbpc_handle* h) {
    if (!h) return;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != h->device) cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Adjoint (reverse mode with checkpointing).
// ---------------------------------------------------------------------------------
namespace {

struct AdjLayout {
    size_t ckpt_bytes, off_f, off_g, off_hp, ckpt, tape_e, tape_m, lam0, lam1, gtw, Lpart, Jpart,
        red, total;
    int nseg, nblocks;
};

AdjLayout adj_layout(const lbpc_handle* h, int nsteps, int k) {
    AdjLayout L{};
    const size_t N = (size_t)h->N, Sf = h->L->f_bytes, Sg = h->L->g_bytes,
                 Cb = h->L->compute_bytes;
    const bool flow = h->p.flow_model != LBPC_FLOW_NONE;
    L.nseg = (nsteps + k - 1) / k;
    L.off_f = 0;
    L.off_g = align_up(flow ? 19 * N * Sf : 0);
    L.off_hp = L.off_g + align_up(6 * N * Sg);
    L.ckpt_bytes = L.off_hp + align_up(8 * N);
    size_t off = 0;
    // slots 0 .. nseg - 2: segment starts; slot nseg - 1: spare for the recompute
    L.ckpt = off; off += (size_t)(L.nseg > 1 ? L.nseg : 0) * L.ckpt_bytes;
    L.tape_e = off; off = align_up(off + (size_t)k * N * Cb);
    L.tape_m = off; off = align_up(off + (flow ? (size_t)k * 4 * N * Cb : 0));
    const size_t lam = (size_t)(flow ? 26 : 7) * N * Cb;
    L.lam0 = off; off = align_up(off + lam);
    L.lam1 = off; off = align_up(off + lam);
    size_t amax = 0;
    for (int f = 0; f < 6; f++) amax = std::max(amax, (size_t)face_area(h->nx, h->ny, h->nz, f));
    L.gtw = off; off = align_up(off + 8 * amax);
    L.nblocks = node_grid_blocks(h->nx, h->ny, h->nz);
    L.Lpart = off; off = align_up(off + 8 * (size_t)L.nblocks * ADJ_WARPS_PER_BLOCK);
    L.Jpart = off; off = align_up(off + 8 * (size_t)L.nblocks);
    L.red = off; off = align_up(off + 8 * 4);
    L.total = off;
    return L;
}

lbpc_status save_state(lbpc_handle* h, char* dst) {
    auto& A = h->adj;
    const size_t N = (size_t)h->N, Sf = h->L->f_bytes, Sg = h->L->g_bytes;
    if (h->p.flow_model != LBPC_FLOW_NONE)
        LBPC_CK(h, cudaMemcpyAsync(dst + A.off_f, h->f[h->cur], 19 * N * Sf, cudaMemcpyDeviceToDevice, h->stream));
    LBPC_CK(h, cudaMemcpyAsync(dst + A.off_g, h->g[h->cur], 6 * N * Sg, cudaMemcpyDeviceToDevice, h->stream));
    LBPC_CK(h, cudaMemcpyAsync(dst + A.off_hp, h->hp, 8 * N, cudaMemcpyDeviceToDevice, h->stream));
    return LBPC_OK;
}

}  // namespace

extern "C" {

size_t lbpc_adjoint_workspace_bytes(const lbpc_handle* h, int nsteps, int ckpt_every) {
    if (!h || nsteps < 1 || ckpt_every < 1) return 0;
    return adj_layout(h, nsteps, ckpt_every).total;
}

lbpc_status lbpc_adjoint_forward(lbpc_handle* h, int nsteps, int ckpt_every, void* dev_ws,
                                 size_t ws_bytes, double* J_host) {
    if (!h) return LBPC_ERR_PARAM;
    if (nsteps < 1 || ckpt_every < 1) return fail(h, LBPC_ERR_PARAM, "nsteps and ckpt_every must be >= 1");
    if (h->p.streaming != LBPC_PULL) return fail(h, LBPC_ERR_STATE, "the adjoint needs pull streaming");
    if (h->p.lambda_s > 0 || h->p.lambda_l > 0)
        return fail(h, LBPC_ERR_STATE, "the adjoint needs one conductivity (no lambda_s / lambda_l)");
    if (h->diverged) return fail(h, LBPC_ERR_STATE, "state diverged");
    const AdjLayout L = adj_layout(h, nsteps, ckpt_every);
    if (!dev_ws || ((uintptr_t)dev_ws) % kAlign != 0 || ws_bytes < L.total)
        return fail(h, LBPC_ERR_WORKSPACE, "adjoint workspace missing, misaligned or smaller than lbpc_adjoint_workspace_bytes()");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    auto& A = h->adj;
    char* w = (char*)dev_ws;
    A.ready = false;
    A.ws = w;
    A.nsteps = nsteps;
    A.k = ckpt_every;
    A.nseg = L.nseg;
    A.nblocks = L.nblocks;
    A.ckpt_bytes = L.ckpt_bytes;
    A.off_f = L.off_f; A.off_g = L.off_g; A.off_hp = L.off_hp;
    A.ckpt = w + L.ckpt;
    A.tape_e = w + L.tape_e;
    A.tape_m = w + L.tape_m;
    A.lam[0] = w + L.lam0;
    A.lam[1] = w + L.lam1;
    A.gtw = (double*)(w + L.gtw);
    A.Lpart = (double*)(w + L.Lpart);
    A.Jpart = (double*)(w + L.Jpart);
    A.red = (double*)(w + L.red);
    // Forward with a checkpoint at the start of every segment but the last, and one of the
    // final state.  The last segment writes its tape as it goes, so the backward sweep
    // starts on it without recomputing it (and needs no checkpoint at its start).
    // A step that ends on a later segment start writes its populations straight into that
    // checkpoint (only h', updated in place, is copied), and the next step reads them from
    // there: the populations of those checkpoints cost no extra copy.
    const int tail = (L.nseg - 1) * ckpt_every;
    if (L.nseg > 1) {
        s = save_state(h, A.ckpt);
        if (s != LBPC_OK) return s;
    }
    const bool flow = h->p.flow_model != LBPC_FLOW_NONE;
    const void* sf = h->f[h->cur];  // where the current populations are
    const void* sg = h->g[h->cur];
    for (int i = 0; i < nsteps; i++) {
        const int nb = 1 - h->cur;  // the lattice buffer the step writes unless redirected
        if (i < tail) {
            const bool to_ckpt = (i + 1) % ckpt_every == 0 && i + 1 < tail;
            char* slot = A.ckpt + (size_t)((i + 1) / ckpt_every) * A.ckpt_bytes;
            void* df = to_ckpt ? (flow ? slot + A.off_f : nullptr) : h->f[nb];
            void* dg = to_ckpt ? slot + A.off_g : h->g[nb];
            h->L->step(h->args, STEP_PULL, sf, df, sg, dg, h->hp, h->stream);
            sf = df;
            sg = dg;
            if (to_ckpt) {
                LBPC_CK(h, cudaMemcpyAsync(slot + A.off_hp, h->hp, 8 * (size_t)h->N,
                                           cudaMemcpyDeviceToDevice, h->stream));
            } else {
                h->cur = nb;
            }
        } else {
            const size_t t = (size_t)(i - tail);
            h->L->step_tape(h->args, sf, h->f[nb], sg, h->g[nb], h->hp,
                            (char*)A.tape_e + t * h->N * h->L->compute_bytes,
                            (char*)A.tape_m + t * 4 * h->N * h->L->compute_bytes, h->stream);
            sf = h->f[nb];
            sg = h->g[nb];
            h->cur = nb;
        }
        h->step++;
        h->launches++;
    }
    // seed lambda_N = d f_l / dh (and J = sum f_l, the direct dJ/dL part)
    h->L->adj_seed(h->args, h->g[h->cur], h->hp, A.lam[0], A.Lpart, A.Jpart, h->stream);
    k_sum<<<1, 256, 0, h->stream>>>(A.Jpart, A.nblocks, A.red);
    h->launches += 2;
    LBPC_CK(h, cudaGetLastError());
    double J = 0.0;
    LBPC_CK(h, cudaMemcpyAsync(&J, A.red, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    if (J_host) *J_host = J;
    A.end_step = h->step;
    A.ready = true;
    return LBPC_OK;
}

lbpc_status lbpc_adjoint_backward(lbpc_handle* h, int face, double* dJ_dTw_host, double* dJ_dSt_host) {
    if (!h) return LBPC_ERR_PARAM;
    if (face < 0 || face > 5) return fail(h, LBPC_ERR_PARAM, "face must be 0..5");
    auto& A = h->adj;
    if (!A.ready || h->step != A.end_step)
        return fail(h, LBPC_ERR_STATE, "call lbpc_adjoint_forward first (and do not step in between)");
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    const size_t N = (size_t)h->N, Cb = h->L->compute_bytes;
    LBPC_CK(h, cudaMemsetAsync(A.gtw, 0, 8 * face_area(h->nx, h->ny, h->nz, face), h->stream));
    int cl = 0;
    for (int seg = A.nseg - 1; seg >= 0; seg--) {
        const int start = seg * A.k, len = std::min(A.k, A.nsteps - start);
        if (seg < A.nseg - 1) {  // the last segment's tape is the forward's
            // recompute the segment, writing the tape, in checkpoint slots seg and seg + 1
            // (both free from here on: slot seg + 1 belongs to a segment already swept, or is
            // the spare slot), with slot seg's h' updated in place: the handle's own lattice
            // keeps the final state throughout
            char* ck[2] = {A.ckpt + (size_t)seg * A.ckpt_bytes,
                           A.ckpt + (size_t)(seg + 1) * A.ckpt_bytes};
            const bool flow = h->p.flow_model != LBPC_FLOW_NONE;
            double* hp = (double*)(ck[0] + A.off_hp);
            for (int t = 0; t < len; t++) {
                char* src = ck[t & 1];
                char* dst = ck[(t + 1) & 1];
                h->L->step_tape(h->args, flow ? src + A.off_f : nullptr,
                                flow ? dst + A.off_f : nullptr, src + A.off_g, dst + A.off_g, hp,
                                (char*)A.tape_e + (size_t)t * N * Cb,
                                (char*)A.tape_m + (size_t)t * 4 * N * Cb, h->stream);
            }
            h->launches += len;
        }
        for (int t = len - 1; t >= 0; t--) {  // reverse sweep
            h->L->adj_reverse(h->args, A.lam[cl], A.lam[1 - cl], (char*)A.tape_e + (size_t)t * N * Cb,
                              (char*)A.tape_m + (size_t)t * 4 * N * Cb, face, A.gtw, A.Lpart, h->stream);
            cl = 1 - cl;
        }
        h->launches += len;
    }
    k_sum<<<1, 256, 0, h->stream>>>(A.Lpart, A.nblocks * ADJ_WARPS_PER_BLOCK, A.red + 1);
    h->launches++;
    LBPC_CK(h, cudaGetLastError());
    double dJdL = 0.0;
    LBPC_CK(h, cudaMemcpyAsync(&dJdL, A.red + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (dJ_dTw_host)
        LBPC_CK(h, cudaMemcpyAsync(dJ_dTw_host, A.gtw, 8 * face_area(h->nx, h->ny, h->nz, face),
                                   cudaMemcpyDeviceToHost, h->stream));
    LBPC_CK(h, cudaStreamSynchronize(h->stream));
    // L = C_p,l dT / St
    if (dJ_dSt_host) *dJ_dSt_host = dJdL * (-h->p.Cp_l * h->d.dT / (h->p.St * h->p.St));
    A.ready = false;
    return LBPC_OK;
}

lbpc_status lbpc_adjoint(lbpc_handle* h, int nsteps, int ckpt_every, void* dev_ws, size_t ws_bytes,
                         int face, double* J_host, double* dJ_dTw_host, double* dJ_dSt_host) {
    lbpc_status s = lbpc_adjoint_forward(h, nsteps, ckpt_every, dev_ws, ws_bytes, J_host);
    if (s != LBPC_OK) return s;
    return lbpc_adjoint_backward(h, face, dJ_dTw_host, dJ_dSt_host);
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Read-only view of a handle for lbpc_noalloc.cu.
// ---------------------------------------------------------------------------------
namespace lbpc_noalloc_access {
lbpc_status view(lbpc_handle* h, View* v) {
    lbpc_status s = set_device(h);
    if (s != LBPC_OK) return s;
    v->L = h->L;
    v->args = &h->args;
    v->layout = current_layout(h);
    v->f = cur_f(h);
    v->g = cur_g(h);
    v->hp = h->hp;
    v->nx = h->nx;
    v->ny = h->ny;
    v->nz = h->nz;
    v->device = h->device;
    v->flow = h->p.flow_model != LBPC_FLOW_NONE;
    v->iso0 = h->p.bc[0] == LBPC_ISOTHERMAL;
    v->nu_scale = h->d.H / (h->d.chi * h->p.Cp_ref * h->d.dT);
    v->fd_scale = h->d.H / h->d.dT;
    v->step = (double)h->step;
    v->stream = h->stream;
    return LBPC_OK;
}

void set_error(lbpc_handle* h, const char* msg) { h->err = msg; }
void count_launches(lbpc_handle* h, int n) { h->launches += n; }
}  // namespace lbpc_noalloc_access
