// lbpc_noalloc.cu -- lbpc_get_scalars_noalloc: the scalar diagnostics of a handle's state
// computed with scratch memory that the library owns statically, so that the call
// allocates nothing and needs no workspace from its caller beyond the handle's own.
//
// Who needs it: callers that must not allocate device memory at the point where they
// read the diagnostics -- e.g. a monitoring loop that runs while another component owns
// every free byte of the device through a pool, code that must not call cudaMalloc /
// cudaFree because those can synchronise the whole device, or a runtime with a memory
// budget fixed before the run starts.  They give the handle and an output buffer; the
// block partial sums live in the array below.
#include <cstdint>
#include <mutex>

#include "lbpc.h"
#include "lbpc_internal.h"

using namespace lbpc;

namespace {

// Scratch of every call on a device: RED_BLOCKS x NRED block partials followed by the
// three front lines of at most LBPC_NOALLOC_MAX_NX nodes each (about 152 KB).  Every call
// overwrites all of it before reading it, so nothing has to start at zero.
constexpr int kPartials = RED_BLOCKS * NRED;
static __device__ __align__(256) double g_noalloc_scratch[kPartials + 3 * LBPC_NOALLOC_MAX_NX];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Same reduction as the workspace-backed diagnostics: fixed-order sums of the block
// partials, then the LBPC_S_* scalars.
__global__ void __launch_bounds__(256)
k_finalize_noalloc(const double* __restrict__ partial, const double* __restrict__ lines, int nx,
                   double area, double nu_scale, double fd_scale, double step, int flow, int iso0,
                   double* __restrict__ result) {
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
        double xc = nx;
        for (int x = 0; x < nx; x++) {
            if (v[x] < 0.5) {
                xc = x == 0 ? -0.5 : (x - 1) + (v[x - 1] - 0.5) / (v[x - 1] - v[x]);
                break;
            }
        }
        front += (xc + 0.5) / 3.0;
    }
    result[LBPC_S_LIQUID_VOL] = sh[0][0];
    result[LBPC_S_NU_HOT] = iso0 ? nu_scale * sh[0][3] / area : 0.0;
    result[LBPC_S_FRONT_MEAN] = sh[0][0] / area;
    result[LBPC_S_SUM_H] = sh[0][1];
    result[LBPC_S_SUM_RHO] = flow ? sh[0][2] : 0.0;
    result[LBPC_S_STEP] = step;
    result[LBPC_S_NU_FD] = fd_scale * sh[0][4] / area;
    result[LBPC_S_FRONT_MID] = front;
    result[LBPC_S_NAN] = sh[0][5];
}

}  // namespace

// Handle internals used here (defined in lbpc_api.cu).
namespace lbpc_noalloc_access {
struct View {
    const Launchers* L;
    const Args* args;
    Layout layout;
    const void* f;
    const void* g;
    const double* hp;
    int nx, ny, nz, device, flow, iso0;
    double nu_scale, fd_scale, step;
    cudaStream_t stream;
};
lbpc_status view(lbpc_handle* h, View* v);
void set_error(lbpc_handle* h, const char* msg);
}  // namespace lbpc_noalloc_access

extern "C" lbpc_status lbpc_get_scalars_noalloc(lbpc_handle* h, double* out_dev) {
    using namespace lbpc_noalloc_access;
    if (!h) return LBPC_ERR_PARAM;
    if (!out_dev) {
        set_error(h, "lbpc_get_scalars_noalloc: null output buffer");
        return LBPC_ERR_PARAM;
    }
    View v;
    lbpc_status s = view(h, &v);  // also makes the handle's device current
    if (s != LBPC_OK) return s;
    if (v.nx > LBPC_NOALLOC_MAX_NX) {
        set_error(h, "lbpc_get_scalars_noalloc: nx exceeds LBPC_NOALLOC_MAX_NX (4096)");
        return LBPC_ERR_PARAM;
    }
    if (v.device < 0 || v.device >= kMaxDevices) {
        set_error(h, "lbpc_get_scalars_noalloc: device index out of range");
        return LBPC_ERR_PARAM;
    }
    double* scratch;
    {
        // One-time set-up per device, with that device current: the host-side name of a
        // __device__ array is not a device address, so ask the runtime for it.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[v.device]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_error(h, "lbpc_get_scalars_noalloc: cudaGetSymbolAddress failed");
                return LBPC_ERR_CUDA;
            }
            g_scratch_addr[v.device] = (double*)p;
        }
        scratch = g_scratch_addr[v.device];
    }
    MacroOut o{};
    o.partial = scratch;
    o.lines = scratch + kPartials;
    v.L->macro(*v.args, v.layout, v.f, v.g, v.hp, o, v.stream);
    k_finalize_noalloc<<<1, 256, 0, v.stream>>>(o.partial, o.lines, v.nx, (double)v.ny * v.nz,
                                                v.nu_scale, v.fd_scale, v.step, v.flow, v.iso0,
                                                out_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(h, cudaGetErrorString(e));
        return LBPC_ERR_CUDA;
    }
    return LBPC_OK;
}
