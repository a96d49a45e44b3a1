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

}  // namespace

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
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = finalize_reduction(o.partial, o.lines, v.nx, (double)v.ny * v.nz, v.nu_scale,
                               v.fd_scale, v.step, v.flow, v.iso0, out_dev, nullptr, v.stream);
    count_launches(h, 2);  // reduction pass + finalize
    if (e != cudaSuccess) {
        set_error(h, cudaGetErrorString(e));
        return LBPC_ERR_CUDA;
    }
    return LBPC_OK;
}
