// sscg_solve_static: the s-step solve with its workspace in a fixed array
// that the library itself places in device memory, for callers that cannot
// allocate device memory (see include/sscg.h).  It runs the existing solve
// unchanged; only the source of the workspace differs.
#include <mutex>

#include "internal.h"

namespace {

// The workspace of every sscg_solve_static call on a device.  In host code
// `g_static_scratch` names a host-side stand-in, not device memory: its
// device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[SSCG_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];  // per device ordinal, set once
std::mutex g_scratch_mutex;

}  // namespace

extern "C" int sscg_solve_static(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x,
                                 const sscg_opts* opts, sscg_info* info) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (!mat || !opts) return sscg::set_err(ctx, SSCG_ERR_INVALID, "null matrix or options");
    size_t need = 0;
    if (sscg_solve_workspace_bytes(mat, opts, &need) != SSCG_OK)
        return sscg::set_err(ctx, SSCG_ERR_INVALID, "invalid solve options");
    if (need > SSCG_STATIC_SCRATCH_BYTES)
        return sscg::set_err(ctx, SSCG_ERR_SPACE,
                             "this solve needs %zu bytes of workspace; the static scratch holds %zu "
                             "(use sscg_solve with caller workspace)",
                             need, (size_t)SSCG_STATIC_SCRATCH_BYTES);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sscg::set_err(ctx, SSCG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev != ctx->device || dev < 0 || dev >= kMaxDevices)
        return sscg::set_err(ctx, SSCG_ERR_INVALID, "make the context's device (%d) current (current: %d)",
                             ctx->device, dev);
    void* ptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {  // set-up, once per device, with that device current
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return sscg::set_err(ctx, SSCG_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        ptr = g_scratch_addr[dev];
    }
    return sscg_solve(ctx, mat, b, x, opts, info, ptr, SSCG_STATIC_SCRATCH_BYTES);
}
