// H integration with library-owned static scratch, for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc or hand it a
// workspace: a Fortran SCF driver without a CUDA allocator of its own, a
// plug-in living inside another framework's memory pool, or code that must
// not allocate between the steps of a captured or real-time loop.  For them
// fgi_integrate_h_static runs the same H integration as fgi_integrate_h with
// its scratch in a fixed-size, file-scope device array instead of a
// caller-owned buffer.
#include <cstdio>
#include <mutex>

#include "../../include/fgi.h"
#include "fgi_internal.h"

namespace {

// The scratch: every GPU that loads the library holds it until the process
// exits.  All calls on a device share it and it keeps the last call's data.
__device__ __align__(256) unsigned char g_static_scratch[FGI_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on `dev` (looked up once per device, with
// that device current: in host code the array's name is only a host-side
// stand-in, never a device address).
cudaError_t scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaError_t e = cudaSetDevice(dev);
        void *p = nullptr;
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (prev >= 0) cudaSetDevice(prev);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int fgi_integrate_h_static(fgi_ctx *ctx, const double *v_dev, double *h_dev, int accumulate,
                                      void *stream)
{
    if (!ctx) return FGI_ERR_ARG;
    const int dev = fgi::internal_device(ctx);
    if (dev < 0 || dev >= kMaxDevices)
        return fgi::internal_error(ctx, FGI_ERR_STATE, "fgi_integrate_h_static: context has no CUDA device");
    size_t need = 0;
    int rc = fgi_workspace_size(ctx, &need);
    if (rc) return rc;
    if (need > FGI_STATIC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "fgi_integrate_h_static: this plan needs %zu bytes of scratch; the static scratch holds %zu "
                 "(use fgi_integrate_h with a caller workspace)",
                 need, (size_t)FGI_STATIC_SCRATCH_BYTES);
        return fgi::internal_error(ctx, FGI_ERR_WORKSPACE, msg);
    }
    void *scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "fgi_integrate_h_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return fgi::internal_error(ctx, FGI_ERR_CUDA, msg);
    }
    // profiling off: the event pool may grow, and this call must not allocate
    return fgi::internal_integrate_h(ctx, v_dev, h_dev, accumulate, scratch, FGI_STATIC_SCRATCH_BYTES, stream,
                                     false);
}
