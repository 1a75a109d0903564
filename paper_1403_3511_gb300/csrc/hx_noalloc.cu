// hx_norm_noalloc: the FP64 norm reduction with its scratch in a fixed device array, for callers
// that must not allocate device memory (see include/hx.h).
//
// The scratch is a file-scope __device__ array: every GPU that loads libhx.so holds it until the
// process exits.  Host code never passes the array's name to a kernel (on the host it is only a
// stand-in symbol); it passes the device address obtained with cudaGetSymbolAddress, looked up
// once per device with that device current.
#include <stdint.h>

#include <mutex>

#include "hx_internal.h"

namespace hx {

// Layout: [0, kNoAllocMaxBlocks) per-block partial sums, then the result, then the arrival
// counter of the last-block reduction (as an unsigned in the first word of the last slot).
constexpr int kNoAllocMaxBlocks = 1024;
constexpr int kNoAllocSlots = kNoAllocMaxBlocks + 2;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots];

constexpr int kMaxDevices = 64;
static double *g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

// The device address of the scratch array on device dev (current), looked up with
// cudaGetSymbolAddress and kept once found.  A failed lookup is not kept: the next call tries again
// (it fails, for example, while a stream is being captured).
static int scratch_for_device(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("hx_norm_noalloc: device %d out of range", dev);
        return HX_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "hx_norm_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = (double *)ptr;
    }
    *out = g_scratch_ptr[dev];
    return HX_OK;
}

// Called by hx_problem_create with the problem's device current: binds the scratch there, so that
// the module holding the array is loaded (and its memory reserved) where allocation is expected,
// not at the first hx_norm_noalloc.
int noalloc_bind(int dev)
{
    double *ptr = nullptr;
    return scratch_for_device(dev, &ptr);
}

}  // namespace hx

using namespace hx;

struct hx_problem : Problem {};

extern "C" HX_API int hx_norm_noalloc(hx_problem *p, const void *c, double *out)
{
    if (!p || !c || !out) { set_error("hx_norm_noalloc: NULL argument"); return HX_EINVAL; }
    if ((uintptr_t)c % (p->cfg.dtype == HX_C64 ? 8 : 16) != 0) {
        set_error("hx_norm_noalloc: vector not aligned to its element size");
        return HX_EINVAL;
    }
    const int G = apply_grid(p);
    if (G > kNoAllocMaxBlocks) {
        set_error("hx_norm_noalloc: the reduction needs %d block partials, the fixed scratch holds %d", G,
                  kNoAllocMaxBlocks);
        return HX_EUNSUPPORTED;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "hx_norm_noalloc: cudaGetDevice");
    if (dev != p->device) {
        set_error("hx_norm_noalloc: current device %d is not the problem's device %d", dev, p->device);
        return HX_EINVAL;
    }
    double *scratch = nullptr;
    int rc = scratch_for_device(dev, &scratch);
    if (rc) return rc;
    double *partials = scratch;
    double *result = scratch + kNoAllocMaxBlocks;
    unsigned *counter = (unsigned *)(scratch + kNoAllocMaxBlocks + 1);
    // the array keeps the previous call's contents: the arrival counter must start at zero
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned), p->stream)) != cudaSuccess)
        return cuda_fail(e, "hx_norm_noalloc: clear counter");
    rc = launch_norm(p, c, p->cfg.dtype == HX_C128, partials, counter, result, p->stream);
    if (rc) return rc;
    double r = 0.0;
    if ((e = cudaMemcpyAsync(&r, result, sizeof(double), cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(p->stream)) != cudaSuccess)
        return cuda_fail(e, "hx_norm_noalloc: read result");
    *out = sqrt(r);
    if (!isfinite(*out)) {
        set_error("hx_norm_noalloc: the norm is not finite (the vector holds a NaN or an infinity, or overflows)");
        return HX_ENONFINITE;
    }
    return HX_OK;
}
