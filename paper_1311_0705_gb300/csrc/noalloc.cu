// Allocation-free variant of hg_trace_rays.
//
// Some callers cannot allocate device memory when they trace: code that
// runs inside a stream capture whose owner forbids allocation nodes,
// real-time loops that must never enter an allocator, and hosts that give
// this library a fixed memory budget up front.  hg_trace_rays takes its
// scratch (a 48-byte start record per ray and a work counter) from the
// stream-ordered allocator; this entry point takes it from one fixed array
// compiled into the library instead, and allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "hg_internal.h"
#include "walk.cuh"

namespace hg {
hg_status trace_rays_prealloc(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                              double kappa, const hg_trace_opts *opts, void *tau, int32_t *ncross,
                              uint8_t *ray_status, RayStart *starts, unsigned long long *counter,
                              cudaStream_t stream);
}

namespace {

// Layout: the work counter in the first 256 bytes, then the start records.
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes = kCounterBytes + (size_t)HG_NOALLOC_MAX_RAYS * sizeof(hg::RayStart);

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mtx;
void *g_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device with that device current.  Host code may not pass the symbol
// itself to a kernel: in host code it names a host-side stand-in.
hg_status scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        hg::set_error("hg_trace_rays_noalloc: no current device: %s", cudaGetErrorString(e));
        return HG_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        hg::set_error("hg_trace_rays_noalloc: device index %d beyond %d", dev, kMaxDevices);
        return HG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mtx);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            hg::set_error("hg_trace_rays_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return HG_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return HG_OK;
}

}  // namespace

extern "C" hg_status hg_trace_rays_noalloc(const hg_grid *g, int64_t n, const double *o, const double *d,
                                           const double *s_max, double kappa, const hg_trace_opts *opts,
                                           void *tau, int32_t *ncross, uint8_t *ray_status, hg_stream stream) {
    if (n < 0 || n > HG_NOALLOC_MAX_RAYS) {
        hg::set_error("hg_trace_rays_noalloc: %lld rays exceed the fixed scratch of %d rays; "
                      "split the batch or use hg_trace_rays",
                      (long long)n, HG_NOALLOC_MAX_RAYS);
        return HG_EINVAL;
    }
    void *base = nullptr;
    hg_status st = scratch_address(&base);
    if (st != HG_OK) return st;
    unsigned char *b = static_cast<unsigned char *>(base);
    // the counter is zeroed by the launch itself (cudaMemsetAsync); the start
    // records are fully rewritten by the setup pass before they are read
    return hg::trace_rays_prealloc(g, n, o, d, s_max, kappa, opts, tau, ncross, ray_status,
                                   reinterpret_cast<hg::RayStart *>(b + kCounterBytes),
                                   reinterpret_cast<unsigned long long *>(b), (cudaStream_t)stream);
}
