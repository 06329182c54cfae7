// fcfs_backward_noalloc: the backward pass for callers that may not allocate
// device memory themselves.  The weight-gradient partial sums, which
// fcfs_backward keeps in a caller-provided workspace, live here in a fixed
// area that is part of the library image on every GPU that loads it.
#include <mutex>

#include "fcfs_host.h"

namespace {

// Size of the built-in scratch area.  Every GPU that loads libfcfs holds it
// until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch area on the current device.  The host-side
// name of the array is only a stand-in, so the address is looked up once per
// device (with that device current) and cached.
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fcfs::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fcfs::fail(FCFS_ERR_UNSUPPORTED, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fcfs::cuda_fail(e, "cudaGetSymbolAddress of the scratch area");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FCFS_OK;
}

}  // namespace

extern "C" int fcfs_backward_noalloc(const fcfs_desc* d, const void* x, const void* gy, void* gx, float* const* gw,
                                     void* stream) {
    fcfs::clear_error();
    int rc = fcfs::validate_desc(d, true);
    if (rc) return rc;
    bool want_w = false;
    for (int a = 0; gw && a < d->ndim; ++a) want_w |= gw[a] != nullptr;
    size_t need = 0;
    if (want_w) {
        need = fcfs_backward_workspace(d);
        if (need > kNoAllocScratchBytes)
            return fcfs::fail(FCFS_ERR_NOMEM,
                              "weight gradient needs %zu bytes of scratch; the built-in area holds %zu "
                              "(use fcfs_backward with a caller workspace)",
                              need, kNoAllocScratchBytes);
    }
    void* ws = nullptr;
    if (need > 0) {
        rc = scratch_address(&ws);
        if (rc) return rc;
    }
    // the weight-gradient kernel writes every partial-sum record before the
    // reduction reads it, so nothing left by an earlier call needs clearing
    return fcfs_backward(d, x, gy, gx, gw, ws, need, stream);
}
