// Bulk-tensor (TMA) copies and mbarrier waits for sm_100-class GPUs, in
// inline PTX.  Every wait is bounded: when the iteration limit runs out the
// kernel records FCFS_DEVERR_TIMEOUT in a device status word, waits (bounded)
// for the copies it still has in flight and returns, so no CTA can hang the
// GPU and the first timeout ends the launch.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace fcfs {

constexpr int FCFS_DEVERR_TIMEOUT = 1;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Make prior generic-proxy writes to shared memory visible to the async
// (TMA) proxy before a bulk copy overwrites the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 3D tiled bulk tensor load (box of the tensor map) into shared memory,
// completion counted on the mbarrier.  c0 (innermost) must be 16-byte aligned
// in elements; c0/c1/c2 may lie outside the tensor (zero fill).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of the barrier.  Returns false (and records
// the timeout in *status) if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(status, FCFS_DEVERR_TIMEOUT);
    return false;
}

// After a bounded wait ran out, a kernel stops walking its tiles: the CTA
// leaves at the next block-wide barrier.  Before it does, one thread waits
// (again bounded) for the n copies the CTA still has in flight, held by ring
// stages stg, stg+1, ... (mod S) starting at barrier phase `phase`, so that
// no copy lands in shared memory after the CTA has exited.
__device__ __forceinline__ void drain_ring(uint64_t* bars, int S, int stg, uint32_t phase, int n, int* status) {
    for (int i = 0; i < n && i < S; ++i) {
        int st = stg + i;
        uint32_t ph = phase;
        if (st >= S) {
            st -= S;
            ph ^= 1u;
        }
        mbar_wait(&bars[st], ph, status);
    }
}


// The tiles one CTA of a persistent grid takes: chunks of `chunk` consecutive
// tiles dealt round-robin over the grid (the costlier edge tiles spread over
// all CTAs and neighbouring tiles run at the same time, sharing their halos
// in L2), or one contiguous run per CTA when chunk is 0 (fewer changes of
// plane, for per-channel weights).  k-th tile of this CTA: tile(k), k < n.
struct TileDeal {
    int b, G, per, chunk, n;
    __device__ __forceinline__ int tile(int k) const {
        if (chunk == 0) return b * per + k;
        const int j = k / chunk;
        return (b + j * G) * chunk + (k - j * chunk);
    }
};

__device__ __forceinline__ TileDeal deal_tiles(int ntiles, int chunk) {
    TileDeal d;
    d.b = blockIdx.x;
    d.G = gridDim.x;
    d.per = (ntiles + d.G - 1) / d.G;
    d.chunk = chunk;
    if (chunk <= 0) {
        d.chunk = 0;
        d.n = max(0, min(ntiles, (d.b + 1) * d.per) - d.b * d.per);
    } else {
        const int nch = (ntiles + chunk - 1) / chunk;
        d.n = nch > d.b ? ((nch - 1 - d.b) / d.G + 1) * chunk : 0;
        if (nch > d.b && (nch - 1 - d.b) % d.G == 0) d.n -= nch * chunk - ntiles;  // the short last chunk
    }
    return d;
}

}  // namespace fcfs
