// Shared pieces of the bulk-copy backward kernels: conversions, tile
// geometry of the input-gradient tiles, copy issue, forward-weight access.
#pragma once

#include <type_traits>

#include "fcfs_internal.cuh"
#include "fcfs_tma.cuh"

namespace fcfs {

// Device status word of the bulk-copy backward kernels (bounded waits); each
// translation unit that includes this header owns its copy.
static __device__ int g_status_bwd_tma = 0;

namespace {

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void store_out(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_out(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

struct DxGeo {
    int plane, c, qx0, qy0, nqx, nqy;
    AxRange X, Y;
    int gx_al, xoff, gy0;
};

__device__ __forceinline__ DxGeo dx_geo(const TmaDxParams& T, int tile) {
    DxGeo g;
    const int txy = T.qtiles_x * T.qtiles_y;
    g.plane = tile / txy;
    const int rem = tile - g.plane * txy;
    const int ty = rem / T.qtiles_x, tx = rem - ty * T.qtiles_x;
    g.c = g.plane % T.C;
    g.qx0 = tx * T.QX;
    g.qy0 = ty * T.QY;
    g.nqx = min(T.QX, T.aj[2].n_x - g.qx0);
    g.nqy = min(T.QY, T.aj[1].n_x - g.qy0);
    g.X = ax_range(T.aj[2], T.pad, g.qx0, g.qx0 + g.nqx - 1);
    g.Y = ax_range(T.aj[1], T.pad, g.qy0, g.qy0 + g.nqy - 1);
    const int gx0 = g.X.alo * T.aj[2].r + T.aj[2].lo_in;
    g.gx_al = gx0 >= 0 ? (gx0 / T.align) * T.align : -(((-gx0) + T.align - 1) / T.align) * T.align;
    g.xoff = gx0 - g.gx_al;
    g.gy0 = g.Y.alo * T.aj[1].r + T.aj[1].lo_in;
    return g;
}

template <typename Tg>
__device__ __forceinline__ void issue(const TmaDxParams& T, const DxGeo& g, void* buf, uint64_t* bar) {
    fence_proxy_async_smem();
    mbar_expect_tx(bar, (uint32_t)(T.GBW * T.GBH * sizeof(Tg)));
    tma_load_3d(buf, &T.tmap, g.gx_al, g.gy0, g.plane, bar);
}

__device__ __forceinline__ float fwd_weight(const AxisP& A, int c, int k) {
    return A.learn ? A.w[(long long)c * A.w_cstride + k] : A.wf[k];
}

}  // namespace
}  // namespace fcfs
