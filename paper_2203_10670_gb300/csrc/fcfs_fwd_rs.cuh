// K1, register-blocked variant for a compile-time phase count R and window
// span SPAN (the same on both axes): the bulk-copy forward of
// fcfs_fwd_tma.cuh with both passes working per window instead of per output.
//
//   pass x  a thread owns one window of one staged row: it loads the SPAN
//           input samples once and produces all R phases,
//             h[j] = sum_k WF_x[j][k] x~[ry][w*s_x + k],
//           where WF[j][k] = W[j][k - off_j] inside phase j's taps, else 0;
//   pass y  a thread owns VW adjacent columns of one window: it loads the
//           SPAN intermediate rows once and produces all R output rows.
//
// The zero-padded span-wide rows add only exact zeros to each sum, so
// results equal the per-output kernel for finite inputs.  Used for the
// interpolating methods (nearest keeps its exact one-tap copy).
#pragma once

#include "fcfs_fwd_tma.cuh"

namespace fcfs {
namespace {

// span-wide weight rows of one axis, WF[j][k], for the current channel
template <int R, int SPAN>
__device__ __forceinline__ void stage_span_weights(float* WF, const AxisP& A, int c) {
    for (int e = threadIdx.x; e < R * SPAN; e += blockDim.x) {
        const int j = e / SPAN, k = e - j * SPAN;
        const int t = k - A.off[j];
        float v = 0.f;
        if (t >= 0 && t < A.nt_src) v = A.learn ? A.w[(long long)c * A.w_cstride + j * A.nt_src + t] : A.wf[j * A.nt_src + t];
        WF[e] = v;
    }
}

template <int R>
__device__ __forceinline__ void sts_row(float* p, const float* h) {
    if (R == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(h[0], h[1], h[2], h[3]);
    } else if (R == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(h[0], h[1]);
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) p[j] = h[j];
    }
}

// XSPEC: window-per-thread x pass (lanes stride s_x samples: bank-conflict
// free for odd s_x, two-way when s_x samples span 8 bytes); otherwise one
// output column per thread.  XV: the s_x samples of a stride span exactly 8
// bytes and every window starts on such a boundary, so a window is read as
// 8-byte vectors (the lanes' loads contiguous, no conflicts) and only its
// SPAN samples enter the sums.
template <int R, int SPAN, typename Tin, typename Tout, int VW, bool XSPEC, bool XV>
__global__ void __launch_bounds__(256, 3) fcfs_fwd2d_rs(const __grid_constant__ TmaFwdParams T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ TileGeo sgeo[2];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    __shared__ float sWFx[R * SPAN], sWFy[R * SPAN];
    const FwdParams& P = T.P;
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    Tin* buf0 = reinterpret_cast<Tin*>(smem_raw);
    Tin* buf1 = reinterpret_cast<Tin*>(smem_raw + T.buf_bytes);
    float* sH = reinterpret_cast<float*>(smem_raw + 2 * T.buf_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);

    const int OX = P.OX, BW = T.BW, WX = P.WX;
    const int SX = AX.s, SY = AY.s;
    // x pass mapping
    const int XT = XSPEC ? WX : OX;  // threads per staged row
    const int G1 = blockDim.x / XT;
    const int xi = threadIdx.x % XT, g1 = threadIdx.x / XT;
    const bool x_active = g1 < G1;
    // y pass mapping: VW columns per thread, window groups
    const int NCOL = OX / VW;
    const int G2 = blockDim.x / NCOL;
    const int cy = threadIdx.x % NCOL, g2 = threadIdx.x / NCOL;
    const bool y_active = g2 < G2;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    const TileDeal deal = deal_tiles((int)T.ntiles, T.chunk);
    const int ntile = deal.n;
    if (ntile <= 0) return;
    // two tiles in flight from the start; each later copy starts once a tile's x pass has read its buffer
    if (threadIdx.x == 0) {
        sgeo[0] = tile_geo(T, deal.tile(0));
        issue_tile<Tin>(T, sgeo[0], buf0, &bars[0]);
        if (ntile > 1) {
            sgeo[1] = tile_geo(T, deal.tile(1));
            issue_tile<Tin>(T, sgeo[1], buf1, &bars[1]);
        }
    }
    const bool learn = AX.learn || AY.learn;
    int cur_c = -1;
    for (int k = 0; k < ntile; ++k) {
        Tin* buf = (k & 1) ? buf1 : buf0;
        if (!mbar_wait(&bars[k & 1], (uint32_t)((k >> 1) & 1), &g_status_fwd_tma)) s_abort = 1;
        __syncthreads();
        if (s_abort) {  // uniform: read after the barrier; this tile's and the prefetched copy in flight
            if (threadIdx.x == 0)
                drain_ring(bars, 2, k & 1, (uint32_t)((k >> 1) & 1), k + 1 < ntile ? 2 : 1, &g_status_fwd_tma);
            return;
        }
        const TileGeo geo = sgeo[k & 1];
        if (cur_c < 0 || (learn && geo.c != cur_c)) {
            stage_span_weights<R, SPAN>(sWFx, AX, geo.c);
            stage_span_weights<R, SPAN>(sWFy, AY, geo.c);
            __syncthreads();
            cur_c = geo.c;
        }
        if (geo.edge) fix_edges<Tin>(T, geo, buf);

        // ---- pass x
        if (x_active) {
            if (XSPEC) {
                if (xi < geo.nwx) {
                    float wf[R][SPAN];
#pragma unroll
                    for (int j = 0; j < R; ++j)
#pragma unroll
                        for (int q = 0; q < SPAN; ++q) wf[j][q] = sWFx[j * SPAN + q];
                    const Tin* src = buf + g1 * BW + geo.xoff + xi * SX;
                    float* dst = sH + g1 * OX + xi * R;
                    for (int ry = g1; ry < geo.rows; ry += G1) {
                        constexpr int VX = 8 / (int)sizeof(Tin);
                        constexpr int SPANL = XV ? (SPAN + VX - 1) / VX * VX : SPAN;
                        float v[SPANL];
                        if constexpr (XV) {
#pragma unroll
                            for (int q = 0; q < SPANL; q += VX) load_vec<VX, Tin>(src + q, v + q);
                        } else {
#pragma unroll
                            for (int q = 0; q < SPAN; ++q) v[q] = to_f<Tin>(src[q]);
                        }
                        float h[R];
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            float acc = -0.f;
#pragma unroll
                            for (int q = 0; q < SPAN; ++q) acc = fmaf(wf[j][q], v[q], acc);
                            h[j] = acc;
                        }
                        sts_row<R>(dst, h);
                        src += G1 * BW;
                        dst += G1 * OX;
                    }
                }
            } else {
                const int jx = xi % R, ixl = xi / R;
                if (ixl < geo.nwx) {
                    float wf[SPAN];
#pragma unroll
                    for (int q = 0; q < SPAN; ++q) wf[q] = sWFx[jx * SPAN + q];
                    const Tin* src = buf + g1 * BW + geo.xoff + ixl * SX;
                    float* dst = sH + g1 * OX + xi;
                    for (int ry = g1; ry < geo.rows; ry += G1) {
                        float acc = -0.f;
#pragma unroll
                        for (int q = 0; q < SPAN; ++q) acc = fmaf(wf[q], to_f<Tin>(src[q]), acc);
                        *dst = acc;
                        src += G1 * BW;
                        dst += G1 * OX;
                    }
                }
            }
        }
        __syncthreads();
        // this tile's buffer is read: the copy two tiles ahead goes into it
        if (threadIdx.x == 0 && k + 2 < ntile) {
            sgeo[k & 1] = tile_geo(T, deal.tile(k + 2));
            issue_tile<Tin>(T, sgeo[k & 1], buf, &bars[k & 1]);
        }

        // ---- pass y: VW columns x all R phases of a window per thread
        const int oxy = cy * VW;
        const int gox = geo.ix0 * R + oxy;
        const int nvalid = min(VW, AX.n_out - gox);
        if (y_active && oxy / R < geo.nwx && nvalid > 0) {
            float wf[R][SPAN];
#pragma unroll
            for (int j = 0; j < R; ++j)
#pragma unroll
                for (int q = 0; q < SPAN; ++q) wf[j][q] = sWFy[j * SPAN + q];
            Tout* ybase = static_cast<Tout*>(P.y) + (long long)geo.plane * AY.n_out * AX.n_out + gox;
            for (int iyl = g2; iyl < geo.nwy; iyl += G2) {
                const float* hp = sH + iyl * SY * OX + oxy;
                float v[SPAN][VW];
#pragma unroll
                for (int q = 0; q < SPAN; ++q) ldsv<VW>(hp + q * OX, v[q]);
                const int oy0 = (geo.iy0 + iyl) * R;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (oy0 + j >= AY.n_out) break;
                    float acc[VW];
#pragma unroll
                    for (int c = 0; c < VW; ++c) acc[c] = -0.f;
#pragma unroll
                    for (int q = 0; q < SPAN; ++q)
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc[c] = fmaf(wf[j][q], v[q][c], acc[c]);
                    if (epi_on(P.epi)) {
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc[c] = epi_apply(P.epi, geo.c, acc[c]);
                    }
                    storev(ybase + (oy0 + j) * AX.n_out, acc, nvalid);
                }
            }
        }
        __syncthreads();
    }
}

template <int R, int SPAN, typename Tin, typename Tout>
cudaError_t run_rs(const TmaFwdParams& T, cudaStream_t st) {
    const size_t smem = (size_t)T.bar_off + 16;
    const int no = T.P.ax[2].n_out;
    const uintptr_t y = (uintptr_t)T.P.y;
    // four columns per thread unless the weight rows already take many registers
    const bool v4 = R * SPAN <= 36 && T.P.OX % 4 == 0 && no % 4 == 0 && y % (4 * sizeof(Tout)) == 0;
    const bool v2 = T.P.OX % 2 == 0 && no % 2 == 0 && y % (2 * sizeof(Tout)) == 0;
    if (!v2) return cudaErrorInvalidValue;
    if (T.threads > 256) return cudaErrorInvalidValue;  // built for three 256-thread CTAs per SM
    // window per thread when lanes' windows (s_x samples apart) hit shared memory
    // banks at most two ways: odd s_x, or s_x samples within 8 bytes
    const int sx = T.P.ax[2].s;
    const bool xs = (sx % 2 == 1 || sx * (int)sizeof(Tin) <= 8) && T.P.WX <= (int)T.threads;
    // 8-byte vector window loads: the stride spans 8 bytes and every window starts on a multiple of
    // s_x samples of the (16-byte aligned) staged row, i.e. lo is a multiple of s_x
    const int lo = T.P.ax[2].lo;
    const bool xv = xs && sx * (int)sizeof(Tin) == 8 && ((lo % sx) + sx) % sx == 0;
    auto k = v4 ? (xv ? fcfs_fwd2d_rs<R, SPAN, Tin, Tout, 4, true, true>
                      : xs ? fcfs_fwd2d_rs<R, SPAN, Tin, Tout, 4, true, false> : fcfs_fwd2d_rs<R, SPAN, Tin, Tout, 4, false, false>)
                : (xv ? fcfs_fwd2d_rs<R, SPAN, Tin, Tout, 2, true, true>
                      : xs ? fcfs_fwd2d_rs<R, SPAN, Tin, Tout, 2, true, false> : fcfs_fwd2d_rs<R, SPAN, Tin, Tout, 2, false, false>);
    int sms = 0, per_sm = 0;
    cudaError_t e = resident_ctas((const void*)k, T.threads, smem, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(T.ntiles, (long long)sms * per_sm);
    k<<<(unsigned)grid, T.threads, smem, st>>>(T);
    return cudaGetLastError();
}

}  // namespace
}  // namespace fcfs
