// K4, register-blocked variant: the input gradient with both adjoint passes
// working per adjoint window (compile-time phase count S = s and window span
// SPAN, the same on both axes).  A thread loads the SPAN samples an adjoint
// window reads once and produces all S outputs from span-wide zero-padded
// weight rows WF[u][k] held in registers.  Intermediate columns are indexed
// relative to the tile's first adjoint window, so whole windows are written
// without bounds tests; edge tiles fold the virtual indices as the
// per-output kernel does.
#include <type_traits>

#include "fcfs_bwd_tma.cuh"

namespace fcfs {
namespace {

// span-wide adjoint weight rows of one axis for channel c, shifted right by
// `shift` positions inside rows of W entries (zero outside the taps)
template <int S, int W>
__device__ __forceinline__ void stage_adj_span(float* WF, const AxisP& A, const AdjP& J, int c, int shift) {
    for (int e = threadIdx.x; e < S * W; e += blockDim.x) {
        const int u = e / W, k = e - u * W;
        const int t = k - shift - J.off[u];
        float v = 0.f;
        if (t >= 0 && t < J.ntu[u]) {
            const int f = J.idx[u * kMaxAdjTaps + t];
            if (f >= 0) v = fwd_weight(A, c, f);
        }
        WF[e] = v;
    }
}

// x pass: one adjoint window per thread (lanes stride r samples).  VW = 1:
// scalar loads (bank-conflict free for odd r or r * sizeof(Tg) <= 4).  VW = r
// (r * sizeof(Tg) = 8 or 16 bytes): a window's samples are read as
// VW-aligned vectors, so the lanes' loads are contiguous; the planner takes
// this path only when every window starts on a VW boundary of the staged row
// (the adjoint's first g offset a multiple of r).  The window's samples are
// summed in tap pairs with packed FP32 FMAs (even and odd taps in the two
// lanes of a pair, added at the end), so the x weight rows are the span
// rounded up to an even count (and to VW).
//
// y pass: YV = 4 adjacent real columns per thread.  Their intermediate
// values are read as one vector per row and each sum runs in the lanes of
// packed FMAs against duplicated weight pairs, in tap order; the YV outputs
// of a row are one vector store.  The intermediate rows are laid out so the
// tile's first real column starts on a 16-byte boundary.  YV = 1: one column
// per thread with scalar FMAs (rows whose length is not a multiple of four).
//
// Two CTAs per SM (the staged tiles take about 110 KB of shared memory), so
// up to 128 registers a thread.
template <int S, int SPAN, int VW, typename Tg, int YV>
__global__ void __launch_bounds__(256, 2) fcfs_bwd_dx2d_rs(const __grid_constant__ TmaDxParams T) {
    constexpr int VP = VW > 2 ? VW : 2;
    constexpr int SPANX = (SPAN + VP - 1) / VP * VP;
    constexpr int NP = SPANX / 2;  // tap pairs of the x pass
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    __shared__ __align__(16) float sWFx[S * SPANX];
    __shared__ float sWFy[S * SPAN];
    __shared__ __align__(16) float2 sWY2[S * SPAN];  // the y weights, each duplicated into a pair
    const AdjP& JX = T.aj[2];
    const AdjP& JY = T.aj[1];
    float* sF = reinterpret_cast<float*>(smem_raw + T.fx_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);
    const int NS = T.stages;
    const int QX = T.QX, GBW = T.GBW, FXP = T.FXP, R = JX.r;
    const int Nx = JX.n_x, Ny = JY.n_x;
    // x pass mapping: a row of windows per group of WAcap threads
    const int XT = T.WAcap;
    const int G1 = blockDim.x / XT;
    const int xi = threadIdx.x % XT, g1 = threadIdx.x / XT;
    // y pass mapping: YV columns per thread, groups over the adjoint windows
    const int NCY = QX / YV;
    const int G2 = blockDim.x / NCY;
    const int cy = threadIdx.x % NCY, g2 = threadIdx.x / NCY;
    // second stage of edge tiles (fold in y): one column per thread
    const int G3 = blockDim.x / QX;
    const int cl = threadIdx.x % QX, g3 = threadIdx.x / QX;

    const TileDeal deal = deal_tiles((int)T.ntiles, T.chunk);
    const int ntile = deal.n;
    auto tile_of = [&](int k) { return deal.tile(k); };
    if (ntile <= 0) return;
    // geometry of the tile in each stage, computed once by the thread that issues its copy
    __shared__ DxGeo sgeo[4];
    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
        s_abort = 0;
        for (int k = 0; k < NS && k < ntile; ++k) {
            sgeo[k] = dx_geo(T, tile_of(k));
            issue<Tg>(T, sgeo[k], smem_raw + k * T.buf_bytes, &bars[k]);
        }
    }
    __syncthreads();
    const bool learn = T.ax[2].learn || T.ax[1].learn;
    int cur_c = -1;
    // the weights stay in registers across tiles (reloaded when the channel changes)
    float2 wf[S][NP];       // x: tap pairs
    // y: each tap duplicated into a pair; wide weight sets are read from shared memory per use
    constexpr bool HOLD_Y = YV > 1 && S * SPAN <= 24;
    float2 wy[HOLD_Y ? S : 1][HOLD_Y ? SPAN : 1];
    int stg = 0;
    uint32_t phase = 0;
    for (int k = 0; k < ntile; ++k) {
        unsigned char* const bufk = smem_raw + stg * T.buf_bytes;
        const Tg* G0 = reinterpret_cast<const Tg*>(bufk);
        // one warp waits for the copy; the barrier releases the others
        if (threadIdx.x < 32 && !mbar_wait(&bars[stg], phase, &g_status_bwd_tma)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) drain_ring(bars, NS, stg, phase, min(NS, ntile - k), &g_status_bwd_tma);
            return;
        }
        const DxGeo geo = sgeo[stg];
        if (cur_c < 0 || (learn && geo.c != cur_c)) {
            // the previous tile ended with a barrier: no thread still reads the weights
            stage_adj_span<S, SPANX>(sWFx, T.ax[2], JX, geo.c, 0);
            stage_adj_span<S, SPAN>(sWFy, T.ax[1], JY, geo.c, 0);
            __syncthreads();
            for (int e = threadIdx.x; e < S * SPAN; e += blockDim.x) sWY2[e] = make_float2(sWFy[e], sWFy[e]);
            cur_c = geo.c;
            __syncthreads();
#pragma unroll
            for (int u = 0; u < S; ++u)
#pragma unroll
                for (int p = 0; p < NP; ++p) wf[u][p] = *reinterpret_cast<const float2*>(sWFx + u * SPANX + 2 * p);
            if constexpr (HOLD_Y) {
#pragma unroll
                for (int u = 0; u < S; ++u)
#pragma unroll
                    for (int qq = 0; qq < SPAN; ++qq) wy[u][qq] = sWY2[u * SPAN + qq];
            }
        }
        // windows start on VW boundaries (planner); a violation is reported, not read past
        if (VW > 1 && (geo.xoff & (VW - 1)) != 0) {
            if (threadIdx.x == 0) atomicOr(&g_status_bwd_tma, 4);
        }

        const int nAX = geo.X.ahi >= geo.X.alo ? geo.X.ahi - geo.X.alo + 1 : 0;
        const int nAY = geo.Y.ahi >= geo.Y.alo ? geo.Y.ahi - geo.Y.alo + 1 : 0;
        const int nGR = nAY ? (nAY - 1) * R + SPAN : 0;
        // intermediate column of extended index v: v - fxb, with fxb = fxw - sh, where fxw is the
        // extended index of the first adjoint window's first output and sh puts the tile's first
        // real column on a multiple of four
        const int fxw = geo.X.alo * S + JX.lo_out;
        const int sh = (fxw - geo.qx0) & 3;
        const int fxb = fxw - sh;
        // ---- pass x (adjoint along x) for every staged g row, tap pairs in packed FMAs
        if (g1 < G1 && xi < nAX) {
            const Tg* src = G0 + g1 * GBW + (geo.xoff & ~(VW - 1)) + xi * R;
            float* dst = sF + g1 * FXP + sh + xi * S;
            // two rows per step (independent chains in flight); the second is skipped past the end
            for (int gr = g1; gr < nGR; gr += 2 * G1) {
                const bool two = gr + G1 < nGR;
                float v[2][SPANX];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const Tg* sk = src + (two ? k : 0) * G1 * GBW;
                    if constexpr (VW > 1) {
#pragma unroll
                        for (int q = 0; q < SPANX; q += VW) load_vec<VW, Tg>(sk + q, v[k] + q);
                    } else {
#pragma unroll
                        for (int q = 0; q < SPANX; ++q) v[k][q] = to_f<Tg>(sk[q]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float o[S];
#pragma unroll
                    for (int u = 0; u < S; ++u) {
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int p = 0; p < NP; ++p)
                            acc = __ffma2_rn(wf[u][p], make_float2(v[k][2 * p], v[k][2 * p + 1]), acc);
                        o[u] = acc.x + acc.y;
                    }
                    if (k == 0 || two) {
#pragma unroll
                        for (int u = 0; u < S; ++u) dst[k * G1 * FXP + u] = o[u];
                    }
                }
                src += 2 * G1 * GBW;
                dst += 2 * G1 * FXP;
            }
        }
        __syncthreads();
        // the g tile is consumed: a tile whose y pass does not stage its outputs in this buffer
        // lets the copy NS tiles ahead start now
        const bool ypath_smem = geo.Y.left || geo.Y.right || !geo.Y.covered;
        const bool early = !ypath_smem;
        if (early && threadIdx.x == 0 && k + NS < ntile) {
            sgeo[stg] = dx_geo(T, tile_of(k + NS));
            issue<Tg>(T, sgeo[stg], bufk, &bars[stg]);
        }
        // ---- fold x: virtual columns onto the real column the padding maps them to
        if (geo.X.left || geo.X.right) {
            for (int gr = threadIdx.x; gr < nGR; gr += blockDim.x) {
                float* row = sF + gr * FXP;
                const int l1 = min(geo.X.vhi, -1), r0 = max(geo.X.vlo, Nx);
                for (int v = geo.X.vlo; v <= l1; ++v) {
                    const int q = ext_index(v, Nx, T.pad);
                    if (q >= geo.qx0 && q < geo.qx0 + geo.nqx) row[q - fxb] += row[v - fxb];
                }
                for (int v = r0; v <= geo.X.vhi; ++v) {
                    const int q = ext_index(v, Nx, T.pad);
                    if (q >= geo.qx0 && q < geo.qx0 + geo.nqx) row[q - fxb] += row[v - fxb];
                }
            }
            __syncthreads();
        }
        // ---- pass y (adjoint along y) on the tile's real columns
        float* sO = reinterpret_cast<float*>(bufk);  // the g tile is consumed
        Tg* const xplane = static_cast<Tg*>(T.gx) + (long long)geo.plane * Ny * Nx;
        if constexpr (YV > 1) {
            const int q = geo.qx0 + cy * YV;
            const int nv = min(YV, geo.qx0 + geo.nqx - q);  // columns of this thread inside the tile
            const int nh = min(nv, geo.X.vhi - q + 1);      // of which the intermediate holds values
            if (g2 < G2 && nv > 0) {
                const float* colp = sF + (q - fxb);
                for (int ay = g2; ay < nAY; ay += G2) {
                    const float* src = colp + ay * R * FXP;
                    float2 acc[S][YV / 2];
#pragma unroll
                    for (int u = 0; u < S; ++u)
#pragma unroll
                        for (int h = 0; h < YV / 2; ++h) acc[u][h] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int qq = 0; qq < SPAN; ++qq) {
                        float v[YV];
                        ldsv<YV>(src + qq * FXP, v);
                        if (nh < YV) {
#pragma unroll
                            for (int k = 0; k < YV; ++k) v[k] = k < nh ? v[k] : 0.f;
                        }
#pragma unroll
                        for (int u = 0; u < S; ++u)
#pragma unroll
                            for (int h = 0; h < YV / 2; ++h)
                                acc[u][h] = __ffma2_rn(HOLD_Y ? wy[HOLD_Y ? u : 0][HOLD_Y ? qq : 0] : sWY2[u * SPAN + qq],
                                                       make_float2(v[2 * h], v[2 * h + 1]), acc[u][h]);
                    }
                    const int vb = (geo.Y.alo + ay) * S + JY.lo_out;
#pragma unroll
                    for (int u = 0; u < S; ++u) {
                        const int vr = vb + u;
                        if (vr < geo.Y.vlo || vr > geo.Y.vhi) continue;
                        float o[YV];
#pragma unroll
                        for (int h = 0; h < YV / 2; ++h) o[2 * h] = acc[u][h].x, o[2 * h + 1] = acc[u][h].y;
                        if (ypath_smem) {
                            float* p = sO + (vr - geo.Y.vlo) * QX + cy * YV;
                            if (nv == YV) storev(p, o, YV);
                            else for (int k = 0; k < nv; ++k) p[k] = o[k];
                        } else {
                            storev(xplane + (long long)vr * Nx + q, o, nv);
                        }
                    }
                }
            }
        } else {
            const int q = geo.qx0 + cl;
            const bool col_ok = g3 < G3 && cl < geo.nqx;
            const bool col_has = col_ok && q <= geo.X.vhi;
            if (col_ok) {
                float wf[S][SPAN];
#pragma unroll
                for (int u = 0; u < S; ++u)
#pragma unroll
                    for (int qq = 0; qq < SPAN; ++qq) wf[u][qq] = sWFy[u * SPAN + qq];
                for (int ay = g3; ay < nAY; ay += G3) {
                    float v[SPAN];
                    if (col_has) {
                        const float* src = sF + ay * R * FXP + (q - fxb);
#pragma unroll
                        for (int qq = 0; qq < SPAN; ++qq) v[qq] = src[qq * FXP];
                    } else {
#pragma unroll
                        for (int qq = 0; qq < SPAN; ++qq) v[qq] = 0.f;
                    }
                    const int vb = (geo.Y.alo + ay) * S + JY.lo_out;
#pragma unroll
                    for (int u = 0; u < S; ++u) {
                        const int vr = vb + u;
                        if (vr < geo.Y.vlo || vr > geo.Y.vhi) continue;
                        float acc = 0.f;
#pragma unroll
                        for (int qq = 0; qq < SPAN; ++qq) acc = fmaf(wf[u][qq], v[qq], acc);
                        if (ypath_smem) sO[(vr - geo.Y.vlo) * QX + cl] = acc;
                        else store_out(xplane + (long long)vr * Nx + q, acc);
                    }
                }
            }
        }
        if (ypath_smem) {
            __syncthreads();
            if (g3 < G3 && cl < geo.nqx) {
                Tg* xcol = xplane + geo.qx0 + cl;
                for (int qy = geo.qy0 + g3; qy < geo.qy0 + geo.nqy; qy += G3) {
                    float acc = (qy >= geo.Y.vlo && qy <= geo.Y.vhi) ? sO[(qy - geo.Y.vlo) * QX + cl] : 0.f;
                    if (geo.Y.left || geo.Y.right) {
                        const int l1 = min(geo.Y.vhi, -1), r0 = max(geo.Y.vlo, Ny);
                        for (int v = geo.Y.vlo; v <= l1; ++v)
                            if (ext_index(v, Ny, T.pad) == qy) acc += sO[(v - geo.Y.vlo) * QX + cl];
                        for (int v = r0; v <= geo.Y.vhi; ++v)
                            if (ext_index(v, Ny, T.pad) == qy) acc += sO[(v - geo.Y.vlo) * QX + cl];
                    }
                    store_out(xcol + (long long)qy * Nx, acc);
                }
            }
        }
        __syncthreads();  // sF and this stage are free again
        if (!early && threadIdx.x == 0 && k + NS < ntile) {
            sgeo[stg] = dx_geo(T, tile_of(k + NS));
            issue<Tg>(T, sgeo[stg], bufk, &bars[stg]);
        }
        if (++stg == NS) {
            stg = 0;
            phase ^= 1;
        }
    }
}

template <int S, int SPAN, int VW, typename Tg, int YV>
cudaError_t launch_rs(const TmaDxParams& T, cudaStream_t st) {
    const size_t smem = (size_t)T.bar_off + 8 * T.stages;
    auto k = fcfs_bwd_dx2d_rs<S, SPAN, VW, Tg, YV>;
    int sms = 0, per_sm = 0;
    cudaError_t e = resident_ctas((const void*)k, T.threads, smem, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(T.ntiles, (long long)sms * per_sm);
    k<<<(unsigned)grid, T.threads, smem, st>>>(T);
    return cudaGetLastError();
}

template <int S, int SPAN, int VW, typename Tg>
cudaError_t run_rs(const TmaDxParams& T, cudaStream_t st) {
    constexpr int VP = VW > 2 ? VW : 2;
    constexpr int SPANX = (SPAN + VP - 1) / VP * VP;
    // measured: the variant pays off when the x pass can own whole windows
    // without bank conflicts and the weight rows stay small; otherwise the
    // per-output kernel is faster (and wider rows are not instantiated)
    if constexpr (S * SPANX > 40) {
        return cudaErrorInvalidValue;
    } else {
        if (T.WAcap > T.threads || T.QX % 4 != 0) return cudaErrorInvalidValue;
        // y pass vector width: rows of gx a multiple of YV elements and the base aligned to YV elements
        const int Nx = T.aj[2].n_x;
        const uintptr_t gx = (uintptr_t)T.gx;
        if (Nx % 4 == 0 && gx % (4 * sizeof(Tg)) == 0) return launch_rs<S, SPAN, VW, Tg, 4>(T, st);
        return launch_rs<S, SPAN, VW, Tg, 1>(T, st);
    }
}

}  // namespace

#define FCFS_DX_RS_PAIRS(X) X(4, 10) X(2, 7) X(2, 4) X(3, 4) X(3, 8)

bool dx_rs_compiled(int S, int span) {
#define CASE(a, b) \
    if (S == a && span == b) return true;
    FCFS_DX_RS_PAIRS(CASE)
#undef CASE
    return false;
}

// x-pass vector width for adjoint stride r and element size es: 1 when scalar
// loads are bank-conflict free, r when a window's samples form 8- or 16-byte
// vectors, 0 when neither holds
int dx_rs_vector_width(int r, int es) {
    if (r % 2 == 1 || r * es <= 4) return 1;
    if (r * es == 8 || r * es == 16) return r;
    return 0;
}

cudaError_t launch_dx_rs(const TmaDxParams& T, int dt, cudaStream_t st) {
    const int S = T.aj[2].s, span = T.rs_span, vw = T.rs_vw;
#define CASE(a, b)                                                    \
    if (S == a && span == b) {                                        \
        if (dt == FCFS_F32) {                                         \
            if (vw == 1) return run_rs<a, b, 1, float>(T, st);        \
            if (vw == 2) return run_rs<a, b, 2, float>(T, st);        \
            if (vw == 4) return run_rs<a, b, 4, float>(T, st);        \
        } else {                                                      \
            if (vw == 1) return run_rs<a, b, 1, __nv_bfloat16>(T, st); \
            if (vw == 4) return run_rs<a, b, 4, __nv_bfloat16>(T, st); \
        }                                                             \
        return cudaErrorInvalidValue;                                 \
    }
    FCFS_DX_RS_PAIRS(CASE)
#undef CASE
    return cudaErrorInvalidValue;
}

int read_status_bwd_rs(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_bwd_tma, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_bwd_tma, &z, sizeof(int));
    }
    return v;
}

}  // namespace fcfs
