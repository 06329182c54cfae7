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

// XSPEC: one adjoint window per thread in the x pass (lanes stride r samples).
// VW = 1: scalar loads (bank-conflict free for odd r or r * sizeof(Tg) <= 4).
// VW = r (r * sizeof(Tg) = 8 or 16 bytes): a window's samples are read as
// VW-aligned vectors, so the lanes' loads are contiguous; the planner takes
// this path only when every window starts on a VW boundary of the staged row
// (the adjoint's first g offset a multiple of r), and the x weight rows are
// the span rounded up to VW.
// Otherwise one intermediate column per thread.  Four CTAs per SM (at most 64
// registers a thread): the passes are latency-bound between barriers, and the
// extra resident CTAs measured faster than the larger register budget.
template <int S, int SPAN, int VW, typename Tg, typename Tx, bool XSPEC>
__global__ void __launch_bounds__(256, 4) fcfs_bwd_dx2d_rs(const __grid_constant__ TmaDxParams T) {
    constexpr int SPANX = (SPAN + VW - 1) / VW * VW;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    __shared__ float sWFx[S * SPANX], sWFy[S * SPAN];
    const AdjP& JX = T.aj[2];
    const AdjP& JY = T.aj[1];
    float* sF = reinterpret_cast<float*>(smem_raw + T.fx_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);
    const int NS = T.stages;
    const int QX = T.QX, GBW = T.GBW, FXP = T.FXP, R = JX.r;
    const int Nx = JX.n_x, Ny = JY.n_x;
    // x pass mapping
    const int XT = XSPEC ? T.WAcap : T.WAcap * S;
    const int G1 = blockDim.x / XT;
    const int xi = threadIdx.x % XT, g1 = threadIdx.x / XT;
    // y pass mapping
    const int G2 = blockDim.x / QX;
    const int cl = threadIdx.x % QX, g2 = threadIdx.x / QX;

    const int ntiles = (int)T.ntiles;
    const int per = (ntiles + gridDim.x - 1) / gridDim.x;
    int tile = blockIdx.x * per;
    const int tile_end = min(ntiles, tile + per);
    if (tile >= tile_end) return;
    // geometry of the tile in each stage, computed once by the thread that issues its copy
    __shared__ DxGeo sgeo[4];
    __shared__ DxWalk walk;  // the next tile to issue
    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
        s_abort = 0;
        dx_walk_init(T, walk, tile);
        for (int k = 0; k < NS && tile + k < tile_end; ++k) {
            sgeo[k] = dx_walk_geo(T, walk);
            issue<Tg>(T, sgeo[k], smem_raw + k * T.buf_bytes, &bars[k]);
            dx_walk_next(T, walk);
        }
    }
    __syncthreads();
    const bool learn = T.ax[2].learn || T.ax[1].learn;
    int cur_c = -1;
    int stg = 0;
    uint32_t phase = 0;
    for (; tile < tile_end; ++tile) {
        unsigned char* const bufk = smem_raw + stg * T.buf_bytes;
        const Tg* G0 = reinterpret_cast<const Tg*>(bufk);
        // one warp waits for the copy; the barrier releases the others
        if (threadIdx.x < 32 && !mbar_wait(&bars[stg], phase, &g_status_bwd_tma)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) drain_ring(bars, NS, stg, phase, min(NS, tile_end - tile), &g_status_bwd_tma);
            return;
        }
        const DxGeo geo = sgeo[stg];
        if (cur_c < 0 || (learn && geo.c != cur_c)) {
            // the previous tile ended with a barrier: no thread still reads the weights
            stage_adj_span<S, SPANX>(sWFx, T.ax[2], JX, geo.c, 0);
            stage_adj_span<S, SPAN>(sWFy, T.ax[1], JY, geo.c, 0);
            cur_c = geo.c;
            __syncthreads();
        }
        // windows start on VW boundaries (planner); a violation is reported, not read past
        if (VW > 1 && (geo.xoff & (VW - 1)) != 0) {
            if (threadIdx.x == 0) atomicOr(&g_status_bwd_tma, 4);
        }

        const int nAX = geo.X.ahi >= geo.X.alo ? geo.X.ahi - geo.X.alo + 1 : 0;
        const int nAY = geo.Y.ahi >= geo.Y.alo ? geo.Y.ahi - geo.Y.alo + 1 : 0;
        const int nGR = nAY ? (nAY - 1) * R + SPAN : 0;
        const int fxb = geo.X.alo * S + JX.lo_out;  // extended index of intermediate column 0
        // ---- pass x (adjoint along x) for every staged g row
        if (g1 < G1) {
            if (XSPEC) {
                if (xi < nAX) {
                    float wf[S][SPANX];
#pragma unroll
                    for (int u = 0; u < S; ++u)
#pragma unroll
                        for (int q = 0; q < SPANX; ++q) wf[u][q] = sWFx[u * SPANX + q];
                    const Tg* src = G0 + g1 * GBW + (geo.xoff & ~(VW - 1)) + xi * R;
                    float* dst = sF + g1 * FXP + xi * S;
                    for (int gr = g1; gr < nGR; gr += G1) {
                        float v[SPANX];
                        if constexpr (VW > 1) {
#pragma unroll
                            for (int q = 0; q < SPANX; q += VW) load_vec<VW, Tg>(src + q, v + q);
                        } else {
#pragma unroll
                            for (int q = 0; q < SPANX; ++q) v[q] = to_f<Tg>(src[q]);
                        }
#pragma unroll
                        for (int u = 0; u < S; ++u) {
                            float acc = 0.f;
#pragma unroll
                            for (int q = 0; q < SPANX; ++q) acc = fmaf(wf[u][q], v[q], acc);
                            dst[u] = acc;
                        }
                        src += G1 * GBW;
                        dst += G1 * FXP;
                    }
                }
            } else {
                const int aw = xi / S, u = xi - aw * S;
                if (aw < nAX) {
                    float wf[SPAN];
#pragma unroll
                    for (int q = 0; q < SPAN; ++q) wf[q] = sWFx[u * SPAN + q];
                    const Tg* src = G0 + g1 * GBW + geo.xoff + aw * R;
                    float* dst = sF + g1 * FXP + xi;
                    for (int gr = g1; gr < nGR; gr += G1) {
                        float acc = 0.f;
#pragma unroll
                        for (int q = 0; q < SPAN; ++q) acc = fmaf(wf[q], to_f<Tg>(src[q]), acc);
                        *dst = acc;
                        src += G1 * GBW;
                        dst += G1 * FXP;
                    }
                }
            }
        }
        __syncthreads();
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
        const bool ypath_smem = geo.Y.left || geo.Y.right || !geo.Y.covered;
        float* sO = reinterpret_cast<float*>(bufk);  // the g tile is consumed
        const int q = geo.qx0 + cl;
        const bool col_ok = g2 < G2 && cl < geo.nqx;
        const bool col_has = col_ok && q <= geo.X.vhi;
        Tx* xcol = static_cast<Tx*>(T.gx) + (long long)geo.plane * Ny * Nx + q;
        if (col_ok) {
            float wf[S][SPAN];
#pragma unroll
            for (int u = 0; u < S; ++u)
#pragma unroll
                for (int qq = 0; qq < SPAN; ++qq) wf[u][qq] = sWFy[u * SPAN + qq];
            const int fcol = q - fxb;
            for (int ay = g2; ay < nAY; ay += G2) {
                float v[SPAN];
                if (col_has) {
                    const float* src = sF + ay * R * FXP + fcol;
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
                    else store_out(xcol + (long long)vr * Nx, acc);
                }
            }
        }
        if (ypath_smem) {
            __syncthreads();
            if (col_ok) {
                for (int qy = geo.qy0 + g2; qy < geo.qy0 + geo.nqy; qy += G2) {
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
        if (threadIdx.x == 0 && tile + NS < tile_end) {
            sgeo[stg] = dx_walk_geo(T, walk);
            issue<Tg>(T, sgeo[stg], bufk, &bars[stg]);
            dx_walk_next(T, walk);
        }
        if (++stg == NS) {
            stg = 0;
            phase ^= 1;
        }
    }
}

template <int S, int SPAN, int VW, typename Tg>
cudaError_t run_rs(const TmaDxParams& T, cudaStream_t st) {
    constexpr int SPANX = (SPAN + VW - 1) / VW * VW;
    // measured: the variant pays off when the x pass can own whole windows
    // without bank conflicts and the weight rows stay small; otherwise the
    // per-output kernel is faster (and wider rows are not instantiated)
    if constexpr (S * SPANX > 40) {
        return cudaErrorInvalidValue;
    } else {
        const size_t smem = (size_t)T.bar_off + 8 * T.stages;
        auto k = fcfs_bwd_dx2d_rs<S, SPAN, VW, Tg, Tg, true>;
        if (T.WAcap > T.threads) return cudaErrorInvalidValue;
        int sms = 0, per_sm = 0;
        cudaError_t e = resident_ctas((const void*)k, T.threads, smem, &sms, &per_sm);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const long long grid = std::min<long long>(T.ntiles, (long long)sms * per_sm);
        k<<<(unsigned)grid, T.threads, smem, st>>>(T);
        return cudaGetLastError();
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
