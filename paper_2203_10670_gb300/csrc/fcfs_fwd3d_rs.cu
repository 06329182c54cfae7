// K3, register-blocked variant for a compile-time phase count R and window
// span SPAN shared by the three axes: the bulk-copy 3D forward of
// fcfs_fwd3d_tma.cu with the y and depth passes working per window:
//
//   pass x      one output column per thread (taps in registers),
//   pass y      a thread owns VW adjacent columns of one window: it loads the
//               SPAN intermediate rows once and writes all R output rows of
//               the window into the ring slot of the current plane;
//   pass depth  a thread owns VW adjacent columns of one output row: for a
//               depth window it loads the SPAN ring planes once and stores
//               all R output planes.
//
// The y and depth passes use span-wide weight rows WF[j][k] (W[j][k - off_j]
// inside phase j's taps, else 0); the zeros add exact zeros to each sum, so
// results equal the per-output kernel for finite inputs.  Used for the
// interpolating methods (nearest keeps its exact one-tap copy).
#include "fcfs_fwd3d_tma.cuh"

namespace fcfs {
namespace {

template <int R, int SPAN>
__device__ __forceinline__ void stage_span3(float* WF, const AxisP& A, int c) {
    for (int e = threadIdx.x; e < R * SPAN; e += blockDim.x) {
        const int j = e / SPAN, k = e - j * SPAN;
        const int t = k - A.off[j];
        float v = 0.f;
        if (t >= 0 && t < A.nt_src) v = A.learn ? A.w[(long long)c * A.w_cstride + j * A.nt_src + t] : A.wf[j * A.nt_src + t];
        WF[e] = v;
    }
}

template <int R, int SPAN, int NT, typename Tin, typename Tout, int VW>
__global__ void __launch_bounds__(256, 3) fcfs_fwd3d_rs(const __grid_constant__ TmaFwd3Params T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    __shared__ Cursor3 cur;
    __shared__ float sWFy[R * SPAN], sWFd[R * SPAN];
    const FwdParams& P = T.P;
    const AxisP &AD = P.ax[0], &AY = P.ax[1], &AX = P.ax[2];
    float* sH = reinterpret_cast<float*>(smem_raw + T.sh_off);
    float* ring = reinterpret_cast<float*>(smem_raw + T.ring_off);
    float* sWx = reinterpret_cast<float*>(smem_raw + T.w_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);
    const int S = T.stages;
    const int OX = P.OX, OY = P.OY, BW = T.BW;
    const int plane_sz = OY * OX;
    // pass x: one output column per thread
    const int G = blockDim.x / OX;
    const int ox = threadIdx.x % OX, g = threadIdx.x / OX;
    const bool act = g < G;
    const int jx = ox % R, ixl = ox / R;
    // passes y and depth: VW columns per thread
    const int NCOL = OX / VW;
    const int G2 = blockDim.x / NCOL;
    const int cy = threadIdx.x % NCOL, g2 = threadIdx.x / NCOL;
    const bool act2 = g2 < G2;
    const int oxy = cy * VW;

    const TileDeal deal = deal_tiles(T.ntiles, T.chunk);
    if (deal.n <= 0) return;
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
        s_abort = 0;
        cur.tile = 0;
        cur.g = geo3(T, deal.tile(0));
        cur.p = cur.g.p_first;
        cur.n = 0;
        cur.k = 0;
        for (int k = 0; k < S; ++k) issue_next<Tin>(T, cur, deal, smem_raw, bars);
    }
    __syncthreads();
    const bool learn = AX.learn || AY.learn || AD.learn;
    int cur_c = -1;
    int k = 0;           // stage of the current job
    uint32_t phase = 0;  // its barrier phase
    int consumed = 0;    // jobs taken so far (cur.n were issued)
    for (int kt = 0; kt < deal.n; ++kt) {
        const Geo3 geo = geo3(T, deal.tile(kt));
        if (cur_c < 0 || (learn && geo.c != cur_c)) {
            // the previous tile ended with a barrier: no thread still reads the weights
            stage3<NT>(sWx, AX, geo.c);
            stage_span3<R, SPAN>(sWFy, AY, geo.c);
            stage_span3<R, SPAN>(sWFd, AD, geo.c);
            cur_c = geo.c;
        }
        const int gox = geo.ix0 * R + oxy;
        const int nvalid = min(VW, AX.n_out - gox);
        const bool col2 = act2 && oxy / R < geo.nwx && nvalid > 0;
        const int noy = min(geo.nwy * R, AY.n_out - geo.iy0 * R);
        int idl = 0;
        int rslot = 0;  // ring slot of plane p
        for (int p = geo.p_first; p <= geo.p_last; ++p) {
            Tin* buf = reinterpret_cast<Tin*>(smem_raw + k * T.buf_bytes);
            // one warp waits for the copy; the barrier releases the others
            if (threadIdx.x < 32 && !mbar_wait(&bars[k], phase, &g_status_fwd3d)) s_abort = 1;
            __syncthreads();
            if (s_abort) {
                if (threadIdx.x == 0) drain_ring(bars, S, k, phase, cur.n - consumed, &g_status_fwd3d);
                return;
            }
            ++consumed;
            const int sd = ext_index(p, AD.n_in, P.pad);
            if (sd < 0) {  // a whole plane of the constant
                const Tin cv = from_f<Tin>(P.padv);
                for (int e = threadIdx.x; e < T.BW * T.BH; e += blockDim.x) buf[e] = cv;
                __syncthreads();
            } else if (geo.edge) {
                fix_edges3<Tin>(T, geo, buf, sd);
            }
            // ---- pass x
            if (act && ixl < geo.nwx) {
                float w[NT];
#pragma unroll
                for (int t = 0; t < NT; ++t) w[t] = sWx[jx * NT + t];
                const Tin* src = buf + g * BW + geo.xoff + ixl * AX.s + AX.off[jx];
                float* dst = sH + g * OX + ox;
                for (int ry = g; ry < geo.rows; ry += G) {
                    float acc = -0.f;
#pragma unroll
                    for (int t = 0; t < NT; ++t) acc = fmaf(w[t], to_f<Tin>(src[t]), acc);
                    *dst = acc;
                    src += G * BW;
                    dst += G * OX;
                }
            }
            __syncthreads();
            // ---- pass y: all R rows of a window into the ring slot of plane p
            float* slot = ring + rslot * plane_sz;
            if (col2) {
                float wf[R][SPAN];
#pragma unroll
                for (int j = 0; j < R; ++j)
#pragma unroll
                    for (int q = 0; q < SPAN; ++q) wf[j][q] = sWFy[j * SPAN + q];
                for (int iyl = g2; iyl < geo.nwy; iyl += G2) {
                    const float* hp = sH + iyl * AY.s * OX + oxy;
                    float v[SPAN][VW];
#pragma unroll
                    for (int q = 0; q < SPAN; ++q) ldsv<VW>(hp + q * OX, v[q]);
                    float* dst = slot + iyl * R * OX + oxy;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        float acc[VW];
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc[c] = -0.f;
#pragma unroll
                        for (int q = 0; q < SPAN; ++q)
#pragma unroll
                            for (int c = 0; c < VW; ++c) acc[c] = fmaf(wf[j][q], v[q][c], acc[c]);
                        storev(dst + j * OX, acc, VW);
                    }
                }
            }
            __syncthreads();
            // ---- pass depth: every window whose planes are all in the ring
            while (idl < geo.nwd && (geo.id0 + idl) * AD.s + AD.lo + AD.span <= p + 1) {
                const int id = geo.id0 + idl;
                const int odb = id * R;
                if (col2) {
                    float wf[R][SPAN];
#pragma unroll
                    for (int j = 0; j < R; ++j)
#pragma unroll
                        for (int q = 0; q < SPAN; ++q) wf[j][q] = sWFd[j * SPAN + q];
                    // the window completes at plane p: its plane q sits in slot (rslot + 1 + q) mod SPAN
                    const float* rp[SPAN];
#pragma unroll
                    for (int q = 0; q < SPAN; ++q) {
                        int sl = rslot + 1 + q;
                        if (sl >= SPAN) sl -= SPAN;
                        rp[q] = ring + sl * plane_sz + oxy;
                    }
                    const long long oplane = (long long)AY.n_out * AX.n_out;
                    Tout* yv = static_cast<Tout*>(P.y) + (long long)geo.plane * AD.n_out * oplane +
                               (long long)geo.iy0 * R * AX.n_out + gox;
                    const int nj = min(R, AD.n_out - odb);
                    for (int oyl = g2; oyl < noy; oyl += G2) {
                        float v[SPAN][VW];
#pragma unroll
                        for (int q = 0; q < SPAN; ++q) ldsv<VW>(rp[q] + oyl * OX, v[q]);
                        Tout* yo = yv + (long long)odb * oplane + (long long)oyl * AX.n_out;
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if (j >= nj) break;
                            float acc[VW];
#pragma unroll
                            for (int c = 0; c < VW; ++c) acc[c] = -0.f;
#pragma unroll
                            for (int q = 0; q < SPAN; ++q)
#pragma unroll
                                for (int c = 0; c < VW; ++c) acc[c] = fmaf(wf[j][q], v[q][c], acc[c]);
                            storev(yo + j * oplane, acc, nvalid);
                        }
                    }
                }
                ++idl;
            }
            __syncthreads();  // ring slots, sH and this stage are free again
            if (threadIdx.x == 0) issue_next<Tin>(T, cur, deal, smem_raw, bars);
            if (++rslot == P.ring) rslot = 0;
            if (++k == S) {
                k = 0;
                phase ^= 1;
            }
        }
    }
}

template <int R, int SPAN, int NT, typename Tin, typename Tout>
cudaError_t run_rs3(const TmaFwd3Params& T, cudaStream_t st) {
    const size_t smem = (size_t)T.bar_off + 8 * T.stages;
    const int no = T.P.ax[2].n_out;
    const uintptr_t y = (uintptr_t)T.P.y;
    const bool v4 = T.P.OX % 4 == 0 && no % 4 == 0 && y % (4 * sizeof(Tout)) == 0;
    const bool v2 = T.P.OX % 2 == 0 && no % 2 == 0 && y % (2 * sizeof(Tout)) == 0;
    if (!v2 || T.threads > 256) return cudaErrorInvalidValue;
    auto k = v4 ? fcfs_fwd3d_rs<R, SPAN, NT, Tin, Tout, 4> : fcfs_fwd3d_rs<R, SPAN, NT, Tin, Tout, 2>;
    int sms = 0, per_sm = 0;
    cudaError_t e = resident_ctas((const void*)k, T.threads, smem, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(T.ntiles, (long long)sms * per_sm);
    k<<<(unsigned)grid, T.threads, smem, st>>>(T);
    return cudaGetLastError();
}

}  // namespace

// (R, span, taps) triples with a compiled instance: bilinear 2/1, 3/2, 4/3,
// 2/3 and bicubic 3/2
#define FCFS_FWD3_RS_CASES(X) X(2, 2, 2) X(3, 3, 2) X(4, 4, 2) X(2, 3, 2) X(3, 5, 4)

// The register-blocked 3D forward for this plan, or cudaErrorInvalidValue
// when no instance matches (same phase count, span and taps on all axes,
// interpolating weights, F32 or BF16 storage in and out).
cudaError_t launch_forward3d_rs(const TmaFwd3Params& T, int din, int dout, cudaStream_t st) {
    const AxisP &A0 = T.P.ax[0], &A1 = T.P.ax[1], &A2 = T.P.ax[2];
    if (din != dout || (din != FCFS_F32 && din != FCFS_BF16)) return cudaErrorInvalidValue;
    if (A0.r != A2.r || A1.r != A2.r || A0.span != A2.span || A1.span != A2.span) return cudaErrorInvalidValue;
    if (A2.nt_src == 1 && !A2.learn) return cudaErrorInvalidValue;  // nearest: exact one-tap copy elsewhere
    const int R = A2.r, SP = A2.span, NT = A2.nt;
#define CASE(r, sp, nt)                                                                    \
    if (R == r && SP == sp && NT == nt)                                                    \
        return din == FCFS_F32 ? run_rs3<r, sp, nt, float, float>(T, st)                   \
                               : run_rs3<r, sp, nt, __nv_bfloat16, __nv_bfloat16>(T, st);
    FCFS_FWD3_RS_CASES(CASE)
#undef CASE
    return cudaErrorInvalidValue;
}

int read_status_fwd3d_rs(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_fwd3d, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_fwd3d, &z, sizeof(int));
    }
    return v;
}

}  // namespace fcfs
