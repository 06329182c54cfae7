// K3 (fast path): persistent, bulk-copy staged 3D forward (Sec. 4 with
// separable per-axis kernels).  A CTA walks (y, x, depth-chunk) tiles; the
// input depth planes a tile needs form a stream of jobs, each a TMA box of
// one plane (depth coordinate remapped by the padding rule), double-buffered
// so the next plane lands while the current one is interpolated along x and
// y into a ring of span_d planes.  Whenever the ring holds a depth window's
// planes, the depth taps produce that window's r_d output planes.
#include "fcfs_fwd3d_tma.cuh"

namespace fcfs {
namespace {

template <int NT, typename Tin, typename Tout>
__global__ void __launch_bounds__(256, 3) fcfs_fwd3d_tma(const __grid_constant__ TmaFwd3Params T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    __shared__ Cursor3 cur;
    const FwdParams& P = T.P;
    const AxisP &AD = P.ax[0], &AY = P.ax[1], &AX = P.ax[2];
    float* sH = reinterpret_cast<float*>(smem_raw + T.sh_off);
    float* ring = reinterpret_cast<float*>(smem_raw + T.ring_off);
    float* sWx = reinterpret_cast<float*>(smem_raw + T.w_off);
    float* sWy = sWx + AX.r * NT;
    float* sWd = sWy + AY.r * NT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);
    const int S = T.stages;
    const int OX = P.OX, OY = P.OY, BW = T.BW;
    const int plane_sz = OY * OX;
    const int G = blockDim.x / OX;
    const int ox = threadIdx.x % OX, g = threadIdx.x / OX;
    const bool act = g < G;
    const int jx = ox % AX.r, ixl = ox / AX.r;

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
            stage3<NT>(sWy, AY, geo.c);
            stage3<NT>(sWd, AD, geo.c);
            cur_c = geo.c;
        }
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
            // ---- x taps
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
            // ---- y taps into the ring slot of plane p
            float* slot = ring + rslot * plane_sz;
            if (act && ixl < geo.nwx) {
                for (int jy = 0; jy < AY.r; ++jy) {
                    float w[NT];
#pragma unroll
                    for (int t = 0; t < NT; ++t) w[t] = sWy[jy * NT + t];
                    const float* col = sH + AY.off[jy] * OX + ox;
                    float* dst = slot + jy * OX + ox;
                    for (int iyl = g; iyl < geo.nwy; iyl += G) {
                        const float* c2 = col + iyl * AY.s * OX;
                        float acc = -0.f;
#pragma unroll
                        for (int t = 0; t < NT; ++t) acc = fmaf(w[t], c2[t * OX], acc);
                        dst[iyl * AY.r * OX] = acc;
                    }
                }
            }
            __syncthreads();
            // ---- depth taps for every window whose planes are all in the ring
            while (idl < geo.nwd && (geo.id0 + idl) * AD.s + AD.lo + AD.span <= p + 1) {
                const int id = geo.id0 + idl;
                const int odb = id * AD.r;
                const int gox = geo.ix0 * AX.r + ox;
                if (act && ixl < geo.nwx && gox < AX.n_out) {
                    const long long oplane = (long long)AY.n_out * AX.n_out;
                    const int noy = min(geo.nwy * AY.r, AY.n_out - geo.iy0 * AY.r);
                    Tout* yv = static_cast<Tout*>(P.y) + (long long)geo.plane * AD.n_out * oplane +
                               (long long)geo.iy0 * AY.r * AX.n_out + gox;
                    for (int jd = 0; jd < AD.r && odb + jd < AD.n_out; ++jd) {
                        // the window completes at plane p: its plane k sits in slot (rslot + 1 + k) mod ring
                        const int sb = rslot + 1 + AD.off[jd];
                        float w[NT];
                        const float* rp[NT];
#pragma unroll
                        for (int t = 0; t < NT; ++t) {
                            w[t] = sWd[jd * NT + t];
                            int sl = sb + t;
                            if (sl >= P.ring) sl -= P.ring;
                            if (sl >= P.ring) sl -= P.ring;
                            rp[t] = ring + sl * plane_sz + ox;
                        }
                        Tout* yo = yv + (long long)(odb + jd) * oplane;
                        for (int oyl = g; oyl < noy; oyl += G) {
                            float acc = -0.f;
#pragma unroll
                            for (int t = 0; t < NT; ++t) acc = fmaf(w[t], rp[t][oyl * OX], acc);
                            yo[(long long)oyl * AX.n_out] = from_f<Tout>(acc);
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

template <int NT, typename Tin, typename Tout>
cudaError_t run3(const TmaFwd3Params& T, cudaStream_t st) {
    const size_t smem = (size_t)T.bar_off + 8 * T.stages;
    if (T.threads > 256) return cudaErrorInvalidValue;
    auto k = fcfs_fwd3d_tma<NT, Tin, Tout>;
    int sms = 0, per_sm = 0;
    cudaError_t e = resident_ctas((const void*)k, T.threads, smem, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(T.ntiles, (long long)sms * per_sm);
    k<<<(unsigned)grid, T.threads, smem, st>>>(T);
    return cudaGetLastError();
}

}  // namespace

#define FCFS_NT3_CASES(X) X(1) X(2) X(3) X(4) X(5)

cudaError_t launch_forward3d_tma(const TmaFwd3Params& T, int nt, int din, int dout, cudaStream_t st) {
    auto go = [&](auto ti, auto to) -> cudaError_t {
        using Tin = std::remove_pointer_t<decltype(ti)>;
        using Tout = std::remove_pointer_t<decltype(to)>;
        switch (nt) {
#define CASE(N) \
    case N: return run3<N, Tin, Tout>(T, st);
            FCFS_NT3_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    };
    if (din == FCFS_F32 && dout == FCFS_F32) return go((float*)nullptr, (float*)nullptr);
    if (din == FCFS_BF16 && dout == FCFS_BF16) return go((__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr);
    return cudaErrorInvalidValue;
}

int read_status_fwd3d(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_fwd3d, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_fwd3d, &z, sizeof(int));
    }
    return v;
}

}  // namespace fcfs
