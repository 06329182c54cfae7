// K4 for volumes (fast path): persistent, bulk-copy staged input gradient of
// the separable 3D FCFS layer (the adjoint of the Sec. 4 map).
//
// A CTA owns a rectangle of real (y, x) input indices and a chunk of real
// depth indices.  Each g plane the chunk's adjoint windows read is copied to
// shared memory (double-buffered: the next plane lands while this one is
// used) and goes through the 2D adjoint of the (y, x) axes with their
// padding folds; the result, one value per real (y, x) of the tile, enters a
// ring of span_d planes.  When the ring holds an adjoint depth window's
// planes, its s_d depth outputs are formed.  A depth output outside [0, D)
// is folded onto the index the padding maps it to; the indices that receive
// such folds accumulate in shared memory (starting from zero, in ascending
// virtual-index order) and are stored when the chunk ends.
#include <type_traits>

#include "fcfs_internal.cuh"
#include "fcfs_bwd_tma.cuh"

namespace fcfs {

namespace {

struct Dx3Geo {
    int plane, c, qx0, qy0, qd0, nqx, nqy, nqd;
    AxRange X, Y, Dr;
    int gx_al, xoff, gy0, g_first, g_last;  // g_last < g_first: no g plane to read
};

__device__ __forceinline__ Dx3Geo dx3_geo(const TmaDx3Params& T, int tile) {
    Dx3Geo g;
    int t = tile;
    const int tx = t % T.qtiles_x;
    t /= T.qtiles_x;
    const int ty = t % T.qtiles_y;
    t /= T.qtiles_y;
    const int td = t % T.qtiles_d;
    g.plane = t / T.qtiles_d;
    g.c = g.plane % T.C;
    const AdjP &JD = T.aj[0], &JY = T.aj[1], &JX = T.aj[2];
    g.qx0 = tx * T.QX;
    g.qy0 = ty * T.QY;
    g.qd0 = td * T.QD;
    g.nqx = min(T.QX, JX.n_x - g.qx0);
    g.nqy = min(T.QY, JY.n_x - g.qy0);
    g.nqd = min(T.QD, JD.n_x - g.qd0);
    g.X = ax_range(JX, T.pad, g.qx0, g.qx0 + g.nqx - 1);
    g.Y = ax_range(JY, T.pad, g.qy0, g.qy0 + g.nqy - 1);
    g.Dr = ax_range(JD, T.pad, g.qd0, g.qd0 + g.nqd - 1);
    const int gx0 = g.X.alo * JX.r + JX.lo_in;
    g.gx_al = gx0 >= 0 ? (gx0 / T.align) * T.align : -(((-gx0) + T.align - 1) / T.align) * T.align;
    g.xoff = gx0 - g.gx_al;
    g.gy0 = g.Y.alo * JY.r + JY.lo_in;
    if (g.Dr.ahi >= g.Dr.alo) {
        g.g_first = g.Dr.alo * JD.r + JD.lo_in;
        g.g_last = g.Dr.ahi * JD.r + JD.lo_in + JD.span - 1;
    } else {
        g.g_first = 0;
        g.g_last = -1;
    }
    return g;
}

template <typename Tg>
__device__ __forceinline__ void issue3(const TmaDx3Params& T, const Dx3Geo& g, int gd, void* buf, uint64_t* bar) {
    fence_proxy_async_smem();
    mbar_expect_tx(bar, (uint32_t)(T.GBW * T.GBH * sizeof(Tg)));
    // g planes outside [0, Do) read as zero (the copy's out-of-range fill)
    tma_load_4d(buf, &T.tmap, g.gx_al, g.gy0, gd, g.plane, bar);
}

// Issue cursor of the job stream (the tiles that read g, their g planes in
// order), kept by thread 0 in shared memory.
struct CursorDx3 {
    Dx3Geo g;
    int tile, gd, n;
    int k;  // stage of the next job to issue
};

template <typename Tg>
__device__ __forceinline__ void issue_next(const TmaDx3Params& T, CursorDx3& c, const TileDeal& d, unsigned char* smem,
                                           uint64_t* bars) {
    if (c.tile >= d.n) return;
    if (c.n > 0 && ++c.gd > c.g.g_last) {
        do {
            if (++c.tile >= d.n) return;
            c.g = dx3_geo(T, d.tile(c.tile));
        } while (c.g.g_last < c.g.g_first);
        c.gd = c.g.g_first;
    }
    issue3<Tg>(T, c.g, c.gd, smem + c.k * T.buf_bytes, &bars[c.k]);
    ++c.n;
    if (++c.k == T.stages) c.k = 0;
}

template <int NT>
__device__ __forceinline__ void stage_adj3(float* dst, const AxisP& A, const AdjP& J, int c) {
    for (int e = threadIdx.x; e < J.s * NT; e += blockDim.x) {
        const int u = e / NT, t = e - u * NT;
        const int k = t < J.ntu[u] ? J.idx[u * kMaxAdjTaps + t] : -1;
        dst[e] = k >= 0 ? fwd_weight(A, c, k) : 0.f;
    }
}

// fold slot of real depth index q, or -1 when no padding contribution lands there
__device__ __forceinline__ int fold_slot(const TmaDx3Params& T, int q) {
    const int D = T.aj[0].n_x;
    if (q < T.nL) return q;
    if (q >= D - T.nR) return T.nL + (q - (D - T.nR));
    return -1;
}

// real depth index that depth output v contributes to (v itself inside [0, D))
__device__ __forceinline__ int depth_target(const TmaDx3Params& T, int v) {
    const int D = T.aj[0].n_x;
    if (v >= 0 && v < D) return v;
    return T.pad == FCFS_PAD_CONSTANT ? -1 : ext_index(v, D, T.pad);
}

template <int NT, typename Tg, typename Tx>
__global__ void __launch_bounds__(256, 2) fcfs_bwd_dx3d_tma(const __grid_constant__ TmaDx3Params T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    __shared__ CursorDx3 cur;
    const AdjP &JD = T.aj[0], &JY = T.aj[1], &JX = T.aj[2];
    float* sF = reinterpret_cast<float*>(smem_raw + T.fx_off);
    float* ring = reinterpret_cast<float*>(smem_raw + T.ring_off);
    float* facc = reinterpret_cast<float*>(smem_raw + T.facc_off);
    float* sWx = reinterpret_cast<float*>(smem_raw + T.w_off);
    float* sWy = sWx + JX.s * NT;
    float* sWd = sWy + JY.s * NT;
    int* xtab = reinterpret_cast<int*>(smem_raw + T.tab_off);  // per virtual column: u << 16 | g offset
    int* ytab = xtab + T.VXcap;                                  // per virtual row: u << 16 | Fx row
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);
    const int S = T.stages;
    const int QX = T.QX, GBW = T.GBW, VXcap = T.VXcap;
    const int plane_sz = T.QY * QX;
    const int G = blockDim.x / QX;
    const int cl = threadIdx.x % QX, gq = threadIdx.x / QX;
    const bool active = gq < G;
    const int Nx = JX.n_x, Ny = JY.n_x, Nd = JD.n_x;
    const int ringn = JD.span;

    const TileDeal deal = deal_tiles(T.ntiles, T.chunk);
    if (deal.n <= 0) return;
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
        s_abort = 0;
        cur.tile = 0;
        cur.g = dx3_geo(T, deal.tile(0));
        while (cur.g.g_last < cur.g.g_first && ++cur.tile < deal.n) cur.g = dx3_geo(T, deal.tile(cur.tile));
        cur.gd = cur.g.g_first;
        cur.n = 0;
        cur.k = 0;
        for (int k = 0; k < S; ++k) issue_next<Tg>(T, cur, deal, smem_raw, bars);
    }
    __syncthreads();
    const bool learn = T.ax[0].learn || T.ax[1].learn || T.ax[2].learn;
    int cur_c = -1;
    int stg = 0;         // stage of the current job
    uint32_t phase = 0;  // its barrier phase
    int consumed = 0;    // jobs taken so far (cur.n were issued)
    for (int kt = 0; kt < deal.n; ++kt) {
        const Dx3Geo gt = dx3_geo(T, deal.tile(kt));
        Tx* xpl = static_cast<Tx*>(T.gx) + (long long)gt.plane * Nd * Ny * Nx;
        const bool col_ok = active && cl < gt.nqx;
        if (gt.g_last < gt.g_first) {
            // no adjoint window touches this chunk: its gradient is zero
            if (col_ok)
                for (int qd = gt.qd0; qd < gt.qd0 + gt.nqd; ++qd)
                    for (int qyl = gq; qyl < gt.nqy; qyl += G)
                        store_out(xpl + ((long long)qd * Ny + gt.qy0 + qyl) * Nx + gt.qx0 + cl, 0.f);
            continue;
        }
        if (cur_c < 0 || (learn && gt.c != cur_c)) {
            // the previous tile ended with a barrier: no thread still reads the weights
            stage_adj3<NT>(sWx, T.ax[2], JX, gt.c);
            stage_adj3<NT>(sWy, T.ax[1], JY, gt.c);
            stage_adj3<NT>(sWd, T.ax[0], JD, gt.c);
            cur_c = gt.c;
        }
        // fold accumulators of this chunk start at zero (each thread owns its positions)
        const bool has_fold = (T.nL > 0 && gt.qd0 < T.nL) || (T.nR > 0 && gt.qd0 + gt.nqd > Nd - T.nR);
        if (has_fold && col_ok)
            for (int f = 0; f < T.nL + T.nR; ++f)
                for (int qyl = gq; qyl < gt.nqy; qyl += G) facc[f * plane_sz + qyl * QX + cl] = 0.f;
        // phase and source offset of every virtual column / row of the tile
        // (the previous tile ended with a barrier: no thread still reads them)
        for (int cx = threadIdx.x; cx < gt.X.vhi - gt.X.vlo + 1; cx += blockDim.x) {
            const int d = gt.X.vlo + cx - JX.lo_out;
            const int a = d / JX.s, u = d - a * JX.s;
            xtab[cx] = u << 16 | ((a - gt.X.alo) * JX.r + JX.off[u]);
        }
        for (int vr = threadIdx.x; vr < gt.Y.vhi - gt.Y.vlo + 1; vr += blockDim.x) {
            const int d = gt.Y.vlo + vr - JY.lo_out;
            const int a = d / JY.s, u = d - a * JY.s;
            ytab[vr] = u << 16 | ((a - gt.Y.alo) * JY.r + JY.off[u]);
        }
        int ad = gt.Dr.alo;  // next adjoint depth window to form
        int rslot = 0;  // ring slot of g plane gd
        for (int gd = gt.g_first; gd <= gt.g_last; ++gd) {
            unsigned char* const bufk = smem_raw + stg * T.buf_bytes;
            // one warp waits for the copy; the barrier releases the others
            if (threadIdx.x < 32 && !mbar_wait(&bars[stg], phase, &g_status_bwd_tma)) s_abort = 1;
            __syncthreads();
            if (s_abort) {
                if (threadIdx.x == 0) drain_ring(bars, S, stg, phase, cur.n - consumed, &g_status_bwd_tma);
                return;
            }
            ++consumed;
            const Tg* G0 = reinterpret_cast<const Tg*>(bufk);
            float* slot = ring + rslot * plane_sz;
            if (gd < 0 || gd >= JD.n_g) {
                // outside the forward output: a zero plane
                if (col_ok)
                    for (int qyl = gq; qyl < gt.nqy; qyl += G) slot[qyl * QX + cl] = 0.f;
            } else {
                const int VX = gt.X.vhi - gt.X.vlo + 1;
                const int nGR = gt.Y.ahi >= gt.Y.alo ? (gt.Y.ahi - gt.Y.alo) * JY.r + JY.span : 0;
                // ---- pass x over every staged g row, extended columns [vlo, vhi]
                if (active) {
                    for (int cx = cl; cx < VX; cx += QX) {
                        const int e = xtab[cx], u = e >> 16;
                        float w[NT];
#pragma unroll
                        for (int t = 0; t < NT; ++t) w[t] = sWx[u * NT + t];
                        const Tg* src = G0 + gq * GBW + gt.xoff + (e & 0xffff);
                        float* dst = sF + gq * VXcap + cx;
                        for (int gr = gq; gr < nGR; gr += G) {
                            float acc = 0.f;
#pragma unroll
                            for (int t = 0; t < NT; ++t) acc = fmaf(w[t], to_f<Tg>(src[t]), acc);
                            *dst = acc;
                            src += G * GBW;
                            dst += G * VXcap;
                        }
                    }
                }
                __syncthreads();
                // ---- fold x: virtual columns onto the real columns of this tile
                if (gt.X.left || gt.X.right) {
                    for (int gr = threadIdx.x; gr < nGR; gr += blockDim.x) {
                        float* row = sF + gr * VXcap;
                        const int l1 = min(gt.X.vhi, -1), r0 = max(gt.X.vlo, Nx);
                        for (int v = gt.X.vlo; v <= l1; ++v) {
                            const int q = ext_index(v, Nx, T.pad);
                            if (q >= gt.qx0 && q < gt.qx0 + gt.nqx) row[q - gt.X.vlo] += row[v - gt.X.vlo];
                        }
                        for (int v = r0; v <= gt.X.vhi; ++v) {
                            const int q = ext_index(v, Nx, T.pad);
                            if (q >= gt.qx0 && q < gt.qx0 + gt.nqx) row[q - gt.X.vlo] += row[v - gt.X.vlo];
                        }
                    }
                    __syncthreads();
                }
                // ---- pass y on the real columns; the g tile is consumed, its buffer holds the rows
                float* sO = reinterpret_cast<float*>(bufk);
                const int q = gt.qx0 + cl;
                const int fcol = q - gt.X.vlo;
                const bool col_has = col_ok && q <= gt.X.vhi;
                if (col_ok) {
                    const int VY = gt.Y.vhi - gt.Y.vlo + 1;
                    for (int vr = gq; vr < VY; vr += G) {
                        const int e = ytab[vr];
                        const float* src = sF + (e & 0xffff) * VXcap + fcol;
                        const float* w = sWy + (e >> 16) * NT;
                        float acc = 0.f;
                        if (col_has) {
#pragma unroll
                            for (int t = 0; t < NT; ++t) acc = fmaf(w[t], src[t * VXcap], acc);
                        }
                        sO[vr * QX + cl] = acc;
                    }
                }
                __syncthreads();
                // ---- fold y into the ring slot of this g plane
                if (col_ok) {
                    for (int qyl = gq; qyl < gt.nqy; qyl += G) {
                        const int qy = gt.qy0 + qyl;
                        float acc = (qy >= gt.Y.vlo && qy <= gt.Y.vhi) ? sO[(qy - gt.Y.vlo) * QX + cl] : 0.f;
                        if (gt.Y.left || gt.Y.right) {
                            const int l1 = min(gt.Y.vhi, -1), r0 = max(gt.Y.vlo, Ny);
                            for (int v = gt.Y.vlo; v <= l1; ++v)
                                if (ext_index(v, Ny, T.pad) == qy) acc += sO[(v - gt.Y.vlo) * QX + cl];
                            for (int v = r0; v <= gt.Y.vhi; ++v)
                                if (ext_index(v, Ny, T.pad) == qy) acc += sO[(v - gt.Y.vlo) * QX + cl];
                        }
                        slot[qyl * QX + cl] = acc;
                    }
                }
            }
            // ---- depth: every adjoint window whose g planes are all in the ring
            // (a thread reads and writes only its own (y, x) positions)
            while (ad <= gt.Dr.ahi && ad * JD.r + JD.lo_in + JD.span <= gd + 1) {
                for (int u = 0; u < JD.s; ++u) {
                    const int v = ad * JD.s + JD.lo_out + u;
                    if (v < gt.Dr.vlo || v > gt.Dr.vhi) continue;
                    const int tq = depth_target(T, v);
                    if (tq < gt.qd0 || tq >= gt.qd0 + gt.nqd) continue;
                    const int fs = fold_slot(T, tq);
                    if (!col_ok) continue;
                    // the window completes at plane gd: its plane k sits in slot (rslot + 1 + k) mod span
                    float w[NT];
                    const float* rp[NT];
                    const int sb = rslot + 1 + JD.off[u];
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        w[t] = sWd[u * NT + t];
                        int sl = sb + t;
                        if (sl >= ringn) sl -= ringn;
                        if (sl >= ringn) sl -= ringn;
                        rp[t] = ring + sl * plane_sz + cl;
                    }
                    for (int qyl = gq; qyl < gt.nqy; qyl += G) {
                        float acc = 0.f;
#pragma unroll
                        for (int t = 0; t < NT; ++t) acc = fmaf(w[t], rp[t][qyl * QX], acc);
                        if (fs >= 0) facc[fs * plane_sz + qyl * QX + cl] += acc;
                        else store_out(xpl + ((long long)tq * Ny + gt.qy0 + qyl) * Nx + gt.qx0 + cl, acc);
                    }
                }
                ++ad;
            }
            __syncthreads();  // the ring slot, sF and this stage are free again
            if (threadIdx.x == 0) issue_next<Tg>(T, cur, deal, smem_raw, bars);
            if (++rslot == ringn) rslot = 0;
            if (++stg == S) {
                stg = 0;
                phase ^= 1;
            }
        }
        // ---- chunk end: folded indices, and real indices no adjoint window reaches
        if (col_ok) {
            for (int qd = gt.qd0; qd < gt.qd0 + gt.nqd; ++qd) {
                const int fs = fold_slot(T, qd);
                const bool covered = qd >= gt.Dr.vlo && qd <= gt.Dr.vhi;
                if (fs < 0 && covered) continue;
                for (int qyl = gq; qyl < gt.nqy; qyl += G)
                    store_out(xpl + ((long long)qd * Ny + gt.qy0 + qyl) * Nx + gt.qx0 + cl,
                              fs >= 0 ? facc[fs * plane_sz + qyl * QX + cl] : 0.f);
            }
        }
    }
}

template <int NT, typename Tg, typename Tx>
cudaError_t run3(const TmaDx3Params& T, cudaStream_t st) {
    const size_t smem = (size_t)T.bar_off + 8 * T.stages;
    auto k = fcfs_bwd_dx3d_tma<NT, Tg, Tx>;
    int sms = 0, per_sm = 0;
    cudaError_t e = resident_ctas((const void*)k, T.threads, smem, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(T.ntiles, (long long)sms * per_sm);
    k<<<(unsigned)grid, T.threads, smem, st>>>(T);
    return cudaGetLastError();
}

}  // namespace

#define FCFS_ADJ3_NT_CASES(X) X(2) X(3) X(4) X(6) X(8)

cudaError_t launch_dx3d_tma(const TmaDx3Params& T, int nt, int dt, cudaStream_t st) {
    auto go = [&](auto tg) -> cudaError_t {
        using Tg = std::remove_pointer_t<decltype(tg)>;
        switch (nt) {
#define CASE(N) \
    case N: return run3<N, Tg, Tg>(T, st);
            FCFS_ADJ3_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    };
    if (dt == FCFS_F32) return go((float*)nullptr);
    if (dt == FCFS_BF16) return go((__nv_bfloat16*)nullptr);
    return cudaErrorInvalidValue;
}

int read_status_bwd_dx3d(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_bwd_tma, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_bwd_tma, &z, sizeof(int));
    }
    return v;
}

}  // namespace fcfs
