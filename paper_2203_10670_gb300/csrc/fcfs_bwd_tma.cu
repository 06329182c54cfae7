// K4 (fast path): persistent, TMA-staged input gradient of the FCFS layer
// for 1D/2D (the adjoint of the Sec. 3.1 / Sec. 4 map, needed to learn the
// weights as Sec. 7 proposes).
//
// The adjoint of one axis is itself a polyphase operator: its window a has s
// phases u whose outputs are the extended input indices v = a*s + lo_out + u,
// and phase u reads g at a*r + lo_in + off[u] + t.  A CTA owns a rectangle of
// REAL input indices; tiles that touch an edge also evaluate the virtual
// indices left of 0 / right of N-1 and fold them onto the indices the padding
// maps them to (replicate: the edge sample, reflect: the mirror, constant:
// dropped).  Per tile:
//   stage  g rectangle by a bulk-tensor copy (double-buffered; g outside the
//          forward output is zero, which is the copy's out-of-range fill),
//   pass x Fx[gr][v] = sum_t W'x[u][t] g[gr][(a-a0)*r + off[u] + t], fold x,
//   pass y dx[v][q] = sum_t W'y[u][t] Fx[(a-a0)*r + off[u] + t][q], fold y
//          (through shared memory on edge tiles), store.
#include <type_traits>

#include "fcfs_internal.cuh"
#include "fcfs_bwd_tma.cuh"

namespace fcfs {


namespace {

template <int NT>
__device__ __forceinline__ void stage_adj_weights(float* dst, const AxisP& A, const AdjP& J, int c) {
    for (int e = threadIdx.x; e < J.s * NT; e += blockDim.x) {
        const int u = e / NT, t = e - u * NT;
        const int k = t < J.ntu[u] ? J.idx[u * kMaxAdjTaps + t] : -1;
        dst[e] = k >= 0 ? fwd_weight(A, c, k) : 0.f;
    }
}

template <int NT, typename Tg, typename Tx>
__global__ void __launch_bounds__(256) fcfs_bwd_dx2d_tma(const __grid_constant__ TmaDxParams T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    const AdjP& JX = T.aj[2];
    const AdjP& JY = T.aj[1];
    float* sF = reinterpret_cast<float*>(smem_raw + T.fx_off);
    float* sWx = reinterpret_cast<float*>(smem_raw + T.w_off);
    float* sWy = sWx + JX.s * NT;
    int* xtab = reinterpret_cast<int*>(smem_raw + T.tab_off);  // per virtual column: u << 16 | g offset
    int* ytab = xtab + T.VXcap;                                  // per virtual row: u << 16 | Fx row
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);
    const int S = T.stages;
    const int QX = T.QX, GBW = T.GBW, VXcap = T.VXcap;
    const int G = blockDim.x / QX;
    const int cl = threadIdx.x % QX, gq = threadIdx.x / QX;
    const bool active = gq < G;
    const int Nx = JX.n_x, Ny = JY.n_x;

    const TileDeal deal = deal_tiles((int)T.ntiles, T.chunk);
    if (deal.n <= 0) return;
    // geometry of the tile in each stage, computed once by the thread that issues its copy
    __shared__ DxGeo sgeo[4];
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
        s_abort = 0;
        for (int k = 0; k < S && k < deal.n; ++k) {
            sgeo[k] = dx_geo(T, deal.tile(k));
            issue<Tg>(T, sgeo[k], smem_raw + k * T.buf_bytes, &bars[k]);
        }
    }
    __syncthreads();
    const bool learn = T.ax[2].learn || T.ax[1].learn;
    int cur_c = -1;
    int stg = 0;
    uint32_t phase = 0;
    for (int kt = 0; kt < deal.n; ++kt) {
        unsigned char* const bufk = smem_raw + stg * T.buf_bytes;
        // one warp waits for the copy; the barrier releases the others
        if (threadIdx.x < 32 && !mbar_wait(&bars[stg], phase, &g_status_bwd_tma)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) drain_ring(bars, S, stg, phase, min(S, deal.n - kt), &g_status_bwd_tma);
            return;
        }
        const DxGeo geo = sgeo[stg];
        const int VX = geo.X.vhi - geo.X.vlo + 1;
        const int VY = geo.Y.vhi - geo.Y.vlo + 1;
        // the previous tile ended with a barrier: no thread still reads the weights or tables
        if (cur_c < 0 || (learn && geo.c != cur_c)) {
            stage_adj_weights<NT>(sWx, T.ax[2], JX, geo.c);
            stage_adj_weights<NT>(sWy, T.ax[1], JY, geo.c);
            cur_c = geo.c;
        }
        for (int cx = threadIdx.x; cx < VX; cx += blockDim.x) {
            const int d = geo.X.vlo + cx - JX.lo_out;  // d >= 0: vlo >= vmin = lo_out
            const int a = d / JX.s, u = d - a * JX.s;
            xtab[cx] = u << 16 | ((a - geo.X.alo) * JX.r + JX.off[u]);
        }
        for (int vr = threadIdx.x; vr < VY; vr += blockDim.x) {
            const int d = geo.Y.vlo + vr - JY.lo_out;
            const int a = d / JY.s, u = d - a * JY.s;
            ytab[vr] = u << 16 | ((a - geo.Y.alo) * JY.r + JY.off[u]);
        }
        __syncthreads();
        const Tg* G0 = reinterpret_cast<const Tg*>(bufk);

        const int nGR = geo.Y.ahi >= geo.Y.alo ? (geo.Y.ahi - geo.Y.alo) * JY.r + JY.span : 0;
        // ---- pass x: adjoint along x for every staged g row, extended columns [vlo, vhi]
        if (active) {
            for (int cx = cl; cx < VX; cx += QX) {
                const int e = xtab[cx], u = e >> 16;
                float w[NT];
#pragma unroll
                for (int t = 0; t < NT; ++t) w[t] = sWx[u * NT + t];
                // taps past the phase's own count carry zero weights and stay inside the box
                const Tg* src = G0 + gq * GBW + geo.xoff + (e & 0xffff);
                float* dst = sF + gq * VXcap + cx;
#pragma unroll 2
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
        // ---- fold x: virtual columns onto the real column the padding maps them to
        if (geo.X.left || geo.X.right) {
            for (int gr = threadIdx.x; gr < nGR; gr += blockDim.x) {
                float* row = sF + gr * VXcap;
                // only the virtual columns left of 0 and right of N-1; a target outside this tile's
                // real columns belongs to (and is folded by) its own tile
                const int l1 = min(geo.X.vhi, -1), r0 = max(geo.X.vlo, Nx);
                for (int v = geo.X.vlo; v <= l1; ++v) {
                    const int q = ext_index(v, Nx, T.pad);
                    if (q >= geo.qx0 && q < geo.qx0 + geo.nqx) row[q - geo.X.vlo] += row[v - geo.X.vlo];
                }
                for (int v = r0; v <= geo.X.vhi; ++v) {
                    const int q = ext_index(v, Nx, T.pad);
                    if (q >= geo.qx0 && q < geo.qx0 + geo.nqx) row[q - geo.X.vlo] += row[v - geo.X.vlo];
                }
            }
            __syncthreads();
        }
        // ---- pass y: adjoint along y on the real columns of the tile, one virtual row per step
        const bool ypath_smem = geo.Y.left || geo.Y.right || !geo.Y.covered;
        float* sO = reinterpret_cast<float*>(bufk);  // the g tile is consumed
        const int q = geo.qx0 + cl;
        const int fcol = q - geo.X.vlo;
        const bool col_ok = active && cl < geo.nqx;
        const bool col_has = col_ok && q <= geo.X.vhi;
        Tx* xcol = static_cast<Tx*>(T.gx) + (long long)geo.plane * Ny * Nx + q;
        if (col_ok) {
            for (int vr = gq; vr < VY; vr += G) {
                const int e = ytab[vr];
                const float* src = sF + (e & 0xffff) * VXcap + fcol;
                const float* w = sWy + (e >> 16) * NT;
                float acc = 0.f;
                if (col_has) {
#pragma unroll
                    for (int t = 0; t < NT; ++t) acc = fmaf(w[t], src[t * VXcap], acc);
                }
                if (ypath_smem) sO[vr * QX + cl] = acc;
                else store_out(xcol + (long long)(geo.Y.vlo + vr) * Nx, acc);
            }
        }
        if (ypath_smem) {
            __syncthreads();
            if (col_ok) {
                for (int qy = geo.qy0 + gq; qy < geo.qy0 + geo.nqy; qy += G) {
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
        __syncthreads();  // sF, the tables and this stage are free again
        if (threadIdx.x == 0 && kt + S < deal.n) {
            sgeo[stg] = dx_geo(T, deal.tile(kt + S));
            issue<Tg>(T, sgeo[stg], bufk, &bars[stg]);
        }
        if (++stg == S) {
            stg = 0;
            phase ^= 1;
        }
    }
}

template <int NT, typename Tg, typename Tx>
cudaError_t run(const TmaDxParams& T, cudaStream_t st) {
    const size_t smem = (size_t)T.bar_off + 8 * T.stages;
    auto k = fcfs_bwd_dx2d_tma<NT, Tg, Tx>;
    int sms = 0, per_sm = 0;
    cudaError_t e = resident_ctas((const void*)k, T.threads, smem, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(T.ntiles, (long long)sms * per_sm);
    k<<<(unsigned)grid, T.threads, smem, st>>>(T);
    return cudaGetLastError();
}

}  // namespace

int read_status_bwd_rs(int clear);
int read_status_bwd_dx3d(int clear);

int read_status_bwd_tma(int clear) {
    const int w = read_status_bwd_rs(clear), w3 = read_status_bwd_dx3d(clear);
    if (w < 0 || w3 < 0) return -1;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_bwd_tma, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_bwd_tma, &z, sizeof(int));
    }
    return v | w | w3;
}

#define FCFS_ADJ_NT_CASES(X) X(2) X(3) X(4) X(6) X(8) X(10) X(12) X(16)

cudaError_t launch_dx_tma(const TmaDxParams& T, int nt, int dg, int dx, cudaStream_t st) {
    auto go = [&](auto tg, auto tx) -> cudaError_t {
        using Tg = std::remove_pointer_t<decltype(tg)>;
        using Tx = std::remove_pointer_t<decltype(tx)>;
        switch (nt) {
#define CASE(N) \
    case N: return run<N, Tg, Tx>(T, st);
            FCFS_ADJ_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    };
    if (dg == FCFS_F32 && dx == FCFS_F32) return go((float*)nullptr, (float*)nullptr);
    if (dg == FCFS_BF16 && dx == FCFS_BF16) return go((__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr);
    return cudaErrorInvalidValue;
}

}  // namespace fcfs

// ===========================================================================
// K5 (fast path): weight gradient of learnable taps, 1D/2D.
//   dWy[jy][t] = sum g[iy*r_y + jy][ox] * U[iy*s_y + off_y[jy] + t][ox],  U = x taps of x~
//   dWx[jx][t] = sum g[oy][ix*r_x + jx] * V[oy][ix*s_x + off_x[jx] + t],  V = y taps of x~
// A persistent CTA walks a contiguous run of forward-shaped tiles, stages x~
// and g by bulk copies, and keeps its dot products in registers across tiles;
// it writes one record per channel it visits.  A second kernel sums the
// records of each weight entry in a fixed order (bitwise reproducible).
// ===========================================================================
namespace fcfs {
namespace {

constexpr int kDwMaxPairs = 2;

struct DwGeo {
    int plane, c, ix0, iy0, nwx, nwy, rows, cols, row0, col0, x_al, xoff, g_al, goff;
    bool edge;
};

__device__ __forceinline__ DwGeo dw_geo(const TmaDwParams& T, int tile) {
    const FwdParams& P = T.P;
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    DwGeo g;
    const int txy = P.tiles_x * P.tiles_y;
    g.plane = tile / txy;
    const int rem = tile - g.plane * txy;
    const int ty = rem / P.tiles_x, tx = rem - ty * P.tiles_x;
    g.c = g.plane % P.C;
    g.ix0 = tx * P.WX;
    g.iy0 = ty * P.WY;
    g.nwx = min(P.WX, AX.n_win - g.ix0);
    g.nwy = min(P.WY, AY.n_win - g.iy0);
    g.cols = (g.nwx - 1) * AX.s + AX.span;
    g.rows = (g.nwy - 1) * AY.s + AY.span;
    g.col0 = g.ix0 * AX.s + AX.lo;
    g.row0 = g.iy0 * AY.s + AY.lo;
    g.x_al = g.col0 >= 0 ? (g.col0 / T.align) * T.align : -(((-g.col0) + T.align - 1) / T.align) * T.align;
    g.xoff = g.col0 - g.x_al;
    const int gc = g.ix0 * AX.r;
    g.g_al = (gc / T.align) * T.align;
    g.goff = gc - g.g_al;
    g.edge = g.col0 < 0 || g.col0 + g.cols > AX.n_in || g.row0 < 0 || g.row0 + g.rows > AY.n_in;
    return g;
}

template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// padding of an edge x~ tile in shared memory (as the forward)
template <typename Tin>
__device__ __forceinline__ void dw_fix_edges(const TmaDwParams& T, const DwGeo& g, Tin* buf, const void* x) {
    const FwdParams& P = T.P;
    const int H = P.ax[1].n_in, W = P.ax[2].n_in;
    const int BW = T.BWx;
    if (P.pad == FCFS_PAD_REFLECT) {
        const Tin* xp = static_cast<const Tin*>(x) + (long long)g.plane * H * W;
        const int BU = min(BW, g.xoff + g.cols);
        for (int e = threadIdx.x; e < g.rows * BU; e += blockDim.x) {
            const int ry = e / BU, cx = e - ry * BU;
            const int sy = ext_index(g.row0 + ry, H, P.pad);
            const int sx = ext_index(g.x_al + cx, W, P.pad);
            buf[ry * BW + cx] = xp[(long long)sy * W + sx];
        }
        __syncthreads();
        return;
    }
    const bool repl = P.pad == FCFS_PAD_REPLICATE;
    const Tin cv = from_f<Tin>(P.padv);
    // only the columns the taps read: [0, xoff + cols) of the box
    const int BU = min(BW, g.xoff + g.cols);
    const int cl = min(BU, max(0, -g.x_al)), cr = max(0, g.x_al + BU - W);
    if (cl > 0 || cr > 0) {
        const int ncol = cl + cr;
        for (int e = threadIdx.x; e < g.rows * ncol; e += blockDim.x) {
            const int ry = e / ncol, k = e - ry * ncol;
            const int gy = g.row0 + ry;
            if (gy < 0 || gy >= H) continue;
            const int cx = k < cl ? k : BU - cr + (k - cl);
            const int src = (k < cl ? 0 : W - 1) - g.x_al;
            buf[ry * BW + cx] = repl ? buf[ry * BW + src] : cv;
        }
        __syncthreads();
    }
    const int rt = max(0, -g.row0), rb = max(0, g.row0 + g.rows - H);
    if (rt > 0 || rb > 0) {
        const int nrow = rt + rb;
        for (int e = threadIdx.x; e < nrow * BU; e += blockDim.x) {
            const int k = e / BU, cx = e - k * BU;
            const int ry = k < rt ? k : g.rows - rb + (k - rt);
            const int src = (k < rt ? 0 : H - 1) - g.row0;
            buf[ry * BW + cx] = repl ? buf[src * BW + cx] : cv;
        }
        __syncthreads();
    }
}

template <int NT, typename Tv>
__global__ void __launch_bounds__(256) fcfs_bwd_dw2d_tma(const __grid_constant__ TmaDwParams T, const void* xptr) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    const FwdParams& P = T.P;
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    // stage b of the x and g copies (selected arithmetically: no local-memory pointer tables)
    auto xb = [&](int b) { return reinterpret_cast<Tv*>(smem_raw + b * T.xbuf_bytes); };
    auto gb = [&](int b) { return reinterpret_cast<Tv*>(smem_raw + 2 * T.xbuf_bytes + b * T.gbuf_bytes); };
    float* sH = reinterpret_cast<float*>(smem_raw + T.sh_off);
    float* sV = reinterpret_cast<float*>(smem_raw + T.sv_off);
    float* sWx = reinterpret_cast<float*>(smem_raw + T.w_off);
    float* sWy = sWx + AX.r * NT;
    float* sRed = reinterpret_cast<float*>(smem_raw + T.red_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);

    const int OX = P.OX, BWx = T.BWx, BWg = T.BWg, ICp = T.ICp;
    const int G1 = blockDim.x / OX;
    const int ox = threadIdx.x % OX, g1 = threadIdx.x / OX;
    const int jx = ox % AX.r, ixl = ox / AX.r;
    const bool xact = g1 < G1;
    const int npair = OX * AY.r;
    const bool per_channel = AX.w_cstride != 0 || AY.w_cstride != 0;
    const uint32_t tx_bytes = (uint32_t)(T.BWx * T.BHx + T.BWg * T.BHg) * sizeof(Tv);

    float accx[NT], accy[kDwMaxPairs][NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        accx[t] = 0.f;
#pragma unroll
        for (int pp = 0; pp < kDwMaxPairs; ++pp) accy[pp][t] = 0.f;
    }

    float* recs = T.ws + (long long)blockIdx.x * T.maxseg * T.rec;
    int* ids = reinterpret_cast<int*>(T.ws + (long long)T.grid * T.maxseg * T.rec) + blockIdx.x * T.maxseg;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    const int per = (T.ntiles + gridDim.x - 1) / gridDim.x;
    int tile = blockIdx.x * per;
    const int tile_end = min(T.ntiles, tile + per);
    // geometry of the tile in each buffer, computed once by the thread that issues its copies
    __shared__ DwGeo sgeo[2];
    auto issue = [&](int t, int b) {
        const DwGeo g = dw_geo(T, t);
        sgeo[b] = g;
        fence_proxy_async_smem();
        mbar_expect_tx(&bars[b], tx_bytes);
        tma_load_3d(xb(b), &T.tmap_x, g.x_al, g.row0, g.plane, &bars[b]);
        tma_load_3d(gb(b), &T.tmap_g, g.g_al, g.iy0 * AY.r, g.plane, &bars[b]);
    };
    // write this CTA's accumulated partials as record `seg` for channel c
    auto flush = [&](int seg, int c) {
        __syncthreads();
        if (xact) {
#pragma unroll
            for (int t = 0; t < NT; ++t) sRed[threadIdx.x * NT + t] = accx[t];
        }
        float* ry = sRed + blockDim.x * NT;
#pragma unroll
        for (int pp = 0; pp < kDwMaxPairs; ++pp) {
            const int q = threadIdx.x + pp * blockDim.x;
            if (q < npair) {
#pragma unroll
                for (int t = 0; t < NT; ++t) ry[q * NT + t] = accy[pp][t];
            }
        }
        __syncthreads();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        const int nx = AX.r * NT, ny = AY.r * NT;
        const int per_jx = G1 * (OX / AX.r);
        float* rec = recs + (long long)seg * T.rec;
        for (int e = warp; e < nx + ny; e += nwarp) {
            float s = 0.f;
            if (e < nx) {
                const int j = e / NT, t = e - j * NT;
                for (int m = lane; m < per_jx; m += 32) {
                    const int gg = m / (OX / AX.r), il = m - gg * (OX / AX.r);
                    s += sRed[(gg * OX + il * AX.r + j) * NT + t];
                }
            } else {
                const int e2 = e - nx, j = e2 / NT, t = e2 - j * NT;
                for (int o = lane; o < OX; o += 32) s += ry[(j * OX + o) * NT + t];
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
            if (lane == 0) rec[e < nx ? P.ax[1].r * NT + e : e - nx] = s;
        }
        if (threadIdx.x == 0) ids[seg] = c;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            accx[t] = 0.f;
#pragma unroll
            for (int pp = 0; pp < kDwMaxPairs; ++pp) accy[pp][t] = 0.f;
        }
    };

    int seg = 0, cur_c = -1;
    if (tile < tile_end && threadIdx.x == 0) issue(tile, 0);
    for (int k = 0; tile < tile_end; ++k, ++tile) {
        Tv* X = xb(k & 1);
        const Tv* Gt = gb(k & 1);
        // one warp waits for the copies; the barrier releases the others
        if (threadIdx.x < 32 && !mbar_wait(&bars[k & 1], (uint32_t)((k >> 1) & 1), &g_status_bwd_tma)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) drain_ring(bars, 2, k & 1, (uint32_t)((k >> 1) & 1), 1, &g_status_bwd_tma);
            return;
        }
        const DwGeo geo = sgeo[k & 1];
        if (threadIdx.x == 0 && tile + 1 < tile_end) issue(tile + 1, (k + 1) & 1);  // the other slot
        const int ch = per_channel ? geo.c : 0;
        if (ch != cur_c) {
            if (cur_c >= 0) flush(seg++, cur_c);
            for (int e = threadIdx.x; e < AX.r * NT; e += blockDim.x) {
                const int j = e / NT, t = e - j * NT;
                sWx[e] = t < AX.nt_src ? (AX.learn ? AX.w[geo.c * AX.w_cstride + j * AX.nt_src + t] : AX.wf[j * AX.nt_src + t]) : 0.f;
            }
            for (int e = threadIdx.x; e < AY.r * NT; e += blockDim.x) {
                const int j = e / NT, t = e - j * NT;
                sWy[e] = t < AY.nt_src ? (AY.learn ? AY.w[geo.c * AY.w_cstride + j * AY.nt_src + t] : AY.wf[j * AY.nt_src + t]) : 0.f;
            }
            cur_c = ch;
            __syncthreads();
        }
        if (geo.edge) dw_fix_edges<Tv>(T, geo, X, xptr);

        // U = x taps of every staged row (thread = output column)
        if (xact && ixl < geo.nwx) {
            float w[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) w[t] = sWx[jx * NT + t];
            const Tv* src = X + g1 * BWx + geo.xoff + ixl * AX.s + AX.off[jx];
            float* dst = sH + g1 * OX + ox;
            for (int ry = g1; ry < geo.rows; ry += G1) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t) acc = fmaf(w[t], to_f<Tv>(src[t]), acc);
                *dst = acc;
                src += G1 * BWx;
                dst += G1 * OX;
            }
        }
        // V = y taps of every staged column (thread = column and phase)
        for (int jy = 0, cx = threadIdx.x; jy < AY.r;) {
            if (cx >= geo.cols) {
                cx -= geo.cols;
                ++jy;
                continue;
            }
            float w[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) w[t] = sWy[jy * NT + t];
            const Tv* src = X + AY.off[jy] * BWx + geo.xoff + cx;
            float* dst = sV + jy * ICp + cx;
            for (int iyl = 0; iyl < geo.nwy; ++iyl) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t) acc = fmaf(w[t], to_f<Tv>(src[t * BWx]), acc);
                *dst = acc;
                src += AY.s * BWx;
                dst += AY.r * ICp;
            }
            cx += blockDim.x;
        }
        __syncthreads();
        // dWx: thread = output column, over its group's rows
        if (xact && ixl < geo.nwx) {
            const int nrow = geo.nwy * AY.r;
            const Tv* gp = Gt + geo.goff + ox;
            const float* vp = sV + ixl * AX.s + AX.off[jx];
            for (int oyl = g1; oyl < nrow; oyl += G1) {
                const float gv = to_f<Tv>(gp[oyl * BWg]);
                const float* v = vp + oyl * ICp;
#pragma unroll
                for (int t = 0; t < NT; ++t) accx[t] = fmaf(gv, v[t], accx[t]);
            }
        }
        // dWy: thread = (column, phase) pairs, over the tile's windows
#pragma unroll
        for (int pp = 0; pp < kDwMaxPairs; ++pp) {
            const int q = threadIdx.x + pp * blockDim.x;
            if (q < npair) {
                const int jy = q / OX, o = q - jy * OX;
                if (o / AX.r < geo.nwx) {
                    const Tv* gp = Gt + jy * BWg + geo.goff + o;
                    const float* up = sH + AY.off[jy] * OX + o;
                    for (int iyl = 0; iyl < geo.nwy; ++iyl) {
                        const float gv = to_f<Tv>(gp[iyl * AY.r * BWg]);
                        const float* u = up + iyl * AY.s * OX;
#pragma unroll
                        for (int t = 0; t < NT; ++t) accy[pp][t] = fmaf(gv, u[t * OX], accy[pp][t]);
                    }
                }
            }
        }
        __syncthreads();  // buffers free for the copies two tiles ahead
    }
    if (cur_c >= 0) flush(seg++, cur_c);
    if (threadIdx.x == 0)
        for (int s2 = seg; s2 < T.maxseg; ++s2) ids[s2] = -1;
}

// Register-blocked weight gradient for learnable taps on both axes with the
// same phase count R and tap count NT (window i of either axis reads x~ at
// i*s + t, t < NT).  Each pass works per window, so a thread loads a window's
// samples once and uses them for all R phases:
//   U  = x taps of x~:   U[row][i*R + jx] = sum_t Wx[jx][t] x~[row][i*s_x + t]
//   V  = y taps of x~:   V[i*R + jy][col] = sum_t Wy[jy][t] x~[i*s_y + t][col]
//   dWx[jx][t] += g[oy][i*R + jx] * V[oy][i*s_x + t]     (thread = window, row group)
//   dWy[jy][t] += g[i*R + jy][ox] * U[i*s_y + t][ox]     (thread = column, window group)
// Every thread holds all R x NT entries of both axes; a flush reduces them in
// a fixed order (warp shuffles, then the warps in index order) into the same
// record layout as the per-output kernel, so the same reduction kernel sums
// the records.
template <int R, int NT, typename Tv>
__global__ void __launch_bounds__(256, 2) fcfs_bwd_dw2d_rb(const __grid_constant__ TmaDwParams T, const void* xptr) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_abort;  // set when a bounded wait ran out: the CTA stops
    __shared__ float sWx[R * NT], sWy[R * NT];
    __shared__ DwGeo sgeo[2];
    const FwdParams& P = T.P;
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    auto xb = [&](int b) { return reinterpret_cast<Tv*>(smem_raw + b * T.xbuf_bytes); };
    auto gb = [&](int b) { return reinterpret_cast<Tv*>(smem_raw + 2 * T.xbuf_bytes + b * T.gbuf_bytes); };
    float* sU = reinterpret_cast<float*>(smem_raw + T.sh_off);   // [rows][OX]
    float* sV = reinterpret_cast<float*>(smem_raw + T.sv_off);   // [OY][ICp]
    float* sRed = reinterpret_cast<float*>(smem_raw + T.red_off);  // [warps][2 R NT]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + T.bar_off);
    constexpr int NE = R * NT;
    const int OX = P.OX, BWx = T.BWx, BWg = T.BWg, ICp = T.ICp, WX = P.WX;
    const int SX = AX.s, SY = AY.s;
    const bool per_channel = AX.w_cstride != 0 || AY.w_cstride != 0;
    const uint32_t tx_bytes = (uint32_t)(T.BWx * T.BHx + T.BWg * T.BHg) * sizeof(Tv);
    // thread mappings: window x row group (U, dWx); column x window group (V, dWy)
    const int GW = blockDim.x / WX;
    const int iw = threadIdx.x % WX, gw = threadIdx.x / WX;
    const bool wact = gw < GW;

    float accx[R][NT], accy[R][NT];
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
        for (int t = 0; t < NT; ++t) accx[j][t] = accy[j][t] = 0.f;

    float* recs = T.ws + (long long)blockIdx.x * T.maxseg * T.rec;
    int* ids = reinterpret_cast<int*>(T.ws + (long long)T.grid * T.maxseg * T.rec) + blockIdx.x * T.maxseg;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    const int per = (T.ntiles + gridDim.x - 1) / gridDim.x;
    int tile = blockIdx.x * per;
    const int tile_end = min(T.ntiles, tile + per);
    auto issue = [&](int t, int b) {
        const DwGeo g = dw_geo(T, t);
        sgeo[b] = g;
        fence_proxy_async_smem();
        mbar_expect_tx(&bars[b], tx_bytes);
        tma_load_3d(xb(b), &T.tmap_x, g.x_al, g.row0, g.plane, &bars[b]);
        tma_load_3d(gb(b), &T.tmap_g, g.g_al, g.iy0 * R, g.plane, &bars[b]);
    };
    // reduce every thread's entries into record `seg` for channel c (fixed order)
    auto flush = [&](int seg, int c) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
        for (int e = 0; e < 2 * NE; ++e) {
            float v = e < NE ? accx[e / NT][e % NT] : accy[(e - NE) / NT][(e - NE) % NT];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0) sRed[warp * 2 * NE + e] = v;
        }
        __syncthreads();
        float* rec = recs + (long long)seg * T.rec;
        for (int e = threadIdx.x; e < 2 * NE; e += blockDim.x) {
            float v = 0.f;
            for (int w = 0; w < nwarp; ++w) v += sRed[w * 2 * NE + e];
            // record layout: dWy entries first, then dWx
            rec[e < NE ? AY.r * NT + e : e - NE] = v;
        }
        if (threadIdx.x == 0) ids[seg] = c;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < R; ++j)
#pragma unroll
            for (int t = 0; t < NT; ++t) accx[j][t] = accy[j][t] = 0.f;
    };

    int seg = 0, cur_c = -1;
    if (tile < tile_end && threadIdx.x == 0) issue(tile, 0);
    for (int k = 0; tile < tile_end; ++k, ++tile) {
        Tv* X = xb(k & 1);
        const Tv* Gt = gb(k & 1);
        // one warp waits for the copies; the barrier releases the others
        if (threadIdx.x < 32 && !mbar_wait(&bars[k & 1], (uint32_t)((k >> 1) & 1), &g_status_bwd_tma)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) drain_ring(bars, 2, k & 1, (uint32_t)((k >> 1) & 1), 1, &g_status_bwd_tma);
            return;
        }
        const DwGeo geo = sgeo[k & 1];
        if (threadIdx.x == 0 && tile + 1 < tile_end) issue(tile + 1, (k + 1) & 1);  // the other slot
        const int ch = per_channel ? geo.c : 0;
        if (ch != cur_c) {
            if (cur_c >= 0) flush(seg++, cur_c);
            for (int e = threadIdx.x; e < NE; e += blockDim.x) {
                sWx[e] = AX.w[geo.c * AX.w_cstride + e];
                sWy[e] = AY.w[geo.c * AY.w_cstride + e];
            }
            cur_c = ch;
            __syncthreads();
        }
        if (geo.edge) dw_fix_edges<Tv>(T, geo, X, xptr);

        // ---- U: x taps of every staged row, a window per thread
        if (wact && iw < geo.nwx) {
            float w[R][NT];
#pragma unroll
            for (int j = 0; j < R; ++j)
#pragma unroll
                for (int t = 0; t < NT; ++t) w[j][t] = sWx[j * NT + t];
            const Tv* src = X + gw * BWx + geo.xoff + iw * SX;
            float* dst = sU + gw * OX + iw * R;
            for (int ry = gw; ry < geo.rows; ry += GW) {
                float v[NT];
#pragma unroll
                for (int t = 0; t < NT; ++t) v[t] = to_f<Tv>(src[t]);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    float a = 0.f;
#pragma unroll
                    for (int t = 0; t < NT; ++t) a = fmaf(w[j][t], v[t], a);
                    dst[j] = a;
                }
                src += GW * BWx;
                dst += GW * OX;
            }
        }
        // ---- V: y taps of every staged column, a window per thread step
        {
            float w[R][NT];
#pragma unroll
            for (int j = 0; j < R; ++j)
#pragma unroll
                for (int t = 0; t < NT; ++t) w[j][t] = sWy[j * NT + t];
            const int GC = blockDim.x / ICp;
            const int cx = threadIdx.x % ICp, gc = threadIdx.x / ICp;
            if (gc < GC && cx < geo.cols) {
                for (int iyl = gc; iyl < geo.nwy; iyl += GC) {
                    const Tv* src = X + iyl * SY * BWx + geo.xoff + cx;
                    float v[NT];
#pragma unroll
                    for (int t = 0; t < NT; ++t) v[t] = to_f<Tv>(src[t * BWx]);
                    float* dst = sV + iyl * R * ICp + cx;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        float a = 0.f;
#pragma unroll
                        for (int t = 0; t < NT; ++t) a = fmaf(w[j][t], v[t], a);
                        dst[j * ICp] = a;
                    }
                }
            }
        }
        __syncthreads();
        // ---- dWx: a window per thread, over its group's output rows
        if (wact && iw < geo.nwx) {
            const int nrow = geo.nwy * R;
            const Tv* gp = Gt + geo.goff + iw * R;
            const float* vp = sV + iw * SX;
            for (int oyl = gw; oyl < nrow; oyl += GW) {
                float gv[R], v[NT];
#pragma unroll
                for (int j = 0; j < R; ++j) gv[j] = to_f<Tv>(gp[oyl * BWg + j]);
#pragma unroll
                for (int t = 0; t < NT; ++t) v[t] = vp[oyl * ICp + t];
#pragma unroll
                for (int j = 0; j < R; ++j)
#pragma unroll
                    for (int t = 0; t < NT; ++t) accx[j][t] = fmaf(gv[j], v[t], accx[j][t]);
            }
        }
        // ---- dWy: a column per thread, over its group's windows
        {
            const int GO = blockDim.x / OX;
            const int o = threadIdx.x % OX, go = threadIdx.x / OX;
            if (go < GO && o / R < geo.nwx) {
                const Tv* gp = Gt + geo.goff + o;
                const float* up = sU + o;
                for (int iyl = go; iyl < geo.nwy; iyl += GO) {
                    float gv[R], u[NT];
#pragma unroll
                    for (int j = 0; j < R; ++j) gv[j] = to_f<Tv>(gp[(iyl * R + j) * BWg]);
#pragma unroll
                    for (int t = 0; t < NT; ++t) u[t] = up[(iyl * SY + t) * OX];
#pragma unroll
                    for (int j = 0; j < R; ++j)
#pragma unroll
                        for (int t = 0; t < NT; ++t) accy[j][t] = fmaf(gv[j], u[t], accy[j][t]);
                }
            }
        }
        __syncthreads();  // buffers free for the copies two tiles ahead
    }
    if (cur_c >= 0) {
        __syncthreads();
        flush(seg++, cur_c);
    }
    if (threadIdx.x == 0)
        for (int s2 = seg; s2 < T.maxseg; ++s2) ids[s2] = -1;
}

// Fixed-order sum of the records of every weight entry (compensated, then a
// shuffle tree); one warp per entry.
__global__ void __launch_bounds__(256) fcfs_dw_reduce_tma(const __grid_constant__ TmaDwParams T) {
    const FwdParams& P = T.P;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nrec = (long long)T.grid * T.maxseg;
    const int* ids = reinterpret_cast<const int*>(T.ws + nrec * T.rec);
    long long base = 0;
    for (int a = 2; a >= 1; --a) {
        const AxisP& A = P.ax[a];
        if (T.gw[a] == nullptr) continue;
        const long long per = (long long)A.r * A.nt_src;
        const long long nch = A.w_cstride ? P.C : 1;
        if (wid >= base + nch * per) {
            base += nch * per;
            continue;
        }
        const long long idx = wid - base;
        const int ch = (int)(idx / per);
        const int jt = (int)(idx - ch * per);
        const int j = jt / A.nt_src, k = jt - j * A.nt_src;
        const int roff = (a == 2 ? P.ax[1].r * A.nt : 0) + j * A.nt + k;
        float s = 0.f, comp = 0.f;
        for (long long m = lane; m < nrec; m += 32) {
            const int id = ids[m];
            if (id < 0 || (A.w_cstride && id != ch)) continue;
            const float y = T.ws[m * T.rec + roff] - comp;
            const float tsum = s + y;
            comp = (tsum - s) - y;
            s = tsum;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) T.gw[a][idx] = s;
        return;
    }
}

}  // namespace

#define FCFS_DW_NT_CASES(X) X(1) X(2) X(3) X(4) X(5) X(7) X(9)

// (R, taps) pairs of the register-blocked weight gradient
#define FCFS_DW_RB_CASES(X) X(2, 5) X(3, 5) X(4, 5) X(5, 5) X(3, 7) X(5, 7) X(5, 3)

bool dw_rb_compiled(int r, int nt) {
#define CASE(a, b) \
    if (r == a && nt == b) return true;
    FCFS_DW_RB_CASES(CASE)
#undef CASE
    return false;
}

cudaError_t launch_dw_tma(const TmaDwParams& T, int nt, int dt, cudaStream_t st, const void* x) {
    const size_t smem = (size_t)T.bar_off + 16;
    auto go = [&](auto tv) -> cudaError_t {
        using Tv = std::remove_pointer_t<decltype(tv)>;
        cudaError_t e = cudaSuccess;
        bool done = false;
        if (T.rb) {
#define CASE(a, b)                                                                            \
    if (!done && T.rb == a && nt == b) {                                                      \
        auto k = fcfs_bwd_dw2d_rb<a, b, Tv>;                                                  \
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
        if (e != cudaSuccess) return e;                                                       \
        k<<<T.grid, T.threads, smem, st>>>(T, x);                                             \
        done = true;                                                                          \
    }
            FCFS_DW_RB_CASES(CASE)
#undef CASE
            if (!done) return cudaErrorInvalidValue;
        }
        if (!done) switch (nt) {
#define CASE(N)                                                                                          \
    case N: {                                                                                            \
        auto k = fcfs_bwd_dw2d_tma<N, Tv>;                                                               \
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
        if (e != cudaSuccess) return e;                                                                  \
        k<<<T.grid, T.threads, smem, st>>>(T, x);                                                        \
        break;                                                                                           \
    }
            FCFS_DW_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        long long entries = 0;
        for (int a = 1; a <= 2; ++a)
            if (T.gw[a]) entries += (long long)(T.P.ax[a].w_cstride ? T.P.C : 1) * T.P.ax[a].r * T.P.ax[a].nt_src;
        if (entries == 0) return cudaSuccess;
        fcfs_dw_reduce_tma<<<(unsigned)((entries * 32 + 255) / 256), 256, 0, st>>>(T);
        return cudaGetLastError();
    };
    if (dt == FCFS_F32) return go((float*)nullptr);
    if (dt == FCFS_BF16) return go((__nv_bfloat16*)nullptr);
    return cudaErrorInvalidValue;
}

}  // namespace fcfs
