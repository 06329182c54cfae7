// Shared pieces of the bulk-copy 3D forward kernels (Sec. 4, separable
// per-axis kernels): tile geometry, padding of staged planes, the job stream
// of (tile, input depth plane) pairs and its multi-stage copy issue.
#pragma once

#include "fcfs_fwd_tma.cuh"

namespace fcfs {

// Device status word of the 3D bulk-copy kernels (bounded waits); each
// translation unit that includes this header owns its copy.
static __device__ int g_status_fwd3d = 0;

namespace {

struct Geo3 {
    int plane, c, ix0, iy0, id0, nwx, nwy, nwd, rows, cols, row0, col0, x_al, xoff, p_first, p_last;
    bool edge;
};

__device__ __forceinline__ Geo3 geo3(const TmaFwd3Params& T, int tile) {
    const FwdParams& P = T.P;
    const AxisP &AD = P.ax[0], &AY = P.ax[1], &AX = P.ax[2];
    Geo3 g;
    int t = tile;
    const int tx = t % P.tiles_x;
    t /= P.tiles_x;
    const int ty = t % P.tiles_y;
    t /= P.tiles_y;
    const int td = t % P.tiles_d;
    g.plane = t / P.tiles_d;
    g.c = g.plane % P.C;
    g.ix0 = tx * P.WX;
    g.iy0 = ty * P.WY;
    g.id0 = td * P.WD;
    g.nwx = min(P.WX, AX.n_win - g.ix0);
    g.nwy = min(P.WY, AY.n_win - g.iy0);
    g.nwd = min(P.WD, AD.n_win - g.id0);
    g.cols = (g.nwx - 1) * AX.s + AX.span;
    g.rows = (g.nwy - 1) * AY.s + AY.span;
    g.col0 = g.ix0 * AX.s + AX.lo;
    g.row0 = g.iy0 * AY.s + AY.lo;
    g.x_al = g.col0 >= 0 ? (g.col0 / T.align) * T.align : -(((-g.col0) + T.align - 1) / T.align) * T.align;
    g.xoff = g.col0 - g.x_al;
    g.edge = g.col0 < 0 || g.col0 + g.cols > AX.n_in || g.row0 < 0 || g.row0 + g.rows > AY.n_in;
    g.p_first = g.id0 * AD.s + AD.lo;
    g.p_last = (g.id0 + g.nwd - 1) * AD.s + AD.lo + AD.span - 1;
    return g;
}

// (y, x) padding of an edge plane tile in shared memory; depth is remapped at
// the copy.  Reflect re-gathers from the remapped plane.
template <typename Tin>
__device__ __forceinline__ void fix_edges3(const TmaFwd3Params& T, const Geo3& g, Tin* buf, int sd) {
    const FwdParams& P = T.P;
    const int H = P.ax[1].n_in, W = P.ax[2].n_in, D = P.ax[0].n_in;
    const int BW = T.BW;
    // only the columns the x taps read: [0, xoff + cols) of the box
    const int BU = min(BW, g.xoff + g.cols);
    if (P.pad == FCFS_PAD_REFLECT) {
        const Tin* xp = static_cast<const Tin*>(P.x) + ((long long)g.plane * D + sd) * H * W;
        for (int e = threadIdx.x; e < g.rows * BU; e += blockDim.x) {
            const int ry = e / BU, cx = e - ry * BU;
            buf[ry * BW + cx] = xp[(long long)ext_index(g.row0 + ry, H, P.pad) * W + ext_index(g.x_al + cx, W, P.pad)];
        }
        __syncthreads();
        return;
    }
    const bool repl = P.pad == FCFS_PAD_REPLICATE;
    const Tin cv = from_f<Tin>(P.padv);
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

template <typename Tin>
__device__ __forceinline__ void issue3(const TmaFwd3Params& T, const Geo3& g, int p, Tin* buf, uint64_t* bar) {
    const AxisP& AD = T.P.ax[0];
    int sd = ext_index(p, AD.n_in, T.P.pad);
    if (sd < 0) sd = 0;  // constant padding in depth: overwritten after the copy
    fence_proxy_async_smem();
    mbar_expect_tx(bar, (uint32_t)(T.BW * T.BH * sizeof(Tin)));
    tma_load_4d(buf, &T.tmap, g.x_al, g.row0, sd, g.plane, bar);
}

template <int NT>
__device__ __forceinline__ void stage3(float* dst, const AxisP& A, int c) {
    for (int e = threadIdx.x; e < A.r * NT; e += blockDim.x) {
        const int j = e / NT, t = e - j * NT;
        dst[e] = t < A.nt_src ? (A.learn ? A.w[(long long)c * A.w_cstride + j * A.nt_src + t] : A.wf[j * A.nt_src + t]) : 0.f;
    }
}

// Issue cursor of the job stream, kept by thread 0 in shared memory.
struct Cursor3 {
    Geo3 g;     // geometry of the tile being issued
    int tile;   // this CTA's tile number (TileDeal index) of the last issued job
    int p;      // plane of the last issued job
    int n;      // jobs issued so far
    int k;      // stage of the next job to issue
};

// Issue the next job of the stream over this CTA's tiles into stage n % stages.
template <typename Tin>
__device__ __forceinline__ void issue_next(const TmaFwd3Params& T, Cursor3& c, const TileDeal& d, unsigned char* smem,
                                           uint64_t* bars) {
    if (c.tile >= d.n) return;
    if (c.n > 0) {
        if (++c.p > c.g.p_last) {
            if (++c.tile >= d.n) return;
            c.g = geo3(T, d.tile(c.tile));
            c.p = c.g.p_first;
        }
    }
    issue3<Tin>(T, c.g, c.p, reinterpret_cast<Tin*>(smem + c.k * T.buf_bytes), &bars[c.k]);
    ++c.n;
    if (++c.k == T.stages) c.k = 0;
}

}  // namespace
}  // namespace fcfs
