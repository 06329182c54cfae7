// Backward FCFS kernels (gradients of the Sec. 3.1 / Sec. 4 layer, needed
// to learn the kernel weights as Sec. 7 proposes):
//   K4 fcfs_bwd_dx2d / fcfs_bwd_dx3d - input gradient as a gather: the
//        pixel-unshuffle and the transposed strided convolution are one
//        polyphase pass per axis, followed by the pad adjoint (fold);
//   K5 fcfs_bwd_dw2d - per-CTA weight-gradient partials (registers, then a
//        fixed-order shared-memory/warp-shuffle reduction), and
//        fcfs_dw_reduce - a deterministic second pass over the partials.
#include <type_traits>

#include "fcfs_internal.cuh"

namespace fcfs {

namespace {

__device__ __forceinline__ int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int NT>
__device__ __forceinline__ void stage_w(float* dst, const AxisP& A, int c) {
    const int n = A.r * NT;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int j = k / NT, t = k - j * NT;
        float v = 0.f;
        if (t < A.nt_src) v = A.learn ? A.w[(long long)c * A.w_cstride + j * A.nt_src + t] : A.wf[j * A.nt_src + t];
        dst[k] = v;
    }
}

// Adjoint of one axis at extended index v, read from a shared-memory row of
// g values for windows [ilo, ...]: sum over the entries of v's residue.
template <int NT>
__device__ __forceinline__ float adj_at(const AxisP& A, const AdjAxis& J, const float* sw, const float* row,
                                        int stride, int v, int ilo, int ihi) {
    const int d = v - A.lo;
    const int a = fdiv(d, A.s);
    const int u = d - a * A.s;
    float acc = 0.f;
    for (int e = J.ustart[u]; e < J.ustart[u + 1]; ++e) {
        const int en = J.ent[e];
        const int i = a - (en >> 16);
        if (i < ilo || i > ihi) continue;
        const int j = (en >> 8) & 0xff, t = en & 0xff;
        acc = fmaf(sw[j * NT + t], row[((i - ilo) * A.r + j) * stride], acc);
    }
    return acc;
}

// Adjoint plus fold of one axis at real index q: every extended index v in
// the window range with ext(v) == q contributes.
template <int NT>
__device__ __forceinline__ float adj_fold(const AxisP& A, const AdjAxis& J, const float* sw, const float* row,
                                          int stride, int q, const WinRange& w, int pad) {
    float acc = 0.f;
    if (q >= J.vmin && q <= J.vmax) acc = adj_at<NT>(A, J, sw, row, stride, q, w.ilo, w.ihi);
    if (w.left)
        for (int v = J.vmin; v < 0; ++v)
            if (ext_index(v, A.n_in, pad) == q) acc += adj_at<NT>(A, J, sw, row, stride, v, w.ilo, w.ihi);
    if (w.right)
        for (int v = A.n_in; v <= J.vmax; ++v)
            if (ext_index(v, A.n_in, pad) == q) acc += adj_at<NT>(A, J, sw, row, stride, v, w.ilo, w.ihi);
    return acc;
}

// Stage the g tile rows [row0, row0+rows) x cols [col0, col0+cols) of one
// plane into shared memory as FP32; indices past the output are zero (the
// surplus phases of the last window have no output).
template <typename Tg>
__device__ __forceinline__ void stage_g(float* sG, int pitch, const Tg* gp, int Ho, int Wo, int row0, int rows,
                                        int col0, int cols) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int r = warp; r < rows; r += nwarp) {
        const int gr = row0 + r;
        float* dst = sG + r * pitch;
        if (gp == nullptr || gr >= Ho) {
            for (int cx = lane; cx < cols; cx += 32) dst[cx] = 0.f;
            continue;
        }
        const Tg* src = gp + (long long)gr * Wo;
        for (int cx = lane; cx < cols; cx += 32) {
            const int gc = col0 + cx;
            dst[cx] = gc < Wo ? load_f(src + gc) : 0.f;
        }
    }
}

// x then y adjoint (with folds) of one (y, x) tile of a staged g plane; each
// result goes to store(qyl, qxl, value).
template <int NT, typename Store>
__device__ __forceinline__ void dx_plane(const BwdParams& P, const float* sWx, const float* sWy, const float* sG,
                                         float* sF, int qx0, int qy0, int nqx, int nqy, const WinRange& wx,
                                         const WinRange& wy, Store store) {
    const AxisP& AX = P.ax[2];
    const AxisP& AY = P.ax[1];
    const int QX = P.QX;
    const int qxl = threadIdx.x % QX, g = threadIdx.x / QX, G = blockDim.x / QX;
    const int GR = (wy.ihi - wy.ilo + 1) * AY.r;
    if (qxl < nqx) {
        for (int gr = g; gr < GR; gr += G)
            sF[gr * QX + qxl] = adj_fold<NT>(AX, P.adj[2], sWx, sG + gr * P.GCp, 1, qx0 + qxl, wx, P.pad);
    }
    __syncthreads();
    if (qxl < nqx) {
        for (int qyl = g; qyl < nqy; qyl += G)
            store(qyl, qxl, adj_fold<NT>(AY, P.adj[1], sWy, sF + qxl, QX, qy0 + qyl, wy, P.pad));
    }
}

template <int NT, typename Tg, typename Tx>
__global__ void __launch_bounds__(512) fcfs_bwd_dx2d(const __grid_constant__ BwdParams P) {
    extern __shared__ float smem[];
    const AxisP& AX = P.ax[2];
    const AxisP& AY = P.ax[1];
    long long t = blockIdx.x;
    const int tx = (int)(t % P.qtiles_x);
    t /= P.qtiles_x;
    const int ty = (int)(t % P.qtiles_y);
    const long long plane = t / P.qtiles_y;
    const int c = (int)(plane % P.C);

    float* sWx = smem;
    float* sWy = sWx + AX.r * NT;
    float* sG = sWy + AY.r * NT;
    float* sF = sG + P.GRcap * P.GCp;

    const int qx0 = P.rqx0 + tx * P.QX, qy0 = P.rqy0 + ty * P.QY;
    const int nqx = min(P.QX, P.rqx1 - qx0), nqy = min(P.QY, P.rqy1 - qy0);
    const WinRange wx = win_range(AX, P.adj[2], P.pad, qx0, qx0 + nqx - 1);
    const WinRange wy = win_range(AY, P.adj[1], P.pad, qy0, qy0 + nqy - 1);

    stage_w<NT>(sWx, AX, c);
    stage_w<NT>(sWy, AY, c);
    const Tg* gp = static_cast<const Tg*>(P.gy) + plane * (long long)AY.n_out * AX.n_out;
    const int GR = (wy.ihi - wy.ilo + 1) * AY.r, GC = (wx.ihi - wx.ilo + 1) * AX.r;
    stage_g<Tg>(sG, P.GCp, (wx.ihi < wx.ilo || wy.ihi < wy.ilo) ? nullptr : gp, AY.n_out, AX.n_out,
                wy.ilo * AY.r, max(GR, 0), wx.ilo * AX.r, max(GC, 0));
    __syncthreads();
    Tx* xo = static_cast<Tx*>(P.gx) + plane * (long long)AY.n_in * AX.n_in + (long long)qy0 * AX.n_in + qx0;
    const int W = AX.n_in;
    dx_plane<NT>(P, sWx, sWy, sG, sF, qx0, qy0, nqx, nqy, wx, wy,
                 [&](int qyl, int qxl, float v) { store_f(xo + (long long)qyl * W + qxl, v); });
}

// 3D input gradient: a CTA owns a (QY x QX) tile of real input positions and
// QD real depth planes.  The (y, x) adjoint of each needed g depth plane is
// kept in a tagged ring; each real depth plane combines the ring entries of
// its depth windows (adjoint + fold along depth).
template <int NT, typename Tg, typename Tx>
__global__ void __launch_bounds__(512) fcfs_bwd_dx3d(const __grid_constant__ BwdParams P) {
    extern __shared__ float smem[];
    __shared__ int tags[256];
    const AxisP& AX = P.ax[2];
    const AxisP& AY = P.ax[1];
    const AxisP& AD = P.ax[0];
    long long t = blockIdx.x;
    const int tx = (int)(t % P.qtiles_x);
    t /= P.qtiles_x;
    const int ty = (int)(t % P.qtiles_y);
    t /= P.qtiles_y;
    const int td = (int)(t % P.qtiles_d);
    const long long plane = t / P.qtiles_d;
    const int c = (int)(plane % P.C);

    float* sWx = smem;
    float* sWy = sWx + AX.r * NT;
    float* sWd = sWy + AY.r * NT;
    float* sG = sWd + AD.r * NT;
    float* sF = sG + P.GRcap * P.GCp;
    float* ring = sF + P.GRcap * P.QX;
    const int QX = P.QX, QY = P.QY;
    const int psz = QX * QY;

    const int qx0 = tx * P.QX, qy0 = ty * P.QY, qd0 = td * P.QD;
    const int nqx = min(P.QX, AX.n_in - qx0), nqy = min(P.QY, AY.n_in - qy0), nqd = min(P.QD, AD.n_in - qd0);
    const WinRange wx = win_range(AX, P.adj[2], P.pad, qx0, qx0 + nqx - 1);
    const WinRange wy = win_range(AY, P.adj[1], P.pad, qy0, qy0 + nqy - 1);
    stage_w<NT>(sWx, AX, c);
    stage_w<NT>(sWy, AY, c);
    stage_w<NT>(sWd, AD, c);
    for (int k = threadIdx.x; k < P.GDcap; k += blockDim.x) tags[k] = -1;
    __syncthreads();

    const long long oplane = (long long)AY.n_out * AX.n_out;
    const Tg* gvol = static_cast<const Tg*>(P.gy) + plane * (long long)AD.n_out * oplane;
    Tx* xvol = static_cast<Tx*>(P.gx) + plane * (long long)AD.n_in * AY.n_in * AX.n_in;
    const int GR = (wy.ihi - wy.ilo + 1) * AY.r, GC = (wx.ihi - wx.ilo + 1) * AX.r;
    const bool empty_yx = wx.ihi < wx.ilo || wy.ihi < wy.ilo;
    const int qxl = threadIdx.x % QX, g = threadIdx.x / QX, G = blockDim.x / QX;

    for (int qdl = 0; qdl < nqd; ++qdl) {
        const int qd = qd0 + qdl;
        const WinRange wd = win_range(AD, P.adj[0], P.pad, qd, qd);
        // make sure every g depth plane of windows [wd.ilo, wd.ihi] is in the ring
        for (int gd = wd.ilo * AD.r; gd <= wd.ihi * AD.r + AD.r - 1; ++gd) {
            if (gd >= AD.n_out) break;
            const int slot = gd % P.GDcap;
            if (tags[slot] == gd) continue;
            stage_g<Tg>(sG, P.GCp, empty_yx ? nullptr : gvol + (long long)gd * oplane, AY.n_out, AX.n_out,
                        wy.ilo * AY.r, max(GR, 0), wx.ilo * AX.r, max(GC, 0));
            __syncthreads();
            float* dst = ring + slot * psz;
            dx_plane<NT>(P, sWx, sWy, sG, sF, qx0, qy0, nqx, nqy, wx, wy,
                         [&](int qyl, int qxl, float v) { dst[qyl * QX + qxl] = v; });
            __syncthreads();
            if (threadIdx.x == 0) tags[slot] = gd;
            __syncthreads();
        }
        // depth adjoint + fold over the ring: the ring rows play the role of g
        if (qxl < nqx) {
            for (int qyl = g; qyl < nqy; qyl += G) {
                float acc = 0.f;
                const int off = qyl * QX + qxl;
                // visit extended depth indices folding onto qd
                auto visit = [&](int v) {
                    const int d = v - AD.lo;
                    const int a = fdiv(d, AD.s);
                    const int u = d - a * AD.s;
                    float s = 0.f;
                    for (int e = P.adj[0].ustart[u]; e < P.adj[0].ustart[u + 1]; ++e) {
                        const int en = P.adj[0].ent[e];
                        const int i = a - (en >> 16);
                        if (i < wd.ilo || i > wd.ihi) continue;
                        const int j = (en >> 8) & 0xff, tt = en & 0xff;
                        const int gd = i * AD.r + j;
                        if (gd >= AD.n_out) continue;
                        s = fmaf(sWd[j * NT + tt], ring[(gd % P.GDcap) * psz + off], s);
                    }
                    return s;
                };
                if (qd >= P.adj[0].vmin && qd <= P.adj[0].vmax) acc = visit(qd);
                if (wd.left)
                    for (int v = P.adj[0].vmin; v < 0; ++v)
                        if (ext_index(v, AD.n_in, P.pad) == qd) acc += visit(v);
                if (wd.right)
                    for (int v = AD.n_in; v <= P.adj[0].vmax; ++v)
                        if (ext_index(v, AD.n_in, P.pad) == qd) acc += visit(v);
                store_f(xvol + ((long long)qd * AY.n_in + qy0 + qyl) * AX.n_in + qx0 + qxl, acc);
            }
        }
        __syncthreads();
    }
}

// Weight-gradient partials of one output tile (same tiling as the forward).
//   dWx[jx][t] += g[oy][ox] * V[oy][ixl*s_x + off_x[jx] + t],  V = y taps of x~
//   dWy[jy][t] += g[oy][ox] * U[iyl*s_y + off_y[jy] + t][ox],  U = x taps of x~
// Each CTA writes one record of r_y*NT + r_x*NT floats.
template <int NT, typename Tin, typename Tg>
__global__ void __launch_bounds__(512) fcfs_bwd_dw2d(const __grid_constant__ BwdParams B) {
    extern __shared__ float smem[];
    const FwdParams& P = B.fw;
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    long long t = blockIdx.x;
    const int tx = (int)(t % P.tiles_x);
    t /= P.tiles_x;
    const int ty = (int)(t % P.tiles_y);
    const long long plane = t / P.tiles_y;
    const int c = (int)(plane % P.C);
    const int OX = P.OX, OY = P.OY, G = P.G;

    float* sWx = smem;
    float* sWy = sWx + AX.r * NT;
    float* sIn = sWy + AY.r * NT;
    float* sU = sIn + P.IR * P.ICp;
    float* sV = sU + P.IR * OX;
    float* sGt = sV + OY * P.ICp;
    float* sRx = sGt + OY * OX;
    float* sRy = sRx + G * OX * NT;

    const int ix0 = tx * P.WX, iy0 = ty * P.WY;
    const int nwx = min(P.WX, AX.n_win - ix0), nwy = min(P.WY, AY.n_win - iy0);
    const int cols = (nwx - 1) * AX.s + AX.span, rows = (nwy - 1) * AY.s + AY.span;
    const int col0 = ix0 * AX.s + AX.lo, row0 = iy0 * AY.s + AY.lo;

    stage_w<NT>(sWx, AX, c);
    stage_w<NT>(sWy, AY, c);
    // x~ tile
    {
        const Tin* xp = static_cast<const Tin*>(B.x) + plane * (long long)AY.n_in * AX.n_in;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        for (int ry = warp; ry < rows; ry += nwarp) {
            const int sy = ext_index(row0 + ry, AY.n_in, P.pad);
            float* dst = sIn + ry * P.ICp;
            for (int cx = lane; cx < cols; cx += 32) {
                const int sx = ext_index(col0 + cx, AX.n_in, P.pad);
                dst[cx] = (sy < 0 || sx < 0) ? P.padv : load_f(xp + (long long)sy * AX.n_in + sx);
            }
        }
    }
    const Tg* gp = static_cast<const Tg*>(B.gy) + plane * (long long)AY.n_out * AX.n_out;
    stage_g<Tg>(sGt, OX, gp, AY.n_out, AX.n_out, iy0 * AY.r, nwy * AY.r, ix0 * AX.r, nwx * AX.r);
    __syncthreads();

    const int ox = threadIdx.x % OX, g = threadIdx.x / OX;
    const int jx = ox % AX.r, ixl = ox / AX.r;
    // U = x taps of every staged row
    if (ixl < nwx) {
        for (int ry = g; ry < rows; ry += G) {
            const float* row = sIn + ry * P.ICp + ixl * AX.s + AX.off[jx];
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < NT; ++k) acc = fmaf(sWx[jx * NT + k], row[k], acc);
            sU[ry * OX + ox] = acc;
        }
    }
    // V = y taps of every staged column
    const int nrow_out = nwy * AY.r;
    for (int e = threadIdx.x; e < nrow_out * cols; e += blockDim.x) {
        const int oyl = e / cols, col = e - oyl * cols;
        const int iyl = oyl / AY.r, jy = oyl - iyl * AY.r;
        const float* src = sIn + (iyl * AY.s + AY.off[jy]) * P.ICp + col;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NT; ++k) acc = fmaf(sWy[jy * NT + k], src[k * P.ICp], acc);
        sV[oyl * P.ICp + col] = acc;
    }
    __syncthreads();

    // dWx: thread (ox, g) over output rows of its group
    {
        float acc[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) acc[k] = 0.f;
        if (ixl < nwx) {
            const int cb = ixl * AX.s + AX.off[jx];
            for (int oyl = g; oyl < nrow_out; oyl += G) {
                const float gv = sGt[oyl * OX + ox];
                const float* v = sV + oyl * P.ICp + cb;
#pragma unroll
                for (int k = 0; k < NT; ++k) acc[k] = fmaf(gv, v[k], acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < NT; ++k) sRx[(g * OX + ox) * NT + k] = acc[k];
    }
    // dWy: pairs (jy, ox), each over the windows of the tile
    for (int p = threadIdx.x; p < AY.r * OX; p += blockDim.x) {
        const int jy = p / OX, oxx = p - jy * OX;
        float acc[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) acc[k] = 0.f;
        if (oxx / AX.r < nwx) {
            for (int iyl = 0; iyl < nwy; ++iyl) {
                const float gv = sGt[(iyl * AY.r + jy) * OX + oxx];
                const float* u = sU + (iyl * AY.s + AY.off[jy]) * OX + oxx;
#pragma unroll
                for (int k = 0; k < NT; ++k) acc[k] = fmaf(gv, u[k * OX], acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < NT; ++k) sRy[p * NT + k] = acc[k];
    }
    __syncthreads();

    // fixed-order reduction: one warp per (axis, phase, tap), lanes stride the
    // contributors, then a shuffle tree
    float* rec = B.ws + blockIdx.x * (long long)B.dw_rec;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int nx = AX.r * NT, ny = AY.r * NT;
    for (int q = warp; q < nx + ny; q += nwarp) {
        float s = 0.f;
        if (q < nx) {
            const int j = q / NT, k = q - j * NT;
            for (int m = lane; m < G * nwx; m += 32) {
                const int gg = m / nwx, il = m - gg * nwx;
                s += sRx[(gg * OX + il * AX.r + j) * NT + k];
            }
        } else {
            const int qq = q - nx;
            const int j = qq / NT, k = qq - j * NT;
            for (int o = lane; o < OX; o += 32) s += sRy[(j * OX + o) * NT + k];
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) rec[q < nx ? B.dw_axis_off[2] + q : B.dw_axis_off[1] + (q - nx)] = s;
    }
}

// Sum the CTA records of each weight entry in a fixed order: one warp per
// entry, lanes stride the records with compensated sums, then a shuffle tree.
__global__ void __launch_bounds__(256) fcfs_dw_reduce(const __grid_constant__ BwdParams B) {
    const FwdParams& P = B.fw;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // entries: axis 2 (x) then axis 1 (y), each [C or 1][r][nt_src]
    long long base = 0;
    for (int a = 2; a >= 1; --a) {
        const AxisP& A = P.ax[a];
        if (B.gw[a] == nullptr) continue;
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
        const int roff = B.dw_axis_off[a] + j * A.nt + k;
        const long long tiles = (long long)P.tiles_x * P.tiles_y;
        const long long nrec = A.w_cstride ? B.n * tiles : P.planes * tiles;
        float s = 0.f, comp = 0.f;
        for (long long m = lane; m < nrec; m += 32) {
            long long recidx;
            if (A.w_cstride) {
                const long long nn = m / tiles, tt = m - nn * tiles;
                recidx = (nn * P.C + ch) * tiles + tt;
            } else {
                recidx = m;
            }
            const float y = B.ws[recidx * B.dw_rec + roff] - comp;
            const float tsum = s + y;
            comp = (tsum - s) - y;
            s = tsum;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) B.gw[a][idx] = s;
        return;
    }
}

template <typename F>
cudaError_t dispatch_bwd_types(int d1, int d2, F&& f) {
    if (d1 == FCFS_F32 && d2 == FCFS_F32) return f((float*)nullptr, (float*)nullptr);
    if (d1 == FCFS_BF16 && d2 == FCFS_BF16) return f((__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr);
    if (d1 == FCFS_F32 && d2 == FCFS_BF16) return f((float*)nullptr, (__nv_bfloat16*)nullptr);
    if (d1 == FCFS_BF16 && d2 == FCFS_F32) return f((__nv_bfloat16*)nullptr, (float*)nullptr);
    return cudaErrorInvalidValue;
}

template <typename K>
cudaError_t launch_k(K k, long long blocks, int threads, size_t smem, cudaStream_t st, const BwdParams& P) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)blocks, threads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

size_t dx_smem_bytes(const BwdParams& P, bool is3d) {
    const int nt = P.ax[2].nt;
    size_t f = (size_t)(P.ax[2].r + P.ax[1].r + (is3d ? P.ax[0].r : 0)) * nt;
    f += (size_t)P.GRcap * P.GCp + (size_t)P.GRcap * P.QX;
    if (is3d) f += (size_t)P.GDcap * P.QX * P.QY;
    return f * sizeof(float);
}

size_t dw_smem_bytes(const BwdParams& B) {
    const FwdParams& P = B.fw;
    const int nt = P.ax[2].nt;
    size_t f = (size_t)(P.ax[2].r + P.ax[1].r) * nt;
    f += (size_t)P.IR * P.ICp + (size_t)P.IR * P.OX + (size_t)P.OY * P.ICp + (size_t)P.OY * P.OX;
    f += (size_t)P.G * P.OX * nt + (size_t)P.ax[1].r * P.OX * nt;
    return f * sizeof(float);
}

#define FCFS_NT_CASES(X) X(1) X(2) X(3) X(4) X(5) X(7) X(9)

cudaError_t launch_dx(const BwdParams& P, int nt, int dg, int dx, bool is3d, cudaStream_t st) {
    const size_t smem = dx_smem_bytes(P, is3d);
    const long long blocks = (long long)P.qtiles_x * P.qtiles_y * (is3d ? P.qtiles_d : 1) * P.planes;
    const int threads = P.QX * P.Gq;
    return dispatch_bwd_types(dg, dx, [&](auto tg, auto tx) -> cudaError_t {
        using Tg = std::remove_pointer_t<decltype(tg)>;
        using Tx = std::remove_pointer_t<decltype(tx)>;
        switch (nt) {
#define CASE(N)                                                                         \
    case N:                                                                             \
        return is3d ? launch_k(fcfs_bwd_dx3d<N, Tg, Tx>, blocks, threads, smem, st, P) \
                    : launch_k(fcfs_bwd_dx2d<N, Tg, Tx>, blocks, threads, smem, st, P);
            FCFS_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    });
}

cudaError_t launch_dw(const BwdParams& P, int nt, int din, int dg, cudaStream_t st) {
    const size_t smem = dw_smem_bytes(P);
    const long long blocks = (long long)P.fw.tiles_x * P.fw.tiles_y * P.planes;
    const int threads = P.fw.OX * P.fw.G;
    return dispatch_bwd_types(din, dg, [&](auto ti, auto tg) -> cudaError_t {
        using Tin = std::remove_pointer_t<decltype(ti)>;
        using Tg = std::remove_pointer_t<decltype(tg)>;
        switch (nt) {
#define CASE(N) \
    case N: return launch_k(fcfs_bwd_dw2d<N, Tin, Tg>, blocks, threads, smem, st, P);
            FCFS_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    });
}

cudaError_t launch_dw_reduce(const BwdParams& P, cudaStream_t st) {
    long long entries = 0;
    for (int a = 1; a <= 2; ++a) {
        if (!P.gw[a]) continue;
        const AxisP& A = P.fw.ax[a];
        entries += (long long)(A.w_cstride ? P.C : 1) * A.r * A.nt_src;
    }
    if (entries == 0) return cudaSuccess;
    const long long threads = entries * 32;
    fcfs_dw_reduce<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace fcfs
