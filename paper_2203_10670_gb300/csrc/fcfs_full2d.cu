// Non-separable 2D FCFS: the 2D convolution of Sec. 4 with one general
// T_y x T_x kernel per phase pair (j_y, j_x) instead of the outer product of
// two axis kernels, the learnable form that lets training change the shape of
// the interpolation kernel (Sec. 7):
//   y[n,c, iy r_y + jy, ix r_x + jx] = sum_{my,mx} W[c][jy][jx][my][mx]
//                                      x~[n,c, iy s_y - L_y + my, ix s_x - L_x + mx]
//   K7 fcfs_full2d_fwd       - padded input tile staged through the index map
//                              with its columns split by residue mod s_x (the
//                              windows of a warp then read consecutive words),
//                              NPH phases of two windows per thread, kernel
//                              weights as shared-memory broadcasts;
//   K8 fcfs_full2d_dx        - input gradient: for every extended index the
//                              windows and taps reaching it are gathered from a
//                              phase-major g tile, four phases per step, then
//                              the pad adjoint folds the virtual cells into the
//                              real ones;
//   K9 fcfs_full2d_dw        - weight-gradient partials, each thread a 4-phase
//                              x 4-tap block of outer products over its share of
//                              the windows (one record per CTA),
//      fcfs_full2d_dw_reduce - fixed-order FP64 reduction of the records.
// No atomics anywhere: every result is bitwise reproducible run to run.
#include <algorithm>
#include <climits>
#include <map>

#include "fcfs_fwd_tile.cuh"
#include "fcfs_host.h"

namespace fcfs {

namespace {

constexpr int kF2MaxExtra = 48;  // pad-fold entries per axis (virtual index -> real index)
constexpr int kF2MaxEntries = 4096;  // r_y r_x T_y T_x per channel
constexpr int kF2FwdWX = 64;  // windows per forward tile row: two per lane

struct F2Axis {
    int n_in, n_out, r, s, T, L, nw;  // nw = ceil(n_out / r) windows
    int next;                         // virtual indices outside [0, n_in) that fold to a real one
    int ext_e[kF2MaxExtra], ext_q[kF2MaxExtra];
};

struct F2Params {
    F2Axis ax[2];  // 0 = rows (y), 1 = columns (x)
    long long planes;
    int C, per_channel;
    int P, E, Ppad;  // phases r_y r_x, entries P T_y T_x, phases padded to the vector width
    int pad;
    float padv;
    const float* w;
    const void* x;
    const void* g;
    void* y;
    void* dx;
    float* ws;
    float* dw;
    int WX, WY;  // windows per tile (forward, weight gradient) or real cells per tile (input gradient)
    int tiles_x, tiles_y;
    int VYc, VXc, NWYc, NWXc;  // input gradient: capacities of the virtual range and of the window range
    int nchunk, ngroups;       // weight gradient: records per plane, window groups per CTA
    int npass;                 // weight gradient: CTAs per (plane, chunk) when the blocks exceed one CTA
};

__device__ __forceinline__ int pmod(int a, int b) {
    const int m = a % b;
    return m < 0 ? m + b : m;
}

// Kernel weights of channel c into shared memory, tap-major with the phases
// innermost: dst[(my*T_x + mx)*Ppad + ph] (zero for ph >= P).
__device__ __forceinline__ void f2_stage_weights(float* dst, const F2Params& p, int c) {
    const int TT = p.ax[0].T * p.ax[1].T;
    const float* src = p.w + (p.per_channel ? (long long)c * p.E : 0LL);
    const int n = TT * p.Ppad;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int tap = k / p.Ppad, ph = k - tap * p.Ppad;
        dst[k] = ph < p.P ? __ldg(src + ph * TT + tap) : 0.f;
    }
}

// Input tile [rows][cols] (extended coordinates row0/col0, padding as an
// index map) with each row's columns split by residue mod s: column col is
// stored at (col mod s) * KW + col / s.  Windows ix = 0, 1, ... read columns
// ix*s + m, which then sit at consecutive words.  One warp per row.
template <typename Tin>
__device__ __forceinline__ void f2_load_tile_split(float* dst, int pitch, int KW, int s, const Tin* src_plane, int H,
                                                   int W, int row0, int col0, int rows, int cols, int pad,
                                                   float padv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int q32 = 32 / s, u32 = 32 - q32 * s;
    const int q0 = lane / s, u0 = lane - q0 * s;
    const bool inside_x = col0 >= 0 && col0 + cols <= W;
    for (int ry = warp; ry < rows; ry += nwarp) {
        const int sy = ext_index(row0 + ry, H, pad);
        float* d = dst + ry * pitch;
        const Tin* src = sy >= 0 ? src_plane + (long long)sy * W : nullptr;
        int q = q0, u = u0;
        for (int cx = lane; cx < cols; cx += 32) {
            float v = padv;
            if (src != nullptr) {
                if (inside_x) {
                    v = load_f(src + col0 + cx);
                } else {
                    const int sx = ext_index(col0 + cx, W, pad);
                    if (sx >= 0) v = load_f(src + sx);
                }
            }
            d[u * KW + q] = v;
            q += q32;
            u += u32;
            if (u >= s) {
                u -= s;
                ++q;
            }
        }
    }
}

// ------------------------------------------------------------------ forward

// CT, CS > 0: a compile-time tap count on both axes and x stride (the common shapes), so the tap loops
// unroll and the split-row offsets of the taps fold into constants; 0: read from the parameters.
template <int NPH, typename Tin, typename Tout, int CT = 0, int CS = 0>
__global__ void __launch_bounds__(256) fcfs_full2d_fwd(const __grid_constant__ F2Params p) {
    extern __shared__ float4 f2_smem4[];
    float* sW = reinterpret_cast<float*>(f2_smem4);
    const F2Axis& AY = p.ax[0];
    const F2Axis& AX = p.ax[1];
    const int ntiles = p.tiles_x * p.tiles_y;
    const long long plane = blockIdx.x / ntiles;
    const int tile = (int)(blockIdx.x - plane * ntiles);
    const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
    const int c = (int)(plane % p.C);
    const int iy0 = ty * p.WY, ix0 = tx * p.WX;
    const int TX = CT ? CT : AX.T, TY = CT ? CT : AY.T, SX = CS ? CS : AX.s;
    const int TT = TY * TX, Ppad = p.Ppad;
    const int rows = (p.WY - 1) * AY.s + TY, cols = (p.WX - 1) * SX + TX;
    const int KW = (cols + SX - 1) / SX, pitch = KW * SX;
    float* sIn = sW + TT * Ppad;

    f2_stage_weights(sW, p, c);
    const Tin* xp = reinterpret_cast<const Tin*>(p.x) + plane * (long long)AY.n_in * AX.n_in;
    f2_load_tile_split<Tin>(sIn, pitch, KW, AX.s, xp, AY.n_in, AX.n_in, iy0 * AY.s - AY.L, ix0 * AX.s - AX.L, rows,
                            cols, p.pad, p.padv);
    __syncthreads();

    Tout* yp = reinterpret_cast<Tout*>(p.y) + plane * (long long)AY.n_out * AX.n_out;
    const int nch = Ppad / NPH;
    const int items = p.WY * nch * 32;  // lane l: windows l and l + 32 of the tile row
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int ixl = it & 31, rest = it >> 5;
        const int ch = rest % nch, iyl = rest / nch;
        const int iy = iy0 + iyl, ixa = ix0 + ixl, ixb = ixa + 32;
        if (iy >= AY.nw || ixa >= AX.nw) continue;
        float a[NPH], b[NPH];
#pragma unroll
        for (int k = 0; k < NPH; ++k) a[k] = b[k] = 0.f;
        const float* src = sIn + iyl * AY.s * pitch + ixl;
        const float* wp = sW + ch * NPH;
#pragma unroll
        for (int my = 0; my < TY; ++my) {
            // tap mx sits at (mx mod s) * KW + mx / s of the split row
            int off = 0, u = 0;
            const float* wq = wp;
#pragma unroll
            for (int mx = 0; mx < TX; ++mx) {
                const float v0 = src[off], v1 = src[off + 32];
                float w[NPH];
                if constexpr (NPH == 4) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wq);
                    w[0] = w4.x, w[1] = w4.y, w[2] = w4.z, w[3] = w4.w;
                } else {
#pragma unroll
                    for (int k = 0; k < NPH; ++k) w[k] = wq[k];
                }
#pragma unroll
                for (int k = 0; k < NPH; ++k) {
                    a[k] = fmaf(w[k], v0, a[k]);
                    b[k] = fmaf(w[k], v1, b[k]);
                }
                wq += Ppad;
                off += KW;
                if (++u == SX) {
                    u = 0;
                    off += 1 - SX * KW;
                }
            }
            src += pitch;
            wp += TX * Ppad;
        }
#pragma unroll
        for (int k = 0; k < NPH; ++k) {
            const int ph = ch * NPH + k;
            if (ph < p.P) {
                const int jy = ph / AX.r, jx = ph - jy * AX.r;
                const int oy = iy * AY.r + jy;
                if (oy < AY.n_out) {
                    Tout* row = yp + (long long)oy * AX.n_out;
                    const int oxa = ixa * AX.r + jx, oxb = ixb * AX.r + jx;
                    if (oxa < AX.n_out) store_f(row + oxa, a[k]);
                    if (ixb < AX.nw && oxb < AX.n_out) store_f(row + oxb, b[k]);
                }
            }
        }
    }
}

// ----------------------------------------------------------- input gradient

// Virtual (extended-index) range a real tile [q0, q1) needs along one axis:
// the tile itself plus every pad-fold entry that lands in it.
__device__ __forceinline__ void f2_virtual_range(const F2Axis& A, int q0, int q1, int* vlo, int* vhi, bool* folds) {
    int lo = q0, hi = q1 - 1;
    bool any = false;
    for (int k = 0; k < A.next; ++k) {
        const int q = A.ext_q[k];
        if (q >= q0 && q < q1) {
            lo = imin(lo, A.ext_e[k]);
            hi = imax(hi, A.ext_e[k]);
            any = true;
        }
    }
    *vlo = lo;
    *vhi = hi;
    *folds = any;
}

template <typename Tg, typename Tdx>
__global__ void __launch_bounds__(256) fcfs_full2d_dx(const __grid_constant__ F2Params p) {
    extern __shared__ float4 f2_smem4[];
    float* sW = reinterpret_cast<float*>(f2_smem4);
    const F2Axis& AY = p.ax[0];
    const F2Axis& AX = p.ax[1];
    const int ntiles = p.tiles_x * p.tiles_y;
    const long long plane = blockIdx.x / ntiles;
    const int tile = (int)(blockIdx.x - plane * ntiles);
    const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
    const int c = (int)(plane % p.C);
    const int qy0 = ty * p.WY, qx0 = tx * p.WX;
    const int qy1 = imin(qy0 + p.WY, AY.n_in), qx1 = imin(qx0 + p.WX, AX.n_in);
    const int TT = AY.T * AX.T, Ppad = p.Ppad;
    const int gplane = p.NWYc * p.NWXc;
    float* sG = sW + TT * Ppad;
    float* sV = sG + Ppad * gplane;

    int vylo, vyhi, vxlo, vxhi;
    bool fy, fx;
    f2_virtual_range(AY, qy0, qy1, &vylo, &vyhi, &fy);
    f2_virtual_range(AX, qx0, qx1, &vxlo, &vxhi, &fx);
    // windows reaching [vlo, vhi]: i s - L <= vhi and i s - L + T - 1 >= vlo
    const int wylo = -floordiv(-(vylo + AY.L - AY.T + 1), AY.s), wyhi = floordiv(vyhi + AY.L, AY.s);
    const int wxlo = -floordiv(-(vxlo + AX.L - AX.T + 1), AX.s), wxhi = floordiv(vxhi + AX.L, AX.s);
    const int nwx = wxhi - wxlo + 1;
    const int VY = vyhi - vylo + 1, VX = vxhi - vxlo + 1;

    f2_stage_weights(sW, p, c);
    // g tile, phase-major: sG[ph][iy - wylo][ix - wxlo]; zero outside the output
    // and on the padding phases [P, Ppad)
    const Tg* gp = reinterpret_cast<const Tg*>(p.g) + plane * (long long)AY.n_out * AX.n_out;
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        const int grow = (wyhi - wylo + 1) * AY.r, gcol = nwx * AX.r;
        const int oy0 = wylo * AY.r, ox0 = wxlo * AX.r;
        const int q32 = 32 / AX.r, u32 = 32 - q32 * AX.r;
        const int q0 = lane / AX.r, u0 = lane - q0 * AX.r;
        for (int rr = warp; rr < grow; rr += nwarp) {
            const int oy = oy0 + rr;
            const int iyl = rr / AY.r, jy = rr - iyl * AY.r;
            const bool row_ok = oy >= 0 && oy < AY.n_out;
            const Tg* grow_p = gp + (long long)oy * AX.n_out;
            float* dst = sG + jy * AX.r * gplane + iyl * p.NWXc;
            int ixl = q0, jx = u0;
            for (int cc = lane; cc < gcol; cc += 32) {
                const int ox = ox0 + cc;
                float v = 0.f;
                if (row_ok && ox >= 0 && ox < AX.n_out) v = load_f(grow_p + ox);
                dst[jx * gplane + ixl] = v;
                ixl += q32;
                jx += u32;
                if (jx >= AX.r) {
                    jx -= AX.r;
                    ++ixl;
                }
            }
        }
        for (int k = p.P * gplane + threadIdx.x; k < Ppad * gplane; k += blockDim.x) sG[k] = 0.f;
    }
    __syncthreads();

    // virtual cells: sV[ey - vylo][ex - vxlo] = sum over (window, phase, tap)
    // reaching (ey, ex).  Tap my reaches ey from window (ey + L - my) / s when
    // my = (ey + L) mod s (mod s); one warp per row, lanes across the row.
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        const int dx0 = vxlo + lane + AX.L;
        const int ux0 = pmod(dx0, AX.s), ix0l = (dx0 - ux0) / AX.s - wxlo;
        const int q32 = 32 / AX.s, u32 = 32 - q32 * AX.s;
        for (int vyl = warp; vyl < VY; vyl += nwarp) {
            const int dy = vylo + vyl + AY.L;
            const int uy = pmod(dy, AY.s), iy0l = (dy - uy) / AY.s - wylo;
            int ux = ux0, ixs = ix0l;
            for (int vxl = lane; vxl < VX; vxl += 32) {
                float acc0 = 0.f, acc1 = 0.f;
                int iyl = iy0l;
                for (int my = uy; my < AY.T; my += AY.s, --iyl) {
                    int ixl = ixs;
                    const float* wrow = sW + my * AX.T * Ppad;
                    const float* grow_s = sG + iyl * p.NWXc;
                    for (int mx = ux; mx < AX.T; mx += AX.s, --ixl) {
                        const float4* wv = reinterpret_cast<const float4*>(wrow + mx * Ppad);
                        const float* gv = grow_s + ixl;
                        for (int ph = 0; ph < Ppad; ph += 4) {
                            const float4 w = *wv++;
                            acc0 = fmaf(w.x, gv[0], acc0);
                            acc1 = fmaf(w.y, gv[gplane], acc1);
                            acc0 = fmaf(w.z, gv[2 * gplane], acc0);
                            acc1 = fmaf(w.w, gv[3 * gplane], acc1);
                            gv += 4 * gplane;
                        }
                    }
                }
                sV[vyl * p.VXc + vxl] = acc0 + acc1;
                // next cell of this lane: 32 columns on
                ixs += q32;
                ux += u32;
                if (ux >= AX.s) {
                    ux -= AX.s;
                    ++ixs;
                }
            }
        }
    }
    __syncthreads();

    // pad adjoint: each real cell adds the virtual cells that fold onto it
    Tdx* dp = reinterpret_cast<Tdx*>(p.dx) + plane * (long long)AY.n_in * AX.n_in;
    const int QXr = qx1 - qx0, QYr = qy1 - qy0;
    for (int k = threadIdx.x; k < QYr * QXr; k += blockDim.x) {
        const int qyl = k / QXr, qxl = k - qyl * QXr;
        const int qy = qy0 + qyl, qx = qx0 + qxl;
        float s;
        if (!fy && !fx) {
            s = sV[(qy - vylo) * p.VXc + (qx - vxlo)];
        } else {
            s = 0.f;
            const int ny = fy ? AY.next : 0, nx = fx ? AX.next : 0;
            for (int a = -1; a < ny; ++a) {
                int ey = qy;
                if (a >= 0) {
                    if (AY.ext_q[a] != qy) continue;
                    ey = AY.ext_e[a];
                }
                const float* row = sV + (ey - vylo) * p.VXc - vxlo;
                for (int b = -1; b < nx; ++b) {
                    int ex = qx;
                    if (b >= 0) {
                        if (AX.ext_q[b] != qx) continue;
                        ex = AX.ext_e[b];
                    }
                    s += row[ex];
                }
            }
        }
        store_f(dp + (long long)qy * AX.n_in + qx, s);
    }
}

// ---------------------------------------------------------- weight gradient

// dW[ph][t] = sum over windows of g[window][ph] * x~[window origin + tap t]: a
// (phases x windows) by (windows x taps) product.  Each thread owns a block of
// 4 phases x 4 taps and runs over every G-th window of each staged tile.
template <typename Tx, typename Tg>
__global__ void __launch_bounds__(256) fcfs_full2d_dw(const __grid_constant__ F2Params p) {
    extern __shared__ float4 f2_smem4[];
    const F2Axis& AY = p.ax[0];
    const F2Axis& AX = p.ax[1];
    const int pass = (int)(blockIdx.x % p.npass);
    const long long pc = blockIdx.x / p.npass;
    const long long plane = pc / p.nchunk;
    const int chunk = (int)(pc - plane * p.nchunk);
    const int ntiles = p.tiles_x * p.tiles_y;
    const int TT = AY.T * AX.T, TX = AX.T, Ppad = p.Ppad;
    const int rows = (p.WY - 1) * AY.s + AY.T, cols = (p.WX - 1) * AX.s + AX.T;
    const int KW = (cols + AX.s - 1) / AX.s, pitch = KW * AX.s;
    const int NTB = (TT + 3) >> 2, NPB = Ppad >> 2, nblk = NPB * NTB;
    float* sG = reinterpret_cast<float*>(f2_smem4);  // [WY*WX windows][Ppad], 16-byte aligned rows
    float* sIn = sG + p.WY * p.WX * Ppad;
    float* sRed = sIn + rows * pitch;

    int G, grp, blk;
    if (p.npass == 1) {
        G = p.ngroups;
        grp = threadIdx.x / nblk;
        blk = threadIdx.x - grp * nblk;
    } else {
        G = 1;
        grp = 0;
        blk = pass * 256 + threadIdx.x;
    }
    const bool active = grp < G && blk < nblk;
    const int pb = active ? blk / NTB : 0, tb = active ? blk - (blk / NTB) * NTB : 0;
    int xoff[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int t = tb * 4 + k;
        int o = 0;
        if (t < TT) {
            const int my = t / TX, mx = t - my * TX, q = mx / AX.s;
            o = my * pitch + (mx - q * AX.s) * KW + q;
        }
        xoff[k] = o;
    }
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;

    const Tx* xp = reinterpret_cast<const Tx*>(p.x) + plane * (long long)AY.n_in * AX.n_in;
    const Tg* gp = reinterpret_cast<const Tg*>(p.g) + plane * (long long)AY.n_out * AX.n_out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int q32 = 32 / AX.r, u32 = 32 - q32 * AX.r;
    const int q0 = lane / AX.r, u0 = lane - q0 * AX.r;
    for (int tile = chunk; tile < ntiles; tile += p.nchunk) {
        const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
        const int iy0 = ty * p.WY, ix0 = tx * p.WX;
        __syncthreads();  // the previous tile's reads are done
        f2_load_tile_split<Tx>(sIn, pitch, KW, AX.s, xp, AY.n_in, AX.n_in, iy0 * AY.s - AY.L, ix0 * AX.s - AX.L,
                               rows, cols, p.pad, p.padv);
        // g tile, window-major: sG[(iyl*WX + ixl)*Ppad + jy*r_x + jx]; zero outside the output
        const int oy0 = iy0 * AY.r, ox0 = ix0 * AX.r, gcol = p.WX * AX.r;
        for (int rr = warp; rr < p.WY * AY.r; rr += nwarp) {
            const int oy = oy0 + rr;
            const int iyl = rr / AY.r, jy = rr - iyl * AY.r;
            const bool row_ok = oy < AY.n_out;
            const Tg* grow_p = gp + (long long)oy * AX.n_out;
            float* dst = sG + iyl * p.WX * Ppad + jy * AX.r;
            int ixl = q0, jx = u0;
            for (int cc = lane; cc < gcol; cc += 32) {
                const int ox = ox0 + cc;
                dst[ixl * Ppad + jx] = (row_ok && ox < AX.n_out) ? load_f(grow_p + ox) : 0.f;
                ixl += q32;
                jx += u32;
                if (jx >= AX.r) {
                    jx -= AX.r;
                    ++ixl;
                }
            }
        }
        __syncthreads();
        if (!active) continue;
        const int nwy = imin(p.WY, AY.nw - iy0), nwx = imin(p.WX, AX.nw - ix0);
        int iyl = 0, ixl = grp;
        while (ixl >= nwx && iyl < nwy) {
            ixl -= nwx;
            ++iyl;
        }
        while (iyl < nwy) {
            const float* xw = sIn + iyl * AY.s * pitch + ixl;
            const float4 g4 = *reinterpret_cast<const float4*>(sG + (iyl * p.WX + ixl) * Ppad + pb * 4);
            const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
            float xv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) xv[k] = xw[xoff[k]];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(gv[i], xv[k], acc[i][k]);
            ixl += G;
            while (ixl >= nwx) {
                ixl -= nwx;
                ++iyl;
            }
        }
    }

    float* rec = p.ws + pc * (long long)p.E;
    if (p.npass == 1) {
        // fixed-order sum over the window groups: sRed[grp][ph][t] on the padded grid
        const int PT = NTB * 4;
        if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) sRed[(grp * Ppad + pb * 4 + i) * PT + tb * 4 + k] = acc[i][k];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
            const int ph = e / TT, t = e - ph * TT;
            float s = 0.f;
            for (int g = 0; g < G; ++g) s += sRed[(g * Ppad + ph) * PT + t];
            rec[e] = s;
        }
    } else if (active) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int ph = pb * 4 + i, t = tb * 4 + k;
                if (ph < p.P && t < TT) rec[ph * TT + t] = acc[i][k];
            }
    }
}

// dW[c][e] (or dW[e] summed over channels in channel order) = sum over the
// batch and the chunks of the records, accumulated in FP64.
__global__ void __launch_bounds__(256) fcfs_full2d_dw_reduce(const __grid_constant__ F2Params p) {
    const int E = p.E;
    const long long nout = p.per_channel ? (long long)p.C * E : E;
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    const int e = (int)(o % E);
    const int c0 = p.per_channel ? (int)(o / E) : 0, c1 = p.per_channel ? c0 + 1 : p.C;
    const long long nb = p.planes / p.C;
    double s = 0.0;
    for (int c = c0; c < c1; ++c)
        for (long long b = 0; b < nb; ++b) {
            const float* r = p.ws + ((b * p.C + c) * p.nchunk) * (long long)E + e;
            for (int k = 0; k < p.nchunk; ++k) s += (double)r[(long long)k * E];
        }
    p.dw[o] = (float)s;
}

// ------------------------------------------------------------------ host

int f2_axis(const fcfs_desc* d, int a, F2Axis* A) {
    const fcfs_axis& ax = d->axis[a];
    memset(A, 0, sizeof *A);
    const int K = ax.K ? ax.K : k_min(ax.method, ax.s);
    A->n_in = (int)d->in_shape[a];
    A->n_out = (int)d->out_shape[a];
    A->r = ax.r;
    A->s = ax.s;
    A->T = 2 * K + 1;
    A->L = K - ax.s / 2;
    A->nw = (A->n_out + A->r - 1) / A->r;
    if (A->nw == 0 || A->n_in == 0) return FCFS_OK;
    // extended indices the windows touch: [-L, (nw-1) s - L + T - 1]
    const long long ev_lo = -(long long)A->L, ev_hi = (long long)(A->nw - 1) * A->s - A->L + A->T - 1;
    for (long long e = ev_lo; e <= ev_hi; ++e) {
        if (e >= 0 && e < A->n_in) {
            e = A->n_in - 1;  // skip the real range
            continue;
        }
        const int q = ext_index((int)e, A->n_in, d->pad);
        if (q < 0) continue;
        if (A->next == kF2MaxExtra)
            return fail(FCFS_ERR_UNSUPPORTED, "axis %d: more than %d padded indices fold onto the input", a,
                        kF2MaxExtra);
        A->ext_e[A->next] = (int)e;
        A->ext_q[A->next] = q;
        ++A->next;
    }
    return FCFS_OK;
}

int f2_params(const fcfs_desc* d, F2Params* p) {
    memset(p, 0, sizeof *p);
    for (int a = 0; a < 2; ++a) {
        int rc = f2_axis(d, a, &p->ax[a]);
        if (rc) return rc;
    }
    p->planes = d->n * d->c;
    p->C = (int)d->c;
    p->per_channel = d->w2d_per_channel;
    p->P = p->ax[0].r * p->ax[1].r;
    p->E = p->P * p->ax[0].T * p->ax[1].T;
    if (p->E > kF2MaxEntries)
        return fail(FCFS_ERR_UNSUPPORTED, "r_y r_x T_y T_x = %d exceeds %d kernel entries", p->E, kF2MaxEntries);
    p->pad = d->pad;
    p->padv = d->pad_value;
    p->w = d->w2d;
    return FCFS_OK;
}

size_t f2_pitch(const F2Params& p, int* rows) {
    *rows = (p.WY - 1) * p.ax[0].s + p.ax[0].T;
    const int cols = (p.WX - 1) * p.ax[1].s + p.ax[1].T;
    return (size_t)((cols + p.ax[1].s - 1) / p.ax[1].s) * p.ax[1].s;
}

size_t f2_fwd_smem(const F2Params& p) {
    int rows;
    const size_t pitch = f2_pitch(p, &rows);
    return sizeof(float) * ((size_t)p.ax[0].T * p.ax[1].T * p.Ppad + (size_t)rows * pitch);
}

// Capacity of the virtual range of any tile of Q real cells along one axis,
// and of the window range that reaches it.
void f2_axis_caps(const F2Axis& A, int Q, int* Vc, int* NWc) {
    int vmax = std::min(Q, std::max(A.n_in, 1));
    std::map<int, std::pair<int, int>> span;  // tile -> virtual [lo, hi]
    for (int k = 0; k < A.next; ++k) {
        const int t = A.ext_q[k] / Q;
        auto it = span.find(t);
        if (it == span.end()) {
            const int q0 = t * Q, q1 = std::min(q0 + Q, A.n_in);
            it = span.emplace(t, std::make_pair(q0, q1 - 1)).first;
        }
        it->second.first = std::min(it->second.first, A.ext_e[k]);
        it->second.second = std::max(it->second.second, A.ext_e[k]);
    }
    for (auto& kv : span) vmax = std::max(vmax, kv.second.second - kv.second.first + 1);
    *Vc = vmax;
    *NWc = (vmax + A.T - 2) / A.s + 1;
}

size_t f2_dx_smem(const F2Params& p) {
    return sizeof(float) * ((size_t)p.ax[0].T * p.ax[1].T * p.Ppad + (size_t)p.Ppad * p.NWYc * p.NWXc +
                            (size_t)p.VYc * p.VXc);
}

// window-major g tile, split input tile, and the group-reduction area (at most
// 256 threads x 16 partial sums)
size_t f2_dw_smem(const F2Params& p) {
    int rows;
    const size_t pitch = f2_pitch(p, &rows);
    return sizeof(float) * ((size_t)p.WY * p.WX * p.Ppad + (size_t)rows * pitch + 256 * 16);
}

constexpr size_t kF2SmemCap = 200 * 1024;

template <typename K>
cudaError_t f2_launch(K kernel, const F2Params& p, long long blocks, size_t smem, cudaStream_t st) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<(unsigned)blocks, 256, smem, st>>>(p);
    return cudaGetLastError();
}

// Window tile of the forward / weight-gradient kernels: WX windows across
// (the forward's lanes take two windows each), rows shrunk until the staged
// tile fits.
int f2_window_tile(F2Params& p, bool for_dw) {
    p.WX = for_dw ? 32 : kF2FwdWX;
    p.WY = 8;
    for (;;) {
        const size_t smem = for_dw ? f2_dw_smem(p) : f2_fwd_smem(p);
        if (smem <= kF2SmemCap) break;
        if (p.WY > 1) {
            p.WY /= 2;
        } else if (for_dw && p.WX > 1) {
            p.WX /= 2;
        } else {
            return fail(FCFS_ERR_UNSUPPORTED, "non-separable kernel tile exceeds shared memory");
        }
    }
    p.tiles_x = (p.ax[1].nw + p.WX - 1) / p.WX;
    p.tiles_y = (p.ax[0].nw + p.WY - 1) / p.WY;
    return FCFS_OK;
}

}  // namespace

int full2d_forward(const fcfs_desc* d, const void* x, void* y, cudaStream_t st) {
    F2Params p;
    int rc = f2_params(d, &p);
    if (rc) return rc;
    const int nph = p.P == 1 ? 1 : 4;
    p.Ppad = (p.P + nph - 1) / nph * nph;
    rc = f2_window_tile(p, false);
    if (rc) return rc;
    const long long blocks = (long long)p.tiles_x * p.tiles_y * p.planes;
    if (blocks > INT_MAX) return fail(FCFS_ERR_UNSUPPORTED, "grid too large");
    p.x = x;
    p.y = y;
    const size_t smem = f2_fwd_smem(p);
    cudaError_t e = cudaErrorInvalidValue;
    // compile-time tap counts for the common square windows (T x T taps, x stride s)
    const int cts = p.ax[0].T == p.ax[1].T ? p.ax[1].T * 16 + p.ax[1].s : 0;
#define F2_FWD(NPH, TI, TO)                                                                          \
    do {                                                                                             \
        if (cts == 5 * 16 + 4) e = f2_launch(fcfs_full2d_fwd<NPH, TI, TO, 5, 4>, p, blocks, smem, st); \
        else if (cts == 5 * 16 + 1) e = f2_launch(fcfs_full2d_fwd<NPH, TI, TO, 5, 1>, p, blocks, smem, st); \
        else if (cts == 3 * 16 + 1) e = f2_launch(fcfs_full2d_fwd<NPH, TI, TO, 3, 1>, p, blocks, smem, st); \
        else e = f2_launch(fcfs_full2d_fwd<NPH, TI, TO>, p, blocks, smem, st);                         \
    } while (0)
#define F2_FWD_OUT(NPH, TI)                      \
    if (d->dtype_out == FCFS_F32) F2_FWD(NPH, TI, float); \
    else F2_FWD(NPH, TI, __nv_bfloat16)
#define F2_FWD_IN(NPH)                                              \
    if (d->dtype_in == FCFS_F32) { F2_FWD_OUT(NPH, float); }         \
    else if (d->dtype_in == FCFS_BF16) { F2_FWD_OUT(NPH, __nv_bfloat16); } \
    else { F2_FWD_OUT(NPH, uint8_t); }
    if (nph == 1) {
        F2_FWD_IN(1)
    } else {
        F2_FWD_IN(4)
    }
#undef F2_FWD_IN
#undef F2_FWD_OUT
#undef F2_FWD
    return e == cudaSuccess ? FCFS_OK : cuda_fail(e, "non-separable forward launch");
}

static int f2_dw_plan(const fcfs_desc* d, F2Params* p) {
    int rc = f2_params(d, p);
    if (rc) return rc;
    p->Ppad = (p->P + 3) / 4 * 4;
    rc = f2_window_tile(*p, true);
    if (rc) return rc;
    const int ntiles = p->tiles_x * p->tiles_y;
    const int TT = p->ax[0].T * p->ax[1].T;
    const int nblk = (p->Ppad / 4) * ((TT + 3) / 4);
    p->ngroups = nblk <= 256 ? 256 / nblk : 1;
    p->npass = nblk <= 256 ? 1 : (nblk + 255) / 256;
    // enough CTAs for four per SM, records capped near 8 MiB where the plane count allows
    const long long want = (608 + p->planes - 1) / std::max(1LL, p->planes);
    const long long cap = std::max(1LL, (8LL << 20) / (4LL * p->E * std::max(1LL, p->planes)));
    p->nchunk = (int)std::max(1LL, std::min({want, cap, (long long)ntiles}));
    if ((long long)p->nchunk * p->planes * p->npass > INT_MAX) return fail(FCFS_ERR_UNSUPPORTED, "grid too large");
    return FCFS_OK;
}

size_t full2d_workspace(const fcfs_desc* d) {
    F2Params p;
    if (f2_dw_plan(d, &p) != FCFS_OK) return 0;
    return sizeof(float) * (size_t)p.planes * p.nchunk * p.E;
}

int full2d_backward(const fcfs_desc* d, const void* x, const void* gy, void* gx, float* gw, void* ws,
                    size_t ws_bytes, cudaStream_t st) {
    if (gx) {
        F2Params p;
        int rc = f2_params(d, &p);
        if (rc) return rc;
        p.Ppad = (p.P + 3) / 4 * 4;
        int Q = 32;
        for (;;) {
            p.WX = p.WY = Q;
            f2_axis_caps(p.ax[0], Q, &p.VYc, &p.NWYc);
            f2_axis_caps(p.ax[1], Q, &p.VXc, &p.NWXc);
            if (f2_dx_smem(p) <= kF2SmemCap) break;
            if (Q == 1) return fail(FCFS_ERR_UNSUPPORTED, "non-separable input-gradient tile exceeds shared memory");
            Q /= 2;
        }
        p.tiles_x = (p.ax[1].n_in + Q - 1) / Q;
        p.tiles_y = (p.ax[0].n_in + Q - 1) / Q;
        const long long blocks = (long long)p.tiles_x * p.tiles_y * p.planes;
        if (blocks > INT_MAX) return fail(FCFS_ERR_UNSUPPORTED, "grid too large");
        p.g = gy;
        p.dx = gx;
        const size_t smem = f2_dx_smem(p);
        cudaError_t e;
        if (d->dtype_out == FCFS_F32) {
            e = d->dtype_in == FCFS_F32 ? f2_launch(fcfs_full2d_dx<float, float>, p, blocks, smem, st)
                                        : f2_launch(fcfs_full2d_dx<float, __nv_bfloat16>, p, blocks, smem, st);
        } else {
            e = d->dtype_in == FCFS_F32 ? f2_launch(fcfs_full2d_dx<__nv_bfloat16, float>, p, blocks, smem, st)
                                        : f2_launch(fcfs_full2d_dx<__nv_bfloat16, __nv_bfloat16>, p, blocks, smem, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "non-separable input-gradient launch");
    }
    if (gw) {
        F2Params p;
        int rc = f2_dw_plan(d, &p);
        if (rc) return rc;
        const size_t need = sizeof(float) * (size_t)p.planes * p.nchunk * p.E;
        if (!ws || ws_bytes < need) return fail(FCFS_ERR_NOMEM, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
        p.x = x;
        p.g = gy;
        p.ws = (float*)ws;
        p.dw = gw;
        const long long blocks = (long long)p.nchunk * p.planes * p.npass;
        const size_t smem = f2_dw_smem(p);
        cudaError_t e;
        if (d->dtype_in == FCFS_F32) {
            e = d->dtype_out == FCFS_F32 ? f2_launch(fcfs_full2d_dw<float, float>, p, blocks, smem, st)
                                         : f2_launch(fcfs_full2d_dw<float, __nv_bfloat16>, p, blocks, smem, st);
        } else {
            e = d->dtype_out == FCFS_F32 ? f2_launch(fcfs_full2d_dw<__nv_bfloat16, float>, p, blocks, smem, st)
                                         : f2_launch(fcfs_full2d_dw<__nv_bfloat16, __nv_bfloat16>, p, blocks, smem, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "non-separable weight-gradient launch");
        const long long nout = p.per_channel ? (long long)p.C * p.E : p.E;
        fcfs_full2d_dw_reduce<<<(unsigned)((nout + 255) / 256), 256, 0, st>>>(p);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "non-separable weight-gradient reduce launch");
    }
    return FCFS_OK;
}

}  // namespace fcfs
