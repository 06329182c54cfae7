// Gather-staged forward tile shared by the 2D forward kernel and the
// serving kernel: stage the padded input tile through the index map, run the
// x taps into a shared-memory FP32 intermediate, run the y taps and store at
// the pixel-shuffled output positions (Sec. 3.1; Sec. 4 per axis).
#pragma once

#include <type_traits>

#include "fcfs_internal.cuh"

namespace fcfs {

// Per-CTA tap weights for one axis, zero-padded from nt_src to NT taps.
template <int NT>
__device__ __forceinline__ void stage_weights(float* dst, const AxisP& A, int c) {
    const int n = A.r * NT;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int j = k / NT, t = k - j * NT;
        float v = 0.f;
        if (t < A.nt_src) {
            v = A.learn ? A.w[(long long)c * A.w_cstride + j * A.nt_src + t] : A.wf[j * A.nt_src + t];
        }
        dst[k] = v;
    }
}

// Input tile [rows][cols] of one depth plane, extended coordinates row0/col0,
// with the padding rule as an index map.  One warp per row, lanes across
// columns (coalesced); interior rows issue eight independent loads per lane
// before storing them, so each warp keeps several loads in flight.
// src_plane == nullptr means the whole plane is the constant pad value
// (constant padding in depth).
template <typename Tin>
__device__ __forceinline__ void load_tile(float* sIn, int pitch, const Tin* src_plane, int H, int W, int row0,
                                          int col0, int rows, int cols, int pad, float padv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const bool inside_x = col0 >= 0 && col0 + cols <= W;
    for (int ry = warp; ry < rows; ry += nwarp) {
        const int sy = ext_index(row0 + ry, H, pad);
        float* dst = sIn + ry * pitch;
        if (src_plane == nullptr || sy < 0) {
            for (int cx = lane; cx < cols; cx += 32) dst[cx] = padv;
            continue;
        }
        const Tin* src = src_plane + (long long)sy * W;
        if constexpr (std::is_same<Tin, uint8_t>::value) {
            if (inside_x) {
                // bytes read as aligned 4-byte words (4x fewer load requests than byte loads); every
                // word read holds at least one byte of the row segment, so it stays in a mapped page
                const uintptr_t a = reinterpret_cast<uintptr_t>(src + col0);
                const uint32_t* wp = reinterpret_cast<const uint32_t*>(a & ~(uintptr_t)3);
                const int mis = (int)(a & 3);
                const int nw = (mis + cols + 3) >> 2;
                constexpr int U = 4;
                for (int k0 = lane; k0 < nw; k0 += 32 * U) {
                    uint32_t w[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) w[u] = k0 + 32 * u < nw ? __ldg(wp + k0 + 32 * u) : 0u;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e0 = 4 * (k0 + 32 * u) - mis;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int e = e0 + b;
                            if (e >= 0 && e < cols) dst[e] = (float)((w[u] >> (8 * b)) & 0xffu);
                        }
                    }
                }
                continue;
            }
        }
        if (inside_x) {
            const Tin* s0 = src + col0;
            constexpr int U = 8;
            for (int cb = lane; cb < cols; cb += 32 * U) {
                float v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = cb + 32 * u < cols ? load_f(s0 + cb + 32 * u) : 0.f;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (cb + 32 * u < cols) dst[cb + 32 * u] = v[u];
            }
        } else {
            for (int cx = lane; cx < cols; cx += 32) {
                const int sx = ext_index(col0 + cx, W, pad);
                dst[cx] = sx < 0 ? padv : load_f(src + sx);
            }
        }
    }
}

// x taps: sH[ry][ox] = sum_t wx[jx][t] * sIn[ry][ixl*s + off[jx] + t]
template <int NT>
__device__ __forceinline__ void pass_x(float* sH, const float* sIn, const float* sWx, const AxisP& AX,
                                       int OX, int pitch, int rows, int nwx, int G) {
    const int ox = threadIdx.x % OX, g = threadIdx.x / OX;
    const int jx = ox % AX.r, ixl = ox / AX.r;
    if (ixl >= nwx || g >= G) return;
    float w[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) w[t] = sWx[jx * NT + t];
    const float* base = sIn + ixl * AX.s + AX.off[jx];
    for (int ry = g; ry < rows; ry += G) {
        const float* row = base + ry * pitch;
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < NT; ++t) acc = fmaf(w[t], row[t], acc);
        sH[ry * OX + ox] = acc;
    }
}

// One tile of the gather-staged 2D forward.  Threads beyond OX * P.G idle in
// the passes (so a launch may use a larger block than the tile needs).
template <int NT, typename Tin, typename Tout>
__device__ __forceinline__ void fwd2d_tile(const FwdParams& P, long long tile, float* smem) {
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    long long t = tile;
    const int tx = (int)(t % P.tiles_x);
    t /= P.tiles_x;
    const int ty = (int)(t % P.tiles_y);
    const long long plane = t / P.tiles_y;
    const int c = (int)(plane % P.C);

    float* sWx = smem;
    float* sWy = sWx + AX.r * NT;
    float* sIn = sWy + AY.r * NT;
    float* sH = sIn + P.IR * P.ICp;

    const int ix0 = tx * P.WX, iy0 = ty * P.WY;
    const int nwx = min(P.WX, AX.n_win - ix0), nwy = min(P.WY, AY.n_win - iy0);
    const int cols = (nwx - 1) * AX.s + AX.span, rows = (nwy - 1) * AY.s + AY.span;
    const int col0 = ix0 * AX.s + AX.lo, row0 = iy0 * AY.s + AY.lo;

    stage_weights<NT>(sWx, AX, c);
    stage_weights<NT>(sWy, AY, c);
    const Tin* xp = static_cast<const Tin*>(P.x) + plane * (long long)AY.n_in * AX.n_in;
    load_tile<Tin>(sIn, P.ICp, xp, AY.n_in, AX.n_in, row0, col0, rows, cols, P.pad, P.padv);
    __syncthreads();

    pass_x<NT>(sH, sIn, sWx, AX, P.OX, P.ICp, rows, nwx, P.G);
    __syncthreads();

    // y taps, written at the pixel-shuffled output position
    const int OX = P.OX;
    const int ox = threadIdx.x % OX, g = threadIdx.x / OX, G = P.G;
    const int gox = ix0 * AX.r + ox;
    if (g >= G || ox / AX.r >= nwx || gox >= AX.n_out) return;
    Tout* yp = static_cast<Tout*>(P.y) + plane * (long long)AY.n_out * AX.n_out + gox;
    for (int iyl = g; iyl < nwy; iyl += G) {
        const int oyb = (iy0 + iyl) * AY.r;
        const int jmax = min(AY.r, AY.n_out - oyb);
        for (int jy = 0; jy < jmax; ++jy) {
            const float* col = sH + (iyl * AY.s + AY.off[jy]) * OX + ox;
            const float* wy = sWy + jy * NT;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < NT; ++k) acc = fmaf(wy[k], col[k * OX], acc);
            store_f(yp + (long long)(oyb + jy) * AX.n_out, epi_on(P.epi) ? epi_apply(P.epi, c, acc) : acc);
        }
    }
}

}  // namespace fcfs
