// Forward FCFS kernels (Sec. 3.1 pseudocode, Sec. 4 for N-d):
//   K1 fcfs_fwd2d  - fused separable polyphase gather for 1D/2D
//   K3 fcfs_fwd3d  - the same with a depth-streaming ring of planes
//   K2 fcfs_nearest - nearest on every axis: an exact gather copy
//
// The r-channel hidden layer of Sec. 3.1 (shape r x N/s per axis) is never
// stored: a CTA stages an input tile (with the padding rule applied as an
// index map), runs the x taps into a shared-memory FP32 intermediate, runs the
// y taps from there, and writes each output at its pixel-shuffled position.
#include <type_traits>

#include "fcfs_fwd_tile.cuh"

namespace fcfs {

namespace {

template <int NT, typename Tin, typename Tout>
__global__ void __launch_bounds__(512) fcfs_fwd2d(const __grid_constant__ FwdParams P) {
    extern __shared__ float smem[];
    fwd2d_tile<NT, Tin, Tout>(P, blockIdx.x, smem);
}

// 3D: a CTA owns an (OY x OX) output tile and WD depth windows.  Each input
// depth plane of its range is staged, x- and y-interpolated once into a ring
// of span_d planes; each depth window then combines the ring with its taps.
template <int NT, typename Tin, typename Tout>
__global__ void __launch_bounds__(512) fcfs_fwd3d(const __grid_constant__ FwdParams P) {
    extern __shared__ float smem[];
    const AxisP& AD = P.ax[0];
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    long long t = blockIdx.x;
    const int tx = (int)(t % P.tiles_x);
    t /= P.tiles_x;
    const int ty = (int)(t % P.tiles_y);
    t /= P.tiles_y;
    const int td = (int)(t % P.tiles_d);
    const long long plane = t / P.tiles_d;
    const int c = (int)(plane % P.C);

    float* sWx = smem;
    float* sWy = sWx + AX.r * NT;
    float* sWd = sWy + AY.r * NT;
    float* sIn = sWd + AD.r * NT;
    float* sH = sIn + P.IR * P.ICp;
    float* ring = sH + P.IR * P.OX;
    const int OX = P.OX, OY = P.OY;
    const int ringsz = OY * OX;

    const int ix0 = tx * P.WX, iy0 = ty * P.WY, id0 = td * P.WD;
    const int nwx = min(P.WX, AX.n_win - ix0), nwy = min(P.WY, AY.n_win - iy0);
    const int nwd = min(P.WD, AD.n_win - id0);
    const int cols = (nwx - 1) * AX.s + AX.span, rows = (nwy - 1) * AY.s + AY.span;
    const int col0 = ix0 * AX.s + AX.lo, row0 = iy0 * AY.s + AY.lo;

    stage_weights<NT>(sWx, AX, c);
    stage_weights<NT>(sWy, AY, c);
    stage_weights<NT>(sWd, AD, c);

    const long long in_plane = (long long)AY.n_in * AX.n_in;
    const long long out_plane = (long long)AY.n_out * AX.n_out;
    const Tin* xvol = static_cast<const Tin*>(P.x) + plane * (long long)AD.n_in * in_plane;
    Tout* yvol = static_cast<Tout*>(P.y) + plane * (long long)AD.n_out * out_plane;

    const int ox = threadIdx.x % OX, g = threadIdx.x / OX, G = blockDim.x / OX;
    const int jx_ok = (ox / AX.r < nwx) && (ix0 * AX.r + ox < AX.n_out);
    const int p_first = id0 * AD.s + AD.lo;
    int next = p_first;  // next extended depth plane to produce

    for (int idl = 0; idl < nwd; ++idl) {
        const int id = id0 + idl;
        const int need_lo = id * AD.s + AD.lo, need_hi = need_lo + AD.span;
        if (next < need_lo) next = need_lo;
        while (next < need_hi) {
            const int sd = ext_index(next, AD.n_in, P.pad);
            load_tile<Tin>(sIn, P.ICp, sd < 0 ? nullptr : xvol + sd * in_plane, AY.n_in, AX.n_in, row0, col0,
                           rows, cols, P.pad, P.padv);
            __syncthreads();
            pass_x<NT>(sH, sIn, sWx, AX, OX, P.ICp, rows, nwx, G);
            __syncthreads();
            float* slot = ring + ((next - p_first) % P.ring) * ringsz;
            if (ox / AX.r < nwx) {
                for (int iyl = g; iyl < nwy; iyl += G) {
                    for (int jy = 0; jy < AY.r; ++jy) {
                        const float* col = sH + (iyl * AY.s + AY.off[jy]) * OX + ox;
                        const float* wy = sWy + jy * NT;
                        float acc = 0.f;
#pragma unroll
                        for (int k = 0; k < NT; ++k) acc = fmaf(wy[k], col[k * OX], acc);
                        slot[(iyl * AY.r + jy) * OX + ox] = acc;
                    }
                }
            }
            __syncthreads();
            ++next;
        }
        // depth taps for the r_d output planes of window id
        const int odb = id * AD.r;
        const int jdmax = min(AD.r, AD.n_out - odb);
        if (jx_ok) {
            const int gox = ix0 * AX.r + ox;
            for (int jd = 0; jd < jdmax; ++jd) {
                const int pbase = need_lo + AD.off[jd] - p_first;
                const float* wd = sWd + jd * NT;
                Tout* yo = yvol + (long long)(odb + jd) * out_plane + gox;
                for (int oyl = g; oyl < nwy * AY.r; oyl += G) {
                    const int oy = iy0 * AY.r + oyl;
                    if (oy >= AY.n_out) break;
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < NT; ++k)
                        acc = fmaf(wd[k], ring[((pbase + k) % P.ring) * ringsz + oyl * OX + ox], acc);
                    store_f(yo + (long long)oy * AX.n_out, acc);
                }
            }
        }
        __syncthreads();
    }
}

// Nearest on every axis: y[o] = x~[src(o)] per axis (the paper's rule rounds
// o s / r half up, Sec. 5.2.1 examples; see nearest_src for the others), an
// exact copy.  One block covers OYT x OXT
// outputs of one (plane, output depth) slice; source indices come from small
// shared-memory maps.
// Source of nearest output o (non-negative integers only): the paper's
// position o s / r rounded half up, rounded down (floor alignment), or the
// pixel centre (o + 1/2) s / r rounded down (half-pixel alignment).
__device__ __forceinline__ int nearest_src(long long o, int r, int s, int align) {
    if (align == FCFS_ALIGN_FLOOR) return (int)(o * s / r);
    if (align == FCFS_ALIGN_HALF_PIXEL) return (int)((2 * o * s + s) / (2LL * r));
    return (int)((2 * o * s + r) / (2LL * r));
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) fcfs_nearest(const __grid_constant__ NearestParams P) {
    __shared__ int colmap[256];
    __shared__ int rowmap[64];
    long long t = blockIdx.x;
    const int tx = (int)(t % P.tiles_x);
    t /= P.tiles_x;
    const int ty = (int)(t % P.tiles_y);
    t /= P.tiles_y;
    const int od = (int)(t % P.n_out[0]);
    const long long plane = t / P.n_out[0];
    const int ox0 = tx * P.OXT, oy0 = ty * P.OYT;
    const int ncol = min(P.OXT, P.n_out[2] - ox0), nrow = min(P.OYT, P.n_out[1] - oy0);
    for (int k = threadIdx.x; k < ncol; k += blockDim.x)
        colmap[k] = ext_index(nearest_src(ox0 + k, P.r[2], P.s[2], P.align), P.n_in[2], P.pad);
    for (int k = threadIdx.x; k < nrow; k += blockDim.x)
        rowmap[k] = ext_index(nearest_src(oy0 + k, P.r[1], P.s[1], P.align), P.n_in[1], P.pad);
    __syncthreads();
    const int sd = ext_index(nearest_src(od, P.r[0], P.s[0], P.align), P.n_in[0], P.pad);
    const long long in_plane = (long long)P.n_in[1] * P.n_in[2];
    const Tin* xp = static_cast<const Tin*>(P.x) + (plane * P.n_in[0] + (sd < 0 ? 0 : sd)) * in_plane;
    Tout* yp = static_cast<Tout*>(P.y) + ((plane * P.n_out[0] + od) * (long long)P.n_out[1] + oy0) * P.n_out[2] + ox0;
    const int lane = threadIdx.x % P.OXT, g = threadIdx.x / P.OXT, G = blockDim.x / P.OXT;
    if (lane >= ncol) return;
    const int sx = colmap[lane];
    for (int k = g; k < nrow; k += G) {
        const int sy = rowmap[k];
        float v;
        if (sd < 0 || sy < 0 || sx < 0) v = P.padv;
        else v = load_f(xp + (long long)sy * P.n_in[2] + sx);
        store_f(yp + (long long)k * P.n_out[2] + lane, v);
    }
}

template <typename F>
cudaError_t dispatch_types(int din, int dout, F&& f) {
    if (din == FCFS_F32 && dout == FCFS_F32) return f((const float*)nullptr, (float*)nullptr);
    if (din == FCFS_BF16 && dout == FCFS_BF16) return f((const __nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr);
    if (din == FCFS_F32 && dout == FCFS_BF16) return f((const float*)nullptr, (__nv_bfloat16*)nullptr);
    if (din == FCFS_BF16 && dout == FCFS_F32) return f((const __nv_bfloat16*)nullptr, (float*)nullptr);
    if (din == FCFS_U8 && dout == FCFS_F32) return f((const uint8_t*)nullptr, (float*)nullptr);
    if (din == FCFS_U8 && dout == FCFS_BF16) return f((const uint8_t*)nullptr, (__nv_bfloat16*)nullptr);
    return cudaErrorInvalidValue;
}

template <int NT, typename Tin, typename Tout>
cudaError_t run2d(const FwdParams& P, size_t smem, cudaStream_t st) {
    auto k = fcfs_fwd2d<NT, Tin, Tout>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)P.tiles_x * P.tiles_y * P.planes;
    k<<<(unsigned)blocks, P.OX * P.G, smem, st>>>(P);
    return cudaGetLastError();
}

template <int NT, typename Tin, typename Tout>
cudaError_t run3d(const FwdParams& P, size_t smem, cudaStream_t st) {
    auto k = fcfs_fwd3d<NT, Tin, Tout>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)P.tiles_x * P.tiles_y * P.tiles_d * P.planes;
    k<<<(unsigned)blocks, P.OX * P.G, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

size_t forward_smem_bytes(const FwdParams& P, bool is3d) {
    const int nt = P.ax[2].nt;
    size_t f = (size_t)(P.ax[2].r + P.ax[1].r + (is3d ? P.ax[0].r : 0)) * nt;
    f += (size_t)P.IR * P.ICp + (size_t)P.IR * P.OX;
    if (is3d) f += (size_t)P.ring * P.OY * P.OX;
    return f * sizeof(float);
}

#define FCFS_NT_CASES(X) X(1) X(2) X(3) X(4) X(5) X(7) X(9)

cudaError_t launch_forward_2d(const FwdParams& P, int nt, int din, int dout, cudaStream_t st) {
    const size_t smem = forward_smem_bytes(P, false);
    return dispatch_types(din, dout, [&](auto tin, auto tout) -> cudaError_t {
        using Tin = std::remove_const_t<std::remove_pointer_t<decltype(tin)>>;
        using Tout = std::remove_pointer_t<decltype(tout)>;
        switch (nt) {
#define CASE(N) \
    case N: return run2d<N, Tin, Tout>(P, smem, st);
            FCFS_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    });
}

cudaError_t launch_forward_3d(const FwdParams& P, int nt, int din, int dout, cudaStream_t st) {
    const size_t smem = forward_smem_bytes(P, true);
    return dispatch_types(din, dout, [&](auto tin, auto tout) -> cudaError_t {
        using Tin = std::remove_const_t<std::remove_pointer_t<decltype(tin)>>;
        using Tout = std::remove_pointer_t<decltype(tout)>;
        switch (nt) {
#define CASE(N) \
    case N: return run3d<N, Tin, Tout>(P, smem, st);
            FCFS_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    });
}

cudaError_t launch_nearest(const NearestParams& P, int din, int dout, cudaStream_t st) {
    return dispatch_types(din, dout, [&](auto tin, auto tout) -> cudaError_t {
        using Tin = std::remove_const_t<std::remove_pointer_t<decltype(tin)>>;
        using Tout = std::remove_pointer_t<decltype(tout)>;
        const long long blocks = (long long)P.tiles_x * P.tiles_y * P.n_out[0] * P.planes;
        fcfs_nearest<Tin, Tout><<<(unsigned)blocks, 256, 0, st>>>(P);
        return cudaGetLastError();
    });
}

}  // namespace fcfs
