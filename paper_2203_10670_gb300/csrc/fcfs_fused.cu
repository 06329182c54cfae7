// FCFS fused with the pointwise layer that follows it in a fully
// convolutional network (Sec. 1: the resize is one layer of an FCN; Sec. 4 for
// the 2D layer):
//   y[n,o,p] = act(sum_c M[o][c] FCFS(x)[n,c,p] + b[o])
//   K10 fcfs_fused2d - a CTA owns one output tile of one image and a block of
//       OB output channels.  In passes of up to eight input channels it stages
//       the padded input tiles, runs the x and y taps of the gather-staged
//       forward into shared-memory FP32 tiles z_c, and adds M[o][c] z_c into
//       per-thread accumulators (PIX pixels x OB output channels, the mix
//       coefficients read as float4 shared-memory broadcasts); four barriers
//       per pass.  Bias, activation and the store follow the last pass: the C
//       intermediate planes never reach HBM.
// Without a mix the bias and activation are applied by the store of the
// planned 2D forward kernels (bulk-copy, register-blocked or gather-staged);
// only nearest on both axes through the gather kernel comes here, one channel
// per block.
#include <algorithm>
#include <climits>
#include <cmath>

#include "fcfs_fwd_tile.cuh"
#include "fcfs_host.h"

namespace fcfs {

namespace {

constexpr int kFusedThreads = 256;
constexpr int kFusedPix = 2;  // output pixels per thread (tiles of at most 512 pixels)

struct FusedParams {
    FwdParams P;       // forward geometry of the separable layer, tile of WX x WY windows
    int c_out;         // output channels
    int ob;            // output channels per CTA (<= the kernel's OB)
    int oblocks;       // CTAs per (tile, image) along the output channels
    const float* mix;  // [c_out][C], NULL = identity (output channel o is input channel o)
    const float* bias; // [c_out] or NULL
    int act;
    float alpha, lo, hi;
    int dtype_out;
    int kc;            // input channels staged per pass (one barrier triple per pass)
    void* y;
};

template <int NT, int OB, typename Tin>
__global__ void __launch_bounds__(kFusedThreads) fcfs_fused2d(const __grid_constant__ FusedParams F) {
    extern __shared__ float smem[];
    const FwdParams& P = F.P;
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    long long t = blockIdx.x;
    const int tx = (int)(t % P.tiles_x);
    t /= P.tiles_x;
    const int ty = (int)(t % P.tiles_y);
    t /= P.tiles_y;
    const int obk = (int)(t % F.oblocks);
    const long long n = t / F.oblocks;
    const int o0 = obk * F.ob, nob = min(F.ob, F.c_out - o0);
    const bool identity = F.mix == nullptr;
    const int c_begin = identity ? o0 : 0, c_end = identity ? o0 + 1 : P.C;
    const bool learn = AX.learn || AY.learn;
    const int KC = F.kc;  // input channels per pass

    // per channel of a pass: x and y weights (learnable: one set per channel), input tile,
    // x-interpolated rows, z tile; then the mix coefficients [c - c_begin][OB]
    const int OX = P.OX, OY = P.OY, pix = OX * OY;
    const int wxn = AX.r * NT, wyn = AY.r * NT;
    const int inn = P.IR * P.ICp, hn = P.IR * OX;
    const int nws = learn ? KC : 1;
    float* sWx = smem;
    float* sWy = sWx + nws * wxn;
    float* sIn = sWy + nws * wyn;
    float* sH = sIn + KC * inn;
    float* sZ = sH + KC * hn;
    // mix coefficients on a 16-byte boundary: read as float4
    float* sM = smem + (((sZ + KC * pix) - smem + 3) & ~3);

    const int ix0 = tx * P.WX, iy0 = ty * P.WY;
    const int nwx = min(P.WX, AX.n_win - ix0), nwy = min(P.WY, AY.n_win - iy0);
    const int cols = (nwx - 1) * AX.s + AX.span, rows = (nwy - 1) * AY.s + AY.span;
    const int col0 = ix0 * AX.s + AX.lo, row0 = iy0 * AY.s + AY.lo;

    for (int k = threadIdx.x; k < (c_end - c_begin) * OB; k += blockDim.x) {
        const int cl = k / OB, o = k - cl * OB;
        float m = 0.f;
        if (o < nob) m = identity ? 1.f : __ldg(F.mix + (long long)(o0 + o) * P.C + c_begin + cl);
        sM[k] = m;
    }
    if (!learn) {
        stage_weights<NT>(sWx, AX, 0);
        stage_weights<NT>(sWy, AY, 0);
    }

    float acc[kFusedPix][OB];
#pragma unroll
    for (int k = 0; k < kFusedPix; ++k)
#pragma unroll
        for (int o = 0; o < OB; ++o) acc[k][o] = 0.f;

    const int ox = threadIdx.x % OX, g = threadIdx.x / OX, G = P.G;
    const bool ycol = g < G && ox / AX.r < nwx;
    for (int cb = c_begin; cb < c_end; cb += KC) {
        const int kn = min(KC, c_end - cb);
        // the barrier that ended the previous pass's mix frees every buffer of this pass
        for (int kc = 0; kc < kn; ++kc) {
            if (learn) {
                stage_weights<NT>(sWx + kc * wxn, AX, cb + kc);
                stage_weights<NT>(sWy + kc * wyn, AY, cb + kc);
            }
            const long long plane = n * P.C + cb + kc;
            const Tin* xp = static_cast<const Tin*>(P.x) + plane * (long long)AY.n_in * AX.n_in;
            load_tile<Tin>(sIn + kc * inn, P.ICp, xp, AY.n_in, AX.n_in, row0, col0, rows, cols, P.pad, P.padv);
        }
        __syncthreads();
        for (int kc = 0; kc < kn; ++kc)
            pass_x<NT>(sH + kc * hn, sIn + kc * inn, sWx + (learn ? kc * wxn : 0), AX, OX, P.ICp, rows, nwx, G);
        __syncthreads();
        // y taps into the z tiles (every phase of every window of the tile)
        if (ycol) {
            for (int kc = 0; kc < kn; ++kc) {
                const float* h = sH + kc * hn;
                const float* wyb = sWy + (learn ? kc * wyn : 0);
                float* z = sZ + kc * pix;
                for (int iyl = g; iyl < nwy; iyl += G) {
                    for (int jy = 0; jy < AY.r; ++jy) {
                        const float* col = h + (iyl * AY.s + AY.off[jy]) * OX + ox;
                        const float* wy = wyb + jy * NT;
                        float a = 0.f;
#pragma unroll
                        for (int k = 0; k < NT; ++k) a = fmaf(wy[k], col[k * OX], a);
                        z[(iyl * AY.r + jy) * OX + ox] = a;
                    }
                }
            }
        }
        __syncthreads();
        // 1x1 mix: acc[p][o] += M[o][c] z_c[p]
        for (int kc = 0; kc < kn; ++kc) {
            const float4* m4 = reinterpret_cast<const float4*>(sM + (cb + kc - c_begin) * OB);
            const float* z = sZ + kc * pix;
            float zv[kFusedPix];
#pragma unroll
            for (int k = 0; k < kFusedPix; ++k) {
                const int p = threadIdx.x + k * kFusedThreads;
                zv[k] = p < pix ? z[p] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < OB / 4; ++q) {
                const float4 mv = m4[q];
#pragma unroll
                for (int k = 0; k < kFusedPix; ++k) {
                    acc[k][4 * q] = fmaf(mv.x, zv[k], acc[k][4 * q]);
                    acc[k][4 * q + 1] = fmaf(mv.y, zv[k], acc[k][4 * q + 1]);
                    acc[k][4 * q + 2] = fmaf(mv.z, zv[k], acc[k][4 * q + 2]);
                    acc[k][4 * q + 3] = fmaf(mv.w, zv[k], acc[k][4 * q + 3]);
                }
            }
        }
        __syncthreads();  // the next pass overwrites the z tiles
    }

    // bias, activation, store at y[n][o0 + o][oy][ox]
#pragma unroll
    for (int k = 0; k < kFusedPix; ++k) {
        const int p = threadIdx.x + k * kFusedThreads;
        if (p >= pix) continue;
        const int oyl = p / OX, oxl = p - oyl * OX;
        const int oy = iy0 * AY.r + oyl, oxg = ix0 * AX.r + oxl;
        if (oy >= AY.n_out || oxg >= AX.n_out) continue;
        const long long pos = (long long)oy * AX.n_out + oxg;
        const long long oplane = (long long)AY.n_out * AX.n_out;
#pragma unroll
        for (int o = 0; o < OB; ++o) {
            if (o >= nob) break;
            float v = acc[k][o];
            if (F.bias) v += __ldg(F.bias + o0 + o);
            v = apply_act(v, F.act, F.alpha, F.lo, F.hi);
            const long long at = (n * F.c_out + o0 + o) * oplane + pos;
            if (F.dtype_out == FCFS_F32) store_f(static_cast<float*>(F.y) + at, v);
            else store_f(static_cast<__nv_bfloat16*>(F.y) + at, v);
        }
    }
}

template <int NT, int OB>
cudaError_t launch_fused_nt(const FusedParams& F, int din, long long blocks, size_t smem, cudaStream_t st) {
    auto go = [&](auto kernel) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kernel<<<(unsigned)blocks, kFusedThreads, smem, st>>>(F);
        return cudaGetLastError();
    };
    if (din == FCFS_F32) return go(fcfs_fused2d<NT, OB, float>);
    if (din == FCFS_BF16) return go(fcfs_fused2d<NT, OB, __nv_bfloat16>);
    return go(fcfs_fused2d<NT, OB, uint8_t>);
}

template <int OB>
cudaError_t launch_fused_ob(const FusedParams& F, int ntk, int din, long long blocks, size_t smem, cudaStream_t st) {
    switch (ntk) {
        case 1: return launch_fused_nt<1, OB>(F, din, blocks, smem, st);
        case 2: return launch_fused_nt<2, OB>(F, din, blocks, smem, st);
        case 3: return launch_fused_nt<3, OB>(F, din, blocks, smem, st);
        case 4: return launch_fused_nt<4, OB>(F, din, blocks, smem, st);
        case 5: return launch_fused_nt<5, OB>(F, din, blocks, smem, st);
        case 7: return launch_fused_nt<7, OB>(F, din, blocks, smem, st);
        case 9: return launch_fused_nt<9, OB>(F, din, blocks, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace fcfs

using namespace fcfs;

extern "C" int fcfs_forward_fused(const fcfs_desc* d, const fcfs_epilogue* e, const void* x, void* y, void* stream) {
    NvtxRange nv("fcfs_forward_fused");
    clear_error();
    int rc = validate_desc(d, true);
    if (rc) return rc;
    if (!e) return fail(FCFS_ERR_ARG, "epilogue is NULL");
    if (d->w2d) return fail(FCFS_ERR_UNSUPPORTED, "the fused layer follows the separable kernels");
    if (d->ndim != 2) return fail(FCFS_ERR_UNSUPPORTED, "the fused layer takes 2D images");
    if (e->c_out < 1) return fail(FCFS_ERR_ARG, "c_out must be >= 1");
    if (d->c < 1) return fail(FCFS_ERR_ARG, "the fused layer needs at least one input channel");
    if (!e->mix && e->c_out != d->c) return fail(FCFS_ERR_ARG, "without a mix c_out must equal c");
    if (e->act < FCFS_ACT_NONE || e->act > FCFS_ACT_CLAMP) return fail(FCFS_ERR_ARG, "unknown activation %d", e->act);
    if (!std::isfinite(e->alpha) || !std::isfinite(e->lo) || !std::isfinite(e->hi))
        return fail(FCFS_ERR_ARG, "alpha, lo and hi must be finite");
    if (e->act == FCFS_ACT_CLAMP && !(e->lo <= e->hi)) return fail(FCFS_ERR_ARG, "clamp needs lo <= hi");
    if (((uintptr_t)e->mix) % 4 || ((uintptr_t)e->bias) % 4) return fail(FCFS_ERR_ARG, "mix or bias misaligned");
    if (d->axis[0].r * d->axis[1].r > 512) return fail(FCFS_ERR_UNSUPPORTED, "the fused layer takes r_y r_x <= 512");
    if (d->n == 0 || d->out_shape[0] == 0 || d->out_shape[1] == 0) return FCFS_OK;
    if (!x || !y) return fail(FCFS_ERR_ARG, "x and y must be device pointers");
    if (((uintptr_t)x) % dtype_size(d->dtype_in) || ((uintptr_t)y) % dtype_size(d->dtype_out))
        return fail(FCFS_ERR_ARG, "x or y not aligned to its element size");

    if (!e->mix && forward_has_epilogue_path(d, x)) {
        // bias and activation only: the planned forward applies them on its store
        Epi epi{e->bias, e->act, e->alpha, e->lo, e->hi};
        return forward_planned(d, x, y, &epi, (cudaStream_t)stream);
    }
    // a mix of up to 96 input channels: the tensor-core kernel
    rc = fused_forward_tc(d, e, x, y, (cudaStream_t)stream);
    if (rc != FCFS_ERR_UNSUPPORTED) return rc;
    clear_error();
    FusedParams F;
    memset(&F, 0, sizeof F);
    int ntk;
    rc = build_forward_params(d, x, nullptr, &F.P, &ntk);
    if (rc) return rc;
    // tiles of at most 512 output pixels: about 8 rows by 64 columns
    const int rx = F.P.ax[2].r, ry = F.P.ax[1].r;
    const int WY = std::max(1, 8 / ry), OY = WY * ry;
    const int WX = std::max(1, (512 / OY) / rx);
    apply_tiles(F.P, false, WX, WY, 1, std::max(1, kFusedThreads / (WX * rx)));
    if (F.P.OX > kFusedThreads || F.P.OX * F.P.OY > kFusedPix * kFusedThreads)
        return fail(FCFS_ERR_UNSUPPORTED, "fused tile too large");
    F.c_out = e->c_out;
    F.mix = e->mix;
    F.bias = e->bias;
    F.act = e->act;
    F.alpha = e->alpha;
    F.lo = e->lo;
    F.hi = e->hi;
    F.dtype_out = d->dtype_out;
    F.y = y;
    const int OB = (!e->mix || e->c_out <= 8) ? 8 : 32;
    F.ob = e->mix ? std::min(OB, e->c_out) : 1;
    F.oblocks = (e->c_out + F.ob - 1) / F.ob;
    const long long blocks = (long long)F.P.tiles_x * F.P.tiles_y * F.oblocks * d->n;
    if (blocks > INT_MAX) return fail(FCFS_ERR_UNSUPPORTED, "grid too large");
    const long long crange = e->mix ? d->c : 1;
    const bool learn = d->axis[0].w || d->axis[1].w;
    auto smem_for = [&](int kc) {
        const size_t per = (size_t)F.P.IR * F.P.ICp + (size_t)F.P.IR * F.P.OX + (size_t)F.P.OX * F.P.OY;
        return sizeof(float) * ((size_t)(learn ? kc : 1) * (rx + ry) * ntk + (size_t)kc * per + 3 +
                                (size_t)crange * OB);
    };
    // up to 8 input channels per pass while the footprint stays near 48 KB
    F.kc = (int)std::max(1LL, std::min<long long>(8, crange));
    while (F.kc > 1 && smem_for(F.kc) > 48 * 1024) --F.kc;
    const size_t smem = smem_for(F.kc);
    if (smem > 200 * 1024) return fail(FCFS_ERR_UNSUPPORTED, "fused tile needs %zu bytes of shared memory", smem);
    cudaError_t ce = OB == 8 ? launch_fused_ob<8>(F, ntk, d->dtype_in, blocks, smem, (cudaStream_t)stream)
                             : launch_fused_ob<32>(F, ntk, d->dtype_in, blocks, smem, (cudaStream_t)stream);
    return ce == cudaSuccess ? FCFS_OK : cuda_fail(ce, "fused forward launch");
}
