// K10 on the tensor cores: FCFS fused with a 1x1 channel mix,
//   y[n,o,p] = act(sum_c M[o][c] FCFS(x)[n,c,p] + b[o])       (Sec. 1, Sec. 4)
// The mix is a (output channels x input channels) by (input channels x
// pixels) product per tile: tcgen05.mma (kind::tf32, M = 128 output channels,
// N = 256 pixels, K = 8 input channels per instruction) accumulates it in
// tensor memory while the CUDA cores produce the next eight FCFS planes.
// FP32 accuracy from TF32 units: every operand x is split into its TF32 head
// h (x with the 13 low mantissa bits cleared) and the remainder l = x - h,
// which FP32 holds exactly; |l| < 2^-10 |x| and l has up to 13 significant
// bits, of which the tensor cores read the top 11 (TF32), so they see l to
// within 2^-10 |l| < 2^-20 |x|.  D += Ah Bh + Ah Bl + Al Bh: the two
// remainder terms are each within 2^-20 |A B| of their exact values and the
// dropped Al Bl term is below 2^-20 |A B|, so every product is accurate to
// about 3 x 2^-20 of its magnitude, inside the FP32 bar of the layer.
//
// Per CTA: one output tile (at most 256 pixels) of one image, 128 output
// channels.  Shared memory holds both splits of the CTA's mix rows (operand
// A, K-major) and two buffers of both splits of eight z planes (operand B,
// K-major: pixel rows, channel columns).  Operand layout: 8-row x 16-byte core
// matrices, element (row, k) at float (row/8)*(KCH*32) + (k/4)*32 +
// (row%8)*4 + k%4 for KCH 4-channel chunks per row group, i.e. the leading
// (K) core-matrix offset 128 bytes and the stride (row-group) offset KCH*128
// bytes.  One thread issues the MMAs and commits them to an mbarrier per B
// buffer; the accumulator is read back with tcgen05.ld for bias, activation
// and the store.  Every mbarrier wait is bounded; the tensor memory is freed
// on every path.
#include <algorithm>
#include <climits>
#include <cmath>

#include "fcfs_fwd_tile.cuh"
#include "fcfs_host.h"
#include "fcfs_tma.cuh"

namespace fcfs {

namespace {

constexpr int kTcThreads = 512;
constexpr int kTcM = 128;  // output channels per CTA (accumulator rows = TMEM lanes)
constexpr int kTcN = 256;  // pixels per CTA (accumulator columns)
constexpr int kTcK = 8;    // input channels per MMA
constexpr int kTcPre = 4;  // prefetched input samples per thread

static __device__ int g_status_fused_tc = 0;

struct TcParams {
    FwdParams P;  // forward geometry (tile of WX x WY windows, OX * OY <= 256 pixels)
    int c_out, oblocks;
    int C8;       // input channels rounded up to 8
    const float* mix;
    const float* bias;
    int act;
    float alpha, lo, hi;
    int dtype_out;
    void* y;
    uint32_t idesc;
    int b_off, w_off, in_off, h_off, bar_off;  // byte offsets in shared memory (A at 0)
};

// float index of element (row, k) in a K-major operand with kch 4-channel chunks per row group
__device__ __forceinline__ int op_index(int row, int k, int kch) {
    return (row >> 3) * (kch * 32) + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

// shared-memory matrix descriptor: no swizzle, byte offsets in 16-byte units
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 consecutive columns of the accumulator (the warp's lane quarter)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NT, typename Tin>
__global__ void __launch_bounds__(kTcThreads) fcfs_fused2d_tc(const __grid_constant__ TcParams F) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const FwdParams& P = F.P;
    const AxisP& AY = P.ax[1];
    const AxisP& AX = P.ax[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long t = blockIdx.x;
    const int tx = (int)(t % P.tiles_x);
    t /= P.tiles_x;
    const int ty = (int)(t % P.tiles_y);
    t /= P.tiles_y;
    const int obk = (int)(t % F.oblocks);
    const long long n = t / F.oblocks;
    const int o0 = obk * kTcM, nob = min(kTcM, F.c_out - o0);
    const int C = P.C, C8 = F.C8, KCHA = C8 / 4;
    const bool learn = AX.learn || AY.learn;

    float* sAh = reinterpret_cast<float*>(smem_raw);
    float* sAl = sAh + kTcM * C8;
    float* sB = reinterpret_cast<float*>(smem_raw + F.b_off);  // [buffer][hi, lo][kTcN * kTcK]
    float* sWx = reinterpret_cast<float*>(smem_raw + F.w_off);
    const int wxn = AX.r * NT, wyn = AY.r * NT, nws = learn ? kTcK : 1;
    float* sWy = sWx + nws * wxn;
    float* sIn = reinterpret_cast<float*>(smem_raw + F.in_off);
    float* sH = reinterpret_cast<float*>(smem_raw + F.h_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + F.bar_off);
    const int inn = P.IR * P.ICp, hn = P.IR * P.OX;

    // operand A: both splits of mix rows o0 .. o0+127 (zero beyond c_out and C)
    for (int e = threadIdx.x; e < kTcM * C8; e += blockDim.x) {
        const int o = e / C8, c = e - o * C8;  // once per element of a small per-CTA operand
        float v = 0.f;
        if (o < nob && c < C) v = __ldg(F.mix + (long long)(o0 + o) * C + c);
        float h, l;
        split_tf32(v, h, l);
        const int at = op_index(o, c, KCHA);
        sAh[at] = h;
        sAl[at] = l;
    }
    for (int e = threadIdx.x; e < 4 * kTcN * kTcK; e += blockDim.x) sB[e] = 0.f;
    if (!learn) {
        stage_weights<NT>(sWx, AX, 0);
        stage_weights<NT>(sWy, AY, 0);
    }
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();  // the operand writes above, for the tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    const int OX = P.OX, OY = P.OY, pix = OX * OY;
    const int ix0 = tx * P.WX, iy0 = ty * P.WY;
    const int nwx = min(P.WX, AX.n_win - ix0), nwy = min(P.WY, AY.n_win - iy0);
    const int cols = (nwx - 1) * AX.s + AX.span, rows = (nwy - 1) * AY.s + AY.span;
    const int col0 = ix0 * AX.s + AX.lo, row0 = iy0 * AY.s + AY.lo;
    const int ox = threadIdx.x % OX, g = threadIdx.x / OX, G = P.G;
    const bool ycol = g < G && ox / AX.r < nwx;
    const int passes = C8 / kTcK;
    const uint32_t a_base = smem_u32(sAh), al_base = smem_u32(sAl);

    // Input tiles of the next pass are prefetched into registers during the current one when the
    // eight tiles fit kTcPre elements per thread; otherwise each pass loads its own synchronously.
    const bool pref = kTcK * rows * cols <= kTcPre * kTcThreads;
    float pre[kTcPre];
    auto gather = [&](int pn) {
        const int cbn = pn * kTcK, knn = max(0, min(kTcK, C - cbn)), per = rows * cols;
#pragma unroll
        for (int k = 0; k < kTcPre; ++k) {
            const int e = threadIdx.x + k * kTcThreads;
            const int kc = e / per, rem = e - kc * per;
            float v = 0.f;
            if (kc < knn) {
                const int ry = rem / cols, cx = rem - ry * cols;
                const int sy = ext_index(row0 + ry, AY.n_in, P.pad), sx = ext_index(col0 + cx, AX.n_in, P.pad);
                const Tin* xp = static_cast<const Tin*>(P.x) + (n * C + cbn + kc) * (long long)AY.n_in * AX.n_in;
                v = (sy < 0 || sx < 0) ? P.padv : load_f(xp + (long long)sy * AX.n_in + sx);
            }
            pre[k] = v;
        }
    };
    auto scatter = [&](int pn) {
        const int cbn = pn * kTcK, knn = max(0, min(kTcK, C - cbn)), per = rows * cols;
#pragma unroll
        for (int k = 0; k < kTcPre; ++k) {
            const int e = threadIdx.x + k * kTcThreads;
            const int kc = e / per, rem = e - kc * per;
            if (kc < knn) {
                const int ry = rem / cols, cx = rem - ry * cols;
                sIn[kc * inn + ry * P.ICp + cx] = pre[k];
            }
        }
    };
    if (pref) {
        gather(0);
        scatter(0);
    }

    for (int p = 0; p < passes; ++p) {
        const int buf = p & 1;
        float* bh = sB + buf * 2 * kTcN * kTcK;
        float* bl = bh + kTcN * kTcK;
        // the MMAs of pass p - 2 read this buffer: wait for their commit
        if (p >= 2 && warp == 0) {
            if (!mbar_wait(&bars[buf], (uint32_t)(((p - 2) >> 1) & 1), &g_status_fused_tc) && lane == 0) s_abort = 1;
        }
        const int cb = p * kTcK, kn = max(0, min(kTcK, C - cb));
        for (int kc = 0; kc < kn; ++kc) {
            if (learn) {
                stage_weights<NT>(sWx + kc * wxn, AX, cb + kc);
                stage_weights<NT>(sWy + kc * wyn, AY, cb + kc);
            }
            if (!pref) {
                const long long plane = n * C + cb + kc;
                const Tin* xp = static_cast<const Tin*>(P.x) + plane * (long long)AY.n_in * AX.n_in;
                load_tile<Tin>(sIn + kc * inn, P.ICp, xp, AY.n_in, AX.n_in, row0, col0, rows, cols, P.pad, P.padv);
            }
        }
        __syncthreads();
        if (pref && p + 1 < passes) gather(p + 1);  // in flight during the x pass
        for (int kc = 0; kc < kn; ++kc)
            pass_x<NT>(sH + kc * hn, sIn + kc * inn, sWx + (learn ? kc * wxn : 0), AX, OX, P.ICp, rows, nwx, G);
        __syncthreads();
        if (pref && p + 1 < passes) scatter(p + 1);  // the x pass no longer reads the input tiles
        // y taps, split into the operand-B buffer: row = pixel, column = channel of the pass
        if (ycol) {
            for (int kc = 0; kc < kn; ++kc) {
                const float* h = sH + kc * hn;
                const float* wyb = sWy + (learn ? kc * wyn : 0);
                for (int iyl = g; iyl < nwy; iyl += G) {
                    for (int jy = 0; jy < AY.r; ++jy) {
                        const float* col = h + (iyl * AY.s + AY.off[jy]) * OX + ox;
                        const float* wy = wyb + jy * NT;
                        float a = 0.f;
#pragma unroll
                        for (int k = 0; k < NT; ++k) a = fmaf(wy[k], col[k * OX], a);
                        float zh, zl;
                        split_tf32(a, zh, zl);
                        const int at = op_index((iyl * AY.r + jy) * OX + ox, kc, 2);
                        bh[at] = zh;
                        bl[at] = zl;
                    }
                }
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0 && !s_abort) {
            tc_fence_after();
            const uint64_t da_h = smem_desc(a_base + p * 2 * 128, 128, KCHA * 128);
            const uint64_t da_l = smem_desc(al_base + p * 2 * 128, 128, KCHA * 128);
            const uint64_t db_h = smem_desc(smem_u32(bh), 128, 256);
            const uint64_t db_l = smem_desc(smem_u32(bl), 128, 256);
            mma_tf32(tmem, da_h, db_h, F.idesc, p > 0 ? 1u : 0u);
            mma_tf32(tmem, da_h, db_l, F.idesc, 1u);
            mma_tf32(tmem, da_l, db_h, F.idesc, 1u);
            mma_commit(&bars[buf]);
        }
    }
    // the last commit covers every MMA this CTA issued
    if (warp == 0) {
        const int p = passes - 1;
        if (!mbar_wait(&bars[p & 1], (uint32_t)((p >> 1) & 1), &g_status_fused_tc) && lane == 0) s_abort = 1;
    }
    __syncthreads();
    tc_fence_after();

    if (!s_abort) {
        // warp w reads accumulator lanes 32 (w % 4) .. + 31 (output channels) and column block w / 4,
        // 16 columns at a time, and turns each 32 x 16 block around in shared memory (the operand-B
        // buffers, free now) so that half-warps store 16 consecutive pixels of one channel
        constexpr int kColBlock = kTcN / (kTcThreads / 128);
        const int q = warp & 3, cblk = warp >> 2;
        float* tr = sB + warp * 32 * 16;  // this warp's 32 x 16 block, columns swizzled by row
        const long long oplane = (long long)AY.n_out * AX.n_out;
        const int hl = lane & 15, hrow = lane >> 4;
        for (int c16 = 0; c16 < kColBlock; c16 += 16) {
            const int col = cblk * kColBlock + c16;
            float v[16];
            __syncwarp();
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, v);  // all 32 lanes, converged
#pragma unroll
            for (int i = 0; i < 16; ++i) tr[lane * 16 + (i ^ (lane & 15))] = v[i];
            __syncwarp();
            const int pp = col + hl;
            int oy = AY.n_out, oxg = 0;
            if (pp < pix) {
                const int oyl = pp / OX, oxl = pp - oyl * OX;
                oy = iy0 * AY.r + oyl;
                oxg = ix0 * AX.r + oxl;
            }
            const bool px_ok = oy < AY.n_out && oxg < AX.n_out;
#pragma unroll 4
            for (int rr = 0; rr < 32; rr += 2) {
                const int r = rr + hrow;
                const int o = o0 + q * 32 + r;
                if (px_ok && o < F.c_out) {
                    float val = tr[r * 16 + (hl ^ (r & 15))];
                    if (F.bias) val += __ldg(F.bias + o);
                    val = apply_act(val, F.act, F.alpha, F.lo, F.hi);
                    const long long at = (n * F.c_out + o) * oplane + (long long)oy * AX.n_out + oxg;
                    if (F.dtype_out == FCFS_F32) store_f(static_cast<float*>(F.y) + at, val);
                    else store_f(static_cast<__nv_bfloat16*>(F.y) + at, val);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
    }
}

template <int NT>
cudaError_t launch_tc_nt(const TcParams& F, int din, long long blocks, size_t smem, cudaStream_t st) {
    auto go = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kernel<<<(unsigned)blocks, kTcThreads, smem, st>>>(F);
        return cudaGetLastError();
    };
    if (din == FCFS_F32) return go(fcfs_fused2d_tc<NT, float>);
    if (din == FCFS_BF16) return go(fcfs_fused2d_tc<NT, __nv_bfloat16>);
    return go(fcfs_fused2d_tc<NT, uint8_t>);
}

}  // namespace

// The tensor-core fused forward for a mix of at most 96 input channels; returns
// FCFS_ERR_UNSUPPORTED (without a message) when the shape does not fit it.
int fused_forward_tc(const fcfs_desc* d, const fcfs_epilogue* e, const void* x, void* y, cudaStream_t st) {
    if (!e->mix || d->c > 96) return FCFS_ERR_UNSUPPORTED;
    TcParams F;
    memset(&F, 0, sizeof F);
    int ntk;
    int rc = build_forward_params(d, x, nullptr, &F.P, &ntk);
    if (rc) return rc;
    const int rx = F.P.ax[2].r, ry = F.P.ax[1].r;
    const int WY = std::max(1, 8 / ry), OY = WY * ry;
    const int WX = std::max(1, (kTcN / OY) / rx);
    if (OY * WX * rx > kTcN || WX * rx > kTcThreads) return FCFS_ERR_UNSUPPORTED;
    apply_tiles(F.P, false, WX, WY, 1, std::max(1, kTcThreads / (WX * rx)));
    if (F.P.OX * F.P.OY > kTcN) return FCFS_ERR_UNSUPPORTED;
    F.c_out = e->c_out;
    F.oblocks = (e->c_out + kTcM - 1) / kTcM;
    F.C8 = (int)((d->c + kTcK - 1) / kTcK * kTcK);
    F.mix = e->mix;
    F.bias = e->bias;
    F.act = e->act;
    F.alpha = e->alpha;
    F.lo = e->lo;
    F.hi = e->hi;
    F.dtype_out = d->dtype_out;
    F.y = y;
    // instruction descriptor: D F32, A and B TF32, both K-major, N = 256, M = 128
    F.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
    const bool learn = d->axis[0].w || d->axis[1].w;
    size_t off = sizeof(float) * 2 * kTcM * F.C8;  // A splits
    F.b_off = (int)off;
    off += sizeof(float) * 4 * kTcN * kTcK;  // two buffers x two splits of operand B
    F.w_off = (int)off;
    off += sizeof(float) * (size_t)(learn ? kTcK : 1) * (rx + ry) * ntk;
    off = (off + 15) / 16 * 16;
    F.in_off = (int)off;
    off += sizeof(float) * (size_t)kTcK * F.P.IR * F.P.ICp;
    F.h_off = (int)off;
    off += sizeof(float) * (size_t)kTcK * F.P.IR * F.P.OX;
    off = (off + 15) / 16 * 16;
    F.bar_off = (int)off;
    off += 16;
    if (off > 200 * 1024) return FCFS_ERR_UNSUPPORTED;
    // at most two CTAs per SM: each holds 256 of the SM's 512 tensor-memory columns
    off = std::max<size_t>(off, 80 * 1024);
    const long long blocks = (long long)F.P.tiles_x * F.P.tiles_y * F.oblocks * d->n;
    if (blocks > INT_MAX) return FCFS_ERR_UNSUPPORTED;
    cudaError_t ce;
    switch (ntk) {
        case 1: ce = launch_tc_nt<1>(F, d->dtype_in, blocks, off, st); break;
        case 2: ce = launch_tc_nt<2>(F, d->dtype_in, blocks, off, st); break;
        case 3: ce = launch_tc_nt<3>(F, d->dtype_in, blocks, off, st); break;
        case 4: ce = launch_tc_nt<4>(F, d->dtype_in, blocks, off, st); break;
        case 5: ce = launch_tc_nt<5>(F, d->dtype_in, blocks, off, st); break;
        case 7: ce = launch_tc_nt<7>(F, d->dtype_in, blocks, off, st); break;
        case 9: ce = launch_tc_nt<9>(F, d->dtype_in, blocks, off, st); break;
        default: return FCFS_ERR_UNSUPPORTED;
    }
    return ce == cudaSuccess ? FCFS_OK : cuda_fail(ce, "tensor-core fused forward launch");
}

int read_status_fused_tc(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_fused_tc, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_fused_tc, &z, sizeof(int));
    }
    return v;
}

}  // namespace fcfs
