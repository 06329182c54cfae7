// Backward of the fused layer y = act(M FCFS(x) + b) (the FCN layer of
// Sec. 1 with the resize of Sec. 3.1 / Sec. 4, forward in fcfs_fused.cu).
// With z = FCFS(x) and v = M z + b (both recomputed, FP32):
//   gv[n,o,p] = gy[n,o,p] act'(v[n,o,p])
//   gM[o][c]  = sum_{n,p} gv[n,o,p] z[n,c,p]      gb[o] = sum_{n,p} gv[n,o,p]
//   gz[n,c,p] = sum_o M[o][c] gv[n,o,p]
// and the gradients of x and of the learnable taps are those of the FCFS
// layer for the upstream gradient gz (fcfs_backward).  The three channel
// products run on one tiled FP32 matrix-product kernel over strided views;
// gM is split over pixel ranges and summed in a fixed order, so every result
// is reproducible bit for bit.
#include <algorithm>
#include <climits>
#include <cmath>

#include "fcfs_host.h"

namespace fcfs {
namespace {

// element (b, i, j) of a strided view: p[b sb + i si + j sj]
struct View {
    const float* p;
    long long sb, si, sj;
};

constexpr int kBM = 64, kBN = 64, kBK = 16;  // product tile; 256 threads, 4 x 4 results each

enum { EPI_STORE = 0, EPI_GRAD = 1 };

struct ActP {
    int act;
    float alpha, lo, hi;
    const float* bias;     // [M] or NULL (added to the product before the derivative)
    const void* gy;        // [b][M][N] of dtype gy_dt
    int gy_dt;
};

__device__ __forceinline__ float act_grad(const ActP& a, float v) {
    switch (a.act) {
        case FCFS_ACT_RELU: return v > 0.f ? 1.f : 0.f;
        case FCFS_ACT_LEAKY_RELU: return v > 0.f ? 1.f : a.alpha;
        case FCFS_ACT_CLAMP: return (v >= a.lo && v <= a.hi) ? 1.f : 0.f;
        default: return 1.f;
    }
}

__device__ __forceinline__ float load_gy(const ActP& a, long long i) {
    return a.gy_dt == FCFS_F32 ? static_cast<const float*>(a.gy)[i]
                               : __bfloat162float(static_cast<const __nv_bfloat16*>(a.gy)[i]);
}

// C(b, m, n) = sum_{k < K} A(b, m, k) B(b, k, n) for m < M, n < N, in k
// order, written at C[b scb + m scm + n].  EPI_GRAD: C = gy(b, m, n)
// act'(C + bias[m]), C and gy dense [b][M][N].  The batch b = blockIdx.z is an
// image, or one pixel range of a split product.
// Split products (S > 1): batch z = image z / S, pixel range z % S of kr
// pixels each (the last one shorter, K the full length), the range's offset
// applied along each operand's k stride.
template <int EPI>
__global__ void __launch_bounds__(256) fused_mm(int M, int N, int K, View A, View B, float* C, long long scb,
                                                long long scm, ActP act, int S, int kr) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int img = b / S, sp = b - img * S;
    const long long k_off = (long long)sp * kr;
    if (S > 1) K = (int)min((long long)kr, (long long)K - k_off);
    const float* Ap = A.p + img * A.sb + k_off * A.sj;
    const float* Bp = B.p + img * B.sb + k_off * B.si;
    const bool a_k_unit = A.sj == 1, b_n_unit = B.sj == 1;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += kBK) {
        // 64 x 16 elements of each operand, four per thread; consecutive threads take the
        // operand's unit-stride index, so the loads coalesce whichever index it is
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + q * 256;
            const int kk = a_k_unit ? (e & (kBK - 1)) : (e >> 6);
            const int mm = a_k_unit ? (e >> 4) : (e & (kBM - 1));
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? Ap[gm * A.si + gk * A.sj] : 0.f;
            const int nn = b_n_unit ? (e & (kBN - 1)) : (e >> 4);
            const int kb = b_n_unit ? (e >> 6) : (e & (kBK - 1));
            const int gn = n0 + nn, gk2 = k0 + kb;
            Bs[kb][nn] = (gn < N && gk2 < K) ? Bp[gk2 * B.si + gn * B.sj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx * 4 + j;
            if (gn >= N) continue;
            const long long ci = b * scb + gm * scm + gn;
            float v = acc[i][j];
            if (EPI == EPI_GRAD) {
                if (act.bias) v += act.bias[gm];
                v = load_gy(act, ci) * act_grad(act, v);
            }
            C[ci] = v;
        }
    }
}

// gv = gy act'(z + bias) without a mix (c_out == c): elementwise over [n][c][P]
__global__ void fused_grad_identity(long long total, int C, long long P, const float* z, float* gv, ActP act) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)((i / P) % C);
        float v = z[i];
        if (act.bias) v += act.bias[c];
        gv[i] = load_gy(act, i) * act_grad(act, v);
    }
}

// out[o] = sum over the nb rows of in[r][o] (r ascending): the split partial sums of gM
__global__ void fused_sum_rows(const float* in, int nb, int len, float* out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= len) return;
    float s = 0.f;
    for (int r = 0; r < nb; ++r) s += in[(long long)r * len + o];
    out[o] = s;
}

// part[s][o] = sum over the images and pixel range s (of kr pixels) of gv[n,o,p]: block (o, s),
// fixed-order partial sums and tree; fused_sum_rows then adds the ranges in order
__global__ void __launch_bounds__(256) fused_bias_grad(const float* gv, int n, int O, long long P, long long kr,
                                                       float* part) {
    __shared__ float red[256];
    const int o = blockIdx.x, sp = blockIdx.y;
    const long long p0 = sp * kr, p1 = min(P, p0 + kr);
    float s = 0.f;
    for (int b = 0; b < n; ++b) {
        const float* row = gv + ((long long)b * O + o) * P;
        for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) s += row[p];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)sp * O + o] = red[0];
}

struct FusedBwdLayout {
    size_t z_off, gv_off, part_off, ws_off, total;
    int splits;  // pixel ranges per image of the gM product
    long long krange;
};

int fused_bwd_layout(const fcfs_desc* d, const fcfs_epilogue* e, FusedBwdLayout* L) {
    const long long P = d->out_shape[0] * d->out_shape[1];
    const long long n = d->n, C = d->c, O = e->c_out;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    fcfs_desc dz = *d;
    dz.dtype_out = FCFS_F32;
    L->z_off = 0;
    L->gv_off = al((size_t)(n * C * P) * 4);
    L->part_off = L->gv_off + al((size_t)(n * O * P) * 4);
    L->splits = (int)std::max<long long>(1, std::min<long long>((304 + n - 1) / n, (P + 4095) / 4096));
    L->krange = (P + L->splits - 1) / L->splits;
    // partial sums of the mix gradient, then (reused) of the bias gradient: at most 64 ranges
    L->ws_off = L->part_off + al((size_t)std::max<long long>(n * L->splits * O * C, 64 * O) * 4);
    L->total = L->ws_off + al(fcfs_backward_workspace(&dz));
    return FCFS_OK;
}

int check_fused(const fcfs_desc* d, const fcfs_epilogue* e) {
    int rc = validate_desc(d, true);
    if (rc) return rc;
    if (!e) return fail(FCFS_ERR_ARG, "epilogue is NULL");
    if (d->w2d) return fail(FCFS_ERR_UNSUPPORTED, "the fused layer follows the separable kernels");
    if (d->ndim != 2) return fail(FCFS_ERR_UNSUPPORTED, "the fused layer takes 2D images");
    if (e->c_out < 1) return fail(FCFS_ERR_ARG, "c_out must be >= 1");
    if (!e->mix && e->c_out != d->c) return fail(FCFS_ERR_ARG, "without a mix c_out must equal c");
    if (e->act < FCFS_ACT_NONE || e->act > FCFS_ACT_CLAMP) return fail(FCFS_ERR_ARG, "unknown activation %d", e->act);
    if (e->act == FCFS_ACT_CLAMP && !(e->lo <= e->hi)) return fail(FCFS_ERR_ARG, "clamp needs lo <= hi");
    if (((uintptr_t)e->mix) % 4 || ((uintptr_t)e->bias) % 4) return fail(FCFS_ERR_ARG, "mix or bias misaligned");
    if (d->dtype_in == FCFS_U8) return fail(FCFS_ERR_UNSUPPORTED, "no gradient for uint8 inputs");
    if (d->dtype_out != FCFS_F32 && d->dtype_out != FCFS_BF16) return fail(FCFS_ERR_ARG, "gy must be FP32 or BF16");
    return FCFS_OK;
}

}  // namespace
}  // namespace fcfs

using namespace fcfs;

extern "C" size_t fcfs_backward_fused_workspace(const fcfs_desc* d, const fcfs_epilogue* e) {
    clear_error();
    if (check_fused(d, e)) return 0;
    FusedBwdLayout L;
    fused_bwd_layout(d, e, &L);
    return L.total;
}

extern "C" int fcfs_backward_fused(const fcfs_desc* d, const fcfs_epilogue* e, const void* x, const void* gy,
                                   void* gx, float* gmix, float* gbias, float* const* gw, void* workspace,
                                   size_t ws_bytes, void* stream) {
    NvtxRange nv("fcfs_backward_fused");
    clear_error();
    int rc = check_fused(d, e);
    if (rc) return rc;
    if (gmix && !e->mix) return fail(FCFS_ERR_ARG, "gmix given but the layer has no mix");
    if (gbias && !e->bias) return fail(FCFS_ERR_ARG, "gbias given but the layer has no bias");
    if (((uintptr_t)gmix) % 4 || ((uintptr_t)gbias) % 4) return fail(FCFS_ERR_ARG, "gmix or gbias misaligned");
    bool want_w = false;
    for (int a = 0; a < 2 && gw; ++a) want_w |= gw[a] != nullptr;
    if (!gx && !gmix && !gbias && !want_w) return FCFS_OK;
    FusedBwdLayout L;
    fused_bwd_layout(d, e, &L);
    if (!workspace || ws_bytes < L.total)
        return fail(FCFS_ERR_ARG, "workspace of %zu bytes needed (fcfs_backward_fused_workspace)", L.total);
    if (((uintptr_t)workspace) % 256) return fail(FCFS_ERR_ARG, "workspace must be 256-byte aligned");
    if (!x || !gy) return fail(FCFS_ERR_ARG, "x and gy must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    const long long P = d->out_shape[0] * d->out_shape[1];
    const int n = (int)d->n, C = (int)d->c, O = e->c_out;
    if (P == 0 || n == 0 || P >= INT_MAX || n > 65535 || (long long)n * std::max(C, O) * P >= (1LL << 40))
        return fail(FCFS_ERR_UNSUPPORTED, "empty or too large fused layer");
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    float* z = reinterpret_cast<float*>(ws + L.z_off);
    float* gv = reinterpret_cast<float*>(ws + L.gv_off);
    float* part = reinterpret_cast<float*>(ws + L.part_off);
    // z = FCFS(x) in FP32
    fcfs_desc dz = *d;
    dz.dtype_out = FCFS_F32;
    rc = fcfs_forward(&dz, x, z, stream);
    if (rc) return rc;
    ActP ap;
    ap.act = e->act;
    ap.alpha = e->alpha;
    ap.lo = e->lo;
    ap.hi = e->hi;
    ap.bias = e->bias;
    ap.gy = gy;
    ap.gy_dt = d->dtype_out;
    // gv = gy act'(M z + b)
    if (e->mix) {
        View A{e->mix, 0, C, 1};          // M[o][c]
        View B{z, (long long)C * P, P, 1};  // z[n][c][p]
        dim3 grid((unsigned)((P + kBN - 1) / kBN), (unsigned)((O + kBM - 1) / kBM), (unsigned)n);
        fused_mm<EPI_GRAD><<<grid, 256, 0, st>>>(O, (int)P, C, A, B, gv, (long long)O * P, P, ap, 1, C);
    } else {
        const long long total = (long long)n * C * P;
        fused_grad_identity<<<(unsigned)std::min<long long>((total + 255) / 256, 152LL * 16), 256, 0, st>>>(total, C, P, z, gv, ap);
    }
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "fused backward: activation gradient");
    // gM = sum over images and pixel ranges of gv z^T (fixed-order sum of the split products)
    if (gmix) {
        // all images' pixel ranges in one launch: part[img S + s][o][c]
        const int S = L.splits;
        View A{gv, (long long)O * P, P, 1};  // (img, o, k) -> gv[img][o][k]
        View B{z, (long long)C * P, 1, P};   // (img, k, c) -> z[img][c][k]
        dim3 grid((unsigned)((C + kBN - 1) / kBN), (unsigned)((O + kBM - 1) / kBM), (unsigned)(n * S));
        fused_mm<EPI_STORE><<<grid, 256, 0, st>>>(O, C, (int)P, A, B, part, (long long)O * C, C, ap, S, (int)L.krange);
        fused_sum_rows<<<(O * C + 255) / 256, 256, 0, st>>>(part, n * S, O * C, gmix);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "fused backward: mix gradient");
    }
    if (gbias) {
        // the mix gradient's partials are summed: their space holds the bias partials now
        const int SB = (int)std::min<long long>(64, (P + 4095) / 4096);
        const long long krb = (P + SB - 1) / SB;
        fused_bias_grad<<<dim3(O, SB), 256, 0, st>>>(gv, n, O, P, krb, part);
        fused_sum_rows<<<(O + 255) / 256, 256, 0, st>>>(part, SB, O, gbias);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "fused backward: bias gradient");
    }
    if (!gx && !want_w) return FCFS_OK;
    // gz = M^T gv (into z's buffer, which the mix gradient has read), then the FCFS backward
    const float* gz = gv;
    if (e->mix) {
        View A{e->mix, 0, 1, C};            // (c, o) -> M[o][c]
        View B{gv, (long long)O * P, P, 1};  // gv[n][o][p]
        dim3 grid((unsigned)((P + kBN - 1) / kBN), (unsigned)((C + kBM - 1) / kBM), (unsigned)n);
        fused_mm<EPI_STORE><<<grid, 256, 0, st>>>(C, (int)P, O, A, B, z, (long long)C * P, P, ap, 1, O);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "fused backward: channel gradient");
        gz = z;
    }
    return fcfs_backward(&dz, x, gz, gx, gw, ws + L.ws_off, L.total - L.ws_off, stream);
}
