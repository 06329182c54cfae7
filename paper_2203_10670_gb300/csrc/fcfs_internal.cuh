// Internal definitions shared by the libfcfs translation units: launch
// parameter blocks, per-axis polyphase tables and small device helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include <type_traits>

#include <cuda.h>

#include "fcfs.h"

namespace fcfs {

constexpr int kMaxR = FCFS_MAX_R;   // phases per axis in the fixed tables
constexpr int kMaxFixedTaps = 4;    // nearest 1, bilinear 2, bicubic 4 (the table holds kMaxR x 4 entries)
constexpr int kMaxAATaps = 16;      // taps a widened (antialiased) phase may count on the host

// One spatial axis in compact polyphase form.  Window i reads the input
// positions [i*s + lo, i*s + lo + span); phase j uses the nt taps starting at
// i*s + lo + off[j].  Learnable weights are dense (off[j] = 0, nt = T,
// lo = -L); the fixed methods keep only the taps inside the kernel support.
struct AxisP {
    int r, s;
    int lo;        // first input offset of a window relative to i*s
    int span;      // input positions one window reads (with taps padded to nt)
    int nt;        // taps per phase as the kernel evaluates them (template width)
    int nt_src;    // taps per phase stored in the table (<= nt; the rest are zero)
    int n_in, n_out, n_win;
    int learn;               // 1: weights from the device pointer w
    const float* w;          // learnable [C or 1][r][nt_src]
    long long w_cstride;     // floats between channels (0 = shared)
    short off[kMaxR];        // per-phase first tap relative to lo
    float wf[kMaxR * kMaxFixedTaps];  // fixed-method table [r][nt_src] (r * nt_src <= kMaxR * 4)
};

// Pointwise epilogue of the forward store (the bias and activation of the
// layer that follows FCFS in a fully convolutional network): act and bias
// zero for none.
struct Epi {
    const float* bias;  // [C] or NULL
    int act;            // fcfs_act
    float alpha, lo, hi;
};

__device__ __forceinline__ bool epi_on(const Epi& e) { return e.act != 0 || e.bias != nullptr; }

// fcfs_act applied to v: relu max(v, 0), leaky relu v >= 0 ? v : alpha v, clamp min(max(v, lo), hi)
__device__ __forceinline__ float apply_act(float v, int act, float alpha, float lo, float hi) {
    if (act == FCFS_ACT_RELU) return fmaxf(v, 0.f);
    if (act == FCFS_ACT_LEAKY_RELU) return v >= 0.f ? v : alpha * v;
    if (act == FCFS_ACT_CLAMP) return fminf(fmaxf(v, lo), hi);
    return v;
}

__device__ __forceinline__ float epi_apply(const Epi& e, int c, float v) {
    if (e.bias) v += e.bias[c];
    return apply_act(v, e.act, e.alpha, e.lo, e.hi);
}

// Forward launch parameters.  Axis 0 = D, 1 = H (y), 2 = W (x); missing axes
// are identity axes of extent 1.
struct FwdParams {
    AxisP ax[3];
    long long planes;  // n * c
    int C;
    int pad;
    float padv;
    // tile shape (windows per tile) and derived sizes
    int WX, WY, WD;
    int OX, OY;        // outputs per tile row/column: WX*r_x, WY*r_y
    int IC, ICp, IR;   // input tile columns (pitch) and rows
    int G;             // thread groups: blockDim.x = OX * G
    int tiles_x, tiles_y, tiles_d;
    int ring;          // 3D: depth planes kept in shared memory
    const void* x;
    void* y;
    Epi epi;           // 2D kernels: applied to every output before its store
};

// Adjoint (transposed) polyphase table of one axis.  With v an extended
// input index and v - lo = a*s + u (0 <= u < s), the forward taps reaching v
// are the entries (k, j, t) of residue u: window i = a - k, phase j, tap t.
// Every (j, t) appears once, so there are r*nt entries in total.
constexpr int kMaxS = 64;
constexpr int kMaxAdj = kMaxR * 9;
struct AdjAxis {
    int ustart[kMaxS + 1];
    int ent[kMaxAdj];  // k << 16 | j << 8 | t
    int vmin, vmax;    // extended indices any window touches
};

// Backward launch parameters.  The input-gradient kernels tile the INPUT
// (real indices q); the weight-gradient kernel tiles the OUTPUT like the
// forward.
struct BwdParams {
    AxisP ax[3];
    AdjAxis adj[3];
    long long planes;
    int C;
    int pad;
    float padv;
    // input-gradient tiling
    int QX, QY, QD;          // real input indices per tile
    int qtiles_x, qtiles_y, qtiles_d;
    int GRcap, GCcap, GDcap; // g tile capacity (rows, cols, depth planes)
    int GCp;                 // g tile pitch
    int Gq;                  // thread groups: blockDim = QX * Gq
    int rqx0, rqx1, rqy0, rqy1;  // 2D gather kernel: real indices [rqx0, rqx1) x [rqy0, rqy1) it computes
    // weight-gradient tiling (output tiles as the forward)
    FwdParams fw;
    int dw_axis_off[3];      // offset of each axis's partials in a CTA record (floats)
    int dw_rec;              // floats per CTA record
    const void* x;
    const void* gy;
    void* gx;
    float* ws;
    float* gw[3];
    long long n;
};

// TMA-staged persistent forward: FwdParams plus the tensor map of the input
// viewed as [planes][H][W] and the staging box (BW x BH elements).
struct TmaFwdParams {
    CUtensorMap tmap;
    FwdParams P;
    int BW, BH;        // box width (multiple of 16 bytes) and height
    int align;         // elements per 16 bytes of the input type
    int buf_bytes;     // bytes of one staging buffer (128-byte multiple)
    int bar_off;       // byte offset of the two mbarriers (16-byte aligned)
    int threads;       // CTA size
    long long ntiles;  // tiles_x * tiles_y * planes (< 2^31)
    int chunk;         // tiles per chunk dealt round-robin to the CTAs (0: one contiguous run per CTA)
};

// Adjoint of one axis as a forward-like polyphase operator: window a of the
// adjoint has s phases u, its outputs are the extended input indices
// v = a*s + lo_out + u, and phase u reads the g positions
// a*r + lo_in + off[u] + t, t < ntu[u] (tap t of phase u is the forward
// weight number idx[u][t] = j*nt_src + t_fwd, or -1 for a zero).
constexpr int kMaxAdjTaps = 16;
struct AdjP {
    int s, r;          // adjoint phases per window / g stride per window
    int lo_in, lo_out;
    int span;          // g positions one adjoint window reads (taps padded to nt)
    int nt;            // template tap count
    int n_g, n_x;      // g length (forward output) and real x length (forward input)
    int vmin, vmax;    // extended indices the forward touches
    short off[kMaxS];
    signed char ntu[kMaxS];
    short idx[kMaxS * kMaxAdjTaps];
};

// Bulk-copy staged input-gradient parameters (1D/2D).
struct TmaDxParams {
    CUtensorMap tmap;   // gy viewed as [planes][Ho][Wo]
    AxisP ax[3];        // forward axes (weights)
    AdjP aj[3];         // adjoint tables
    int C, pad;
    int QX, QY;         // real input indices per tile
    int qtiles_x, qtiles_y;
    int GBW, GBH;       // g box (width a multiple of 16 bytes)
    int align;          // g elements per 16 bytes
    int VXcap, VYcap;   // virtual columns / rows a tile may evaluate
    int stages;         // g tiles in flight (2..4)
    int buf_bytes, fx_off, w_off, tab_off, bar_off;
    int threads;
    long long ntiles;
    const void* gy;
    void* gx;
    // register-blocked variant: span every adjoint window reads (same on both
    // axes), adjoint windows per tile row, pitch of the window-relative Fx
    int rs_span, WAcap, FXP;
    int rs_vw;  // register-blocked x pass: elements per vector load of a window (1 = scalar loads)
    int chunk;  // register-blocked kernel: tiles per chunk dealt round-robin to the CTAs (0: one run per CTA)
};

// Bulk-copy staged input-gradient parameters (3D): the 2D tile of real
// (y, x) indices plus a chunk of QD real depth indices; g planes stream
// through a ring of aj[0].span adjoint-interpolated planes.  Depth indices
// that receive folded padding contributions, [0, nL) and [D - nR, D), are
// accumulated in shared memory and stored at the end of their chunk.
struct TmaDx3Params {
    CUtensorMap tmap;   // gy viewed as [planes][Do][Ho][Wo]
    AxisP ax[3];
    AdjP aj[3];
    int C, pad;
    int QX, QY, QD;
    int qtiles_x, qtiles_y, qtiles_d;
    int GBW, GBH, align;
    int VXcap, VYcap;
    int nL, nR;
    int stages;  // g plane buffers in flight (2..4)
    int buf_bytes, fx_off, ring_off, facc_off, w_off, tab_off, bar_off;
    int threads;
    int ntiles;
    int chunk;  // tiles per chunk dealt round-robin to the CTAs (0: one contiguous run per CTA)
    const void* gy;
    void* gx;
};

// Bulk-copy staged weight-gradient parameters (1D/2D): forward tile
// geometry, tensor maps of x and gy, and the record layout of the partials.
struct TmaDwParams {
    CUtensorMap tmap_x;   // x  as [planes][H][W]
    CUtensorMap tmap_g;   // gy as [planes][Ho][Wo]
    FwdParams P;
    int BWx, BHx, BWg, BHg;  // boxes (widths multiples of 16 bytes)
    int align;               // elements per 16 bytes (x and gy share the storage type)
    int xbuf_bytes, gbuf_bytes, sh_off, sv_off, w_off, red_off, bar_off;
    int ICp;                 // pitch of the V intermediate
    int threads, maxseg, rec;  // CTA size, records per CTA, floats per record
    int ntiles, grid;
    int rb;                  // phase count of the register-blocked kernel, 0: per-output kernel
    float* ws;               // [grid][maxseg][rec] floats, then [grid][maxseg] plane ids
    float* gw[3];
    long long n;
};

// Bulk-copy staged 3D forward: FwdParams (with depth tiling), the tensor map
// of the input viewed as [planes][D][H][W], staging box and shared layout.
struct TmaFwd3Params {
    CUtensorMap tmap;
    FwdParams P;
    int BW, BH, align;
    int stages;  // plane buffers in flight (2..4)
    int buf_bytes, sh_off, ring_off, w_off, bar_off;
    int threads;
    int ntiles;
    int chunk;  // tiles per chunk dealt round-robin to the CTAs (0: one contiguous run per CTA)
};

struct NearestParams {
    int r[3], s[3], n_in[3], n_out[3];
    long long planes;
    int pad;
    int align;  // fcfs_align: source index rule
    float padv;
    int OXT, OYT;  // outputs per block along x and y
    int tiles_x, tiles_y;
    const void* x;
    void* y;
};

// SMs of the current device and resident CTAs per SM for kernel `func` at
// `threads` threads and `smem` dynamic shared-memory bytes.  Queried once per
// (device, kernel, threads, bytes) and cached, so a launch costs no driver
// queries after the first; the kernel's dynamic shared-memory limit is only
// ever raised (to the largest size asked for so far).
inline cudaError_t resident_ctas(const void* func, int threads, size_t smem, int* sms, int* per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    using Key = std::tuple<int, const void*, int, size_t>;
    static std::mutex mu;
    static std::map<Key, std::pair<int, int>> cache;
    static std::map<std::pair<int, const void*>, size_t> limit;
    const Key key{dev, func, threads, smem};
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *sms = it->second.first;
        *per_sm = it->second.second;
        return cudaSuccess;
    }
    size_t& lim = limit[{dev, func}];
    if (smem > lim) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        lim = smem;
    }
    int n = 0, p = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, func, threads, smem);
    if (e != cudaSuccess) return e;
    cache[key] = {n, p};
    *sms = n;
    *per_sm = p;
    return cudaSuccess;
}

__host__ __device__ inline int ext_index(int q, int n, int pad) {
    if ((unsigned)q < (unsigned)n) return q;
    if (pad == FCFS_PAD_CONSTANT) return -1;
    if (pad == FCFS_PAD_REPLICATE) return q < 0 ? 0 : n - 1;
    if (n == 1) return 0;
    int p = 2 * (n - 1);
    int m = q % p;
    if (m < 0) m += p;
    return m < n ? m : p - m;
}

__device__ __forceinline__ float load_f(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_f(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p)));
}
__device__ __forceinline__ float load_f(const uint8_t* p) { return (float)__ldg(p); }

// VW consecutive staged samples as FP32 (VW * sizeof(Tg) = 8 or 16 bytes,
// aligned to that size)
template <int VW, typename Tg>
__device__ __forceinline__ void load_vec(const Tg* p, float* v) {
    if constexpr (std::is_same<Tg, float>::value) {
        if constexpr (VW == 2) {
            const float2 t = *reinterpret_cast<const float2*>(p);
            v[0] = t.x, v[1] = t.y;
        } else {
            static_assert(VW == 4, "FP32 vector loads of 2 or 4 samples");
            const float4 t = *reinterpret_cast<const float4*>(p);
            v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
        }
    } else {
        static_assert(VW == 4 || VW == 8, "BF16 vector loads of 4 or 8 samples");
        if constexpr (VW == 4) {
            const uint2 t = *reinterpret_cast<const uint2*>(p);
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.y));
            v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
        } else {
            const uint4 t = *reinterpret_cast<const uint4*>(p);
            const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
                v[2 * k] = a.x, v[2 * k + 1] = a.y;
            }
        }
    }
}

__device__ __forceinline__ void store_f(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_f(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Stores of n <= 4 adjacent outputs (the caller guarantees VW-element alignment).
__device__ __forceinline__ void storev(float* p, const float* a, int n) {
    if (n == 4) *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
    else if (n == 2) *reinterpret_cast<float2*>(p) = make_float2(a[0], a[1]);
    else for (int i = 0; i < n; ++i) p[i] = a[i];
}
__device__ __forceinline__ void storev(__nv_bfloat16* p, const float* a, int n) {
    if (n == 4) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(a[0], a[1]), hi = __floats2bfloat162_rn(a[2], a[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&lo);
        u.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(p) = u;
    } else if (n == 2) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a[0], a[1]);
    } else {
        for (int i = 0; i < n; ++i) p[i] = __float2bfloat16_rn(a[i]);
    }
}

template <int VW>
__device__ __forceinline__ void ldsv(const float* p, float* v) {
    if (VW == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else if (VW == 2) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
        v[0] = *p;
    }
}

__host__ __device__ inline int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// Window range [ilo, ihi] of one axis whose taps reach the extended indices
// that fold onto real indices [q0, q1] (inclusive), and whether the tile
// takes the virtual indices left of 0 / right of N-1.
struct WinRange {
    int ilo, ihi, left, right;
};

__host__ __device__ inline WinRange win_range(const AxisP& A, const AdjAxis& J, int pad, int q0, int q1) {
    WinRange w;
    const int N = A.n_in;
    w.left = pad != FCFS_PAD_CONSTANT && J.vmin < 0 && q0 <= -J.vmin;
    const int rlim = imin(N - 1, 2 * (N - 1) - J.vmax);
    w.right = pad != FCFS_PAD_CONSTANT && J.vmax > N - 1 && q1 >= rlim;
    int vlo = w.left ? J.vmin : q0;
    int vhi = w.right ? J.vmax : q1;
    vlo = imax(vlo, J.vmin);
    vhi = imin(vhi, J.vmax);
    if (vlo > vhi) {
        w.ilo = 0;
        w.ihi = -1;
        return w;
    }
    const int a = vlo - A.lo - A.span + 1;
    w.ilo = imax(0, a >= 0 ? (a + A.s - 1) / A.s : -((-a) / A.s));
    const int b = vhi - A.lo;
    w.ihi = imin(A.n_win - 1, b >= 0 ? b / A.s : -((-b + A.s - 1) / A.s));
    return w;
}

__host__ __device__ inline int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Extended-index range [vlo, vhi] a tile of real indices [q0, q1] evaluates,
// the adjoint windows [alo, ahi] that produce it, and whether the tile takes
// the virtual indices beyond either edge.
struct AxRange {
    int vlo, vhi, alo, ahi;
    bool left, right, covered;
};

__host__ __device__ inline AxRange ax_range(const AdjP& J, int pad, int q0, int q1) {
    AxRange R;
    const int N = J.n_x;
    R.left = pad != FCFS_PAD_CONSTANT && J.vmin < 0 && q0 <= -J.vmin;
    const int rlim = imin(N - 1, 2 * (N - 1) - J.vmax);
    R.right = pad != FCFS_PAD_CONSTANT && J.vmax > N - 1 && q1 >= rlim;
    R.vlo = imax(R.left ? J.vmin : q0, J.vmin);
    R.vhi = imin(R.right ? J.vmax : q1, J.vmax);
    R.covered = q1 <= R.vhi;
    if (R.vlo > R.vhi) {
        R.alo = 0;
        R.ahi = -1;
        R.vhi = R.vlo - 1;
    } else {
        R.alo = floordiv(R.vlo - J.lo_out, J.s);
        R.ahi = floordiv(R.vhi - J.lo_out, J.s);
    }
    return R;
}

// host-side launchers (fcfs_fwd.cu / fcfs_bwd.cu)
cudaError_t launch_forward_2d(const FwdParams& P, int nt, int din, int dout, cudaStream_t st);
cudaError_t launch_forward_3d(const FwdParams& P, int nt, int din, int dout, cudaStream_t st);
cudaError_t launch_nearest(const NearestParams& P, int din, int dout, cudaStream_t st);
cudaError_t launch_forward_tma(const TmaFwdParams& T, int nt, int din, int dout, cudaStream_t st);
size_t forward_tma_smem_bytes(const TmaFwdParams& T);
bool forward_rs_available(const TmaFwdParams& T, int din, int dout);
cudaError_t launch_forward_rs(const TmaFwdParams& T, int din, cudaStream_t st);
int read_status_fwd_tma(int clear);
int read_status_bwd_tma(int clear);
cudaError_t launch_dx_tma(const TmaDxParams& T, int nt, int dg, int dx, cudaStream_t st);
cudaError_t launch_dx_rs(const TmaDxParams& T, int dt, cudaStream_t st);
cudaError_t launch_forward3d_tma(const TmaFwd3Params& T, int nt, int din, int dout, cudaStream_t st);
cudaError_t launch_forward3d_rs(const TmaFwd3Params& T, int din, int dout, cudaStream_t st);
cudaError_t launch_dx3d_tma(const TmaDx3Params& T, int nt, int dt, cudaStream_t st);
bool dx_rs_compiled(int S, int span);
int dx_rs_vector_width(int r, int es);
cudaError_t launch_dw_tma(const TmaDwParams& T, int nt, int dt, cudaStream_t st, const void* x);
bool dw_rb_compiled(int r, int nt);
size_t forward_smem_bytes(const FwdParams& P, bool is3d);
size_t dx_smem_bytes(const BwdParams& P, bool is3d);
size_t dw_smem_bytes(const BwdParams& P);
cudaError_t launch_dx(const BwdParams& P, int nt, int dg, int dx, bool is3d, cudaStream_t st);
int read_status_psk(int clear);
int read_status_psk_bf16(int clear);
cudaError_t launch_dw(const BwdParams& P, int nt, int din, int dg, cudaStream_t st);
cudaError_t launch_dw_reduce(const BwdParams& P, cudaStream_t st);

}  // namespace fcfs
