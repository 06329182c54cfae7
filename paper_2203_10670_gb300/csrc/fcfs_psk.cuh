// Polyphase strip kernel (PSK): one separable polyphase pass pair over a 2D
// plane, organised for sm_100-class GPUs as a producer/consumer pipeline.
//
// The pass pair is the FCFS layer of Sec. 3.1 / Sec. 4 in register-blocked
// form,
//   out[iy R_y + jy + oy0][ix R_x + jx + ox0]
//     = sum_ky WFy[jy][ky] sum_kx WFx[jx][kx] in~[iy s_y + lo_y + ky][ix s_x + lo_x + kx],
// with span-wide weight rows WF[j][k] (zero outside a phase's taps).  The
// forward runs it on x with the layer's tables; the interior of the input
// gradient runs it on the upstream gradient g with the adjoint tables (the
// adjoint of one axis is itself polyphase: s phases per window, stride r).
//
// Work split: a tile is a strip of consecutive x windows (one per consumer
// thread) and a band of y windows.  A thread walks down its window column one
// window step (s new rows) at a time: each new row is reduced in registers to
// its R x-pass values, which join the thread's ring of the last SPAN rows (in
// registers); the y window is then complete and its R x R outputs are
// stored.  No block-wide barrier separates the passes, and the x pass of a
// row is done once per band (no halo rows between the y windows of a band).
// Phases, stride and span are compile-time and the same on both axes, so the
// S rows of a step are independent FMA chains the scheduler can overlap.
//
// Staging: a producer warp copies the tile's input rows into a ring of NS
// stages of CH rows with one bulk copy per row (cp.async.bulk, completion
// counted on the stage's "full" mbarrier); consumer warps release a stage on
// its "empty" mbarrier.  Rows outside the input are copies of the row the
// padding rule maps them to (replicate, reflect) or flagged as constant;
// columns outside the input are read through the padding rule by the threads
// whose windows reach them.  Every wait is bounded; a wait that runs out
// records FCFS_DEVERR_TIMEOUT, the consumers leave, and the producer waits
// (bounded) for the copies it issued before the CTA exits.
#pragma once

#include "fcfs_internal.cuh"
#include "fcfs_tma.cuh"

namespace fcfs {

constexpr int kPskMaxW = 128;      // span-form weight entries per axis (R * SPAN)
constexpr int kPskWarps = 4;       // consumer warps per CTA (128 windows per strip)
constexpr int kPskThreads = (kPskWarps + 1) * 32;

// One axis of a strip pass: window w reads input positions w*s + lo + k
// (k < SPAN) and writes outputs w*R + j + out_off (j < R).
struct PskAxis {
    int s, lo;
    int n_in;     // real input extent (positions outside follow the padding rule)
    int n_out;    // outputs outside [0, n_out) are not stored
    int out_off;
    int w0, w1;   // windows [w0, w1) of this launch
};

struct PskParams {
    PskAxis ay, ax;
    long long planes;
    int C;
    int pad;            // extension rule of the staged input
    float padv;         // its constant
    const void* in;     // [planes][ay.n_in][ax.n_in]
    void* out;          // [planes][ay.n_out][ax.n_out]
    // tiling
    int strip_w, band_h;     // windows per strip (<= consumer threads) and per band
    int nstrips, nbands;
    int ntiles;
    int pitch;               // elements per staged row (16-byte multiple in bytes)
    int al;                  // input elements per 16 bytes
    int CH, NS;              // rows per stage, stages
    int w_off, flag_off, bar_off;  // shared-memory layout (bytes)
    int xvec;                // bytes per vector window load in the x pass (0: scalar)
    // span-form weights: fixed tables, or per-channel gathers from learnable weights
    int learn_x, learn_y;
    const float* wl_x;
    const float* wl_y;
    long long wcs_x, wcs_y;  // floats between channels (0 = shared)
    float wf_x[kPskMaxW], wf_y[kPskMaxW];
    short wi_x[kPskMaxW], wi_y[kPskMaxW];  // learnable: entry index in the channel's table, -1 = zero
    Epi epi;                 // store epilogue (forward), act 0 and no bias when unused
};

}  // namespace fcfs

#ifdef FCFS_PSK_KERNELS

namespace fcfs {

static __device__ int g_status_psk = 0;

namespace {

template <typename T>
__device__ __forceinline__ float psk_f(T v);
template <>
__device__ __forceinline__ float psk_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float psk_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float psk_f<uint8_t>(uint8_t v) { return (float)v; }

template <typename T>
__device__ __forceinline__ T psk_cast(float v);
template <>
__device__ __forceinline__ float psk_cast<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 psk_cast<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up when another warp raised the CTA's abort
// flag.  The try_wait carries a suspend-time hint: a waiting warp sleeps until
// the phase completes (or the hint runs out) instead of spinning, so it takes
// no issue slots from the warps that compute.
__device__ __forceinline__ bool psk_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool psk_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    for (int it = 0; it < (1 << 18); ++it) {
        if (psk_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    atomicOr(&g_status_psk, FCFS_DEVERR_TIMEOUT);
    return false;
}

// Tile geometry (every thread computes it the same way).
struct PskTile {
    int plane, c;
    int wxa, nwx, wya, nwy;  // first window and count per axis
    int r0, nrows;           // first input row (may be negative) and rows of the tile
    int c0, x_al, xoff;      // first input column, its 16-byte aligned start, c0 - x_al
    int nchunks;
};

template <int SPX, int SPY>
__device__ __forceinline__ PskTile psk_tile(const PskParams& P, int t) {
    PskTile g;
    const int per_plane = P.nstrips * P.nbands;
    g.plane = t / per_plane;
    const int rem = t - g.plane * per_plane;
    const int band = rem / P.nstrips, strip = rem - band * P.nstrips;
    g.c = g.plane % P.C;
    g.wxa = P.ax.w0 + strip * P.strip_w;
    g.nwx = min(P.strip_w, P.ax.w1 - g.wxa);
    g.wya = P.ay.w0 + band * P.band_h;
    g.nwy = min(P.band_h, P.ay.w1 - g.wya);
    g.r0 = g.wya * P.ay.s + P.ay.lo;
    g.nrows = (g.nwy - 1) * P.ay.s + SPY;
    g.c0 = g.wxa * P.ax.s + P.ax.lo;
    g.x_al = g.c0 >= 0 ? (g.c0 / P.al) * P.al : -(((-g.c0) + P.al - 1) / P.al) * P.al;
    g.xoff = g.c0 - g.x_al;
    g.nchunks = (g.nrows + P.CH - 1) / P.CH;
    return g;
}

// span-form weights of one axis for channel c into shared memory
template <int R, int SPAN>
__device__ __forceinline__ void psk_stage_w(float* dst, const PskParams& P, bool xaxis, int c, int tid, int nthr) {
    const int learn = xaxis ? P.learn_x : P.learn_y;
    const float* wl = xaxis ? P.wl_x : P.wl_y;
    const long long cs = xaxis ? P.wcs_x : P.wcs_y;
    for (int e = tid; e < R * SPAN; e += nthr) {
        float v;
        if (learn) {
            const int i = xaxis ? P.wi_x[e] : P.wi_y[e];
            v = i >= 0 ? wl[(long long)c * cs + i] : 0.f;
        } else {
            v = xaxis ? P.wf_x[e] : P.wf_y[e];
        }
        dst[e] = v;
    }
}

// x table with rows padded to SPXP entries (16-byte rows for vector reads)
template <int R, int SPAN, int SPANP>
__device__ __forceinline__ void psk_stage_wx(float* dst, const PskParams& P, int c, int lane) {
    for (int e = lane; e < R * SPANP; e += 32) {
        const int j = e / SPANP, k = e - j * SPANP;
        float v = 0.f;
        if (k < SPAN) {
            const int f = j * SPAN + k;
            if (P.learn_x) {
                const int i = P.wi_x[f];
                v = i >= 0 ? P.wl_x[(long long)c * P.wcs_x + i] : 0.f;
            } else {
                v = P.wf_x[f];
            }
        }
        dst[e] = v;
    }
}

// load SPX samples of a window from a staged row: scalar (XV = 0), or vectors of XV bytes
template <int SPX, int XV, typename Tin>
__device__ __forceinline__ void load_window(const Tin* p, float* v) {
    if constexpr (XV > 0) {
        constexpr int E = XV / sizeof(Tin);
#pragma unroll
        for (int q = 0; q < (SPX + E - 1) / E; ++q) {
            if constexpr (XV == 16) {
                const uint4 u = *reinterpret_cast<const uint4*>(p + q * E);
                const Tin* e = reinterpret_cast<const Tin*>(&u);
#pragma unroll
                for (int i = 0; i < E; ++i)
                    if (q * E + i < SPX) v[q * E + i] = psk_f<Tin>(e[i]);
            } else {
                const uint2 u = *reinterpret_cast<const uint2*>(p + q * E);
                const Tin* e = reinterpret_cast<const Tin*>(&u);
#pragma unroll
                for (int i = 0; i < E; ++i)
                    if (q * E + i < SPX) v[q * E + i] = psk_f<Tin>(e[i]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < SPX; ++k) v[k] = psk_f<Tin>(p[k]);
    }
}

// Bytes of the vector stores of R adjacent outputs.
template <int R, typename Tout>
struct StoreVec {
    static constexpr int bytes = std::is_same<Tout, float>::value ? (R % 4 == 0 ? 16 : R % 2 == 0 ? 8 : 4)
                                                                  : (R % 4 == 0 ? 8 : R % 2 == 0 ? 4 : 2);
};

// R adjacent outputs of one row at p (aligned to StoreVec<R, Tout>::bytes, all in range)
template <int R, typename Tout>
__device__ __forceinline__ void store_row_vec(Tout* p, const float* a) {
    if constexpr (std::is_same<Tout, float>::value) {
        if constexpr (R % 4 == 0) {
#pragma unroll
            for (int q = 0; q < R; q += 4) *reinterpret_cast<float4*>(p + q) = make_float4(a[q], a[q + 1], a[q + 2], a[q + 3]);
        } else if constexpr (R % 2 == 0) {
#pragma unroll
            for (int q = 0; q < R; q += 2) *reinterpret_cast<float2*>(p + q) = make_float2(a[q], a[q + 1]);
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j) p[j] = a[j];
        }
    } else {
        if constexpr (R % 4 == 0) {
#pragma unroll
            for (int q = 0; q < R; q += 4) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(a[q], a[q + 1]), hi = __floats2bfloat162_rn(a[q + 2], a[q + 3]);
                uint2 u;
                u.x = *reinterpret_cast<uint32_t*>(&lo);
                u.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(p + q) = u;
            }
        } else if constexpr (R % 2 == 0) {
#pragma unroll
            for (int q = 0; q < R; q += 2) *reinterpret_cast<__nv_bfloat162*>(p + q) = __floats2bfloat162_rn(a[q], a[q + 1]);
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j) p[j] = psk_cast<Tout>(a[j]);
        }
    }
}

// R adjacent outputs of one row starting at column ox, each stored when inside [0, n_out)
template <int R, typename Tout>
__device__ __noinline__ void store_row_checked(Tout* rowp, int ox, int n_out, const float* a) {
    for (int j = 0; j < R; ++j)
        if (ox + j >= 0 && ox + j < n_out) rowp[ox + j] = psk_cast<Tout>(a[j]);
}

// x pass of one row for a window that reaches outside the input, or a
// constant row: samples through the padding rule (rarely taken; out of line)
template <int R, int SPAN, int SPANP, typename Tin>
__device__ __noinline__ void psk_xrow_slow(const Tin* rowp, int flag, int wc0, int x_al, const PskParams& P,
                                           const float* sWx, float* h) {
    float wsum[R];
    for (int j = 0; j < R; ++j) {
        float s = 0.f;
        for (int k = 0; k < SPAN; ++k) s += sWx[j * SPANP + k];
        wsum[j] = s;
    }
    if (flag) {
        for (int j = 0; j < R; ++j) h[j] = P.padv * wsum[j];
        return;
    }
    const int W = P.ax.n_in;
    float v[SPAN];
    for (int k = 0; k < SPAN; ++k) {
        const int c = wc0 + k;
        if (c >= 0 && c < W) v[k] = psk_f<Tin>(rowp[c - x_al]);
        else if (P.pad == FCFS_PAD_CONSTANT) v[k] = P.padv;
        else v[k] = psk_f<Tin>(rowp[ext_index(c, W, P.pad) - x_al]);
    }
    for (int j = 0; j < R; ++j) {
        float a = 0.f;
        for (int k = 0; k < SPAN; ++k) a = fmaf(sWx[j * SPANP + k], v[k], a);
        h[j] = a;
    }
}

// CTAs per SM the register budget is sized for: four for the small window
// shapes, three for the rest (the y ring and both weight tables in registers).
template <int R, int S, int SPAN>
struct PskMinBlocks {
    static constexpr int v = (R * SPAN <= 12 && R <= 3) ? 4 : 3;
};

// R phases, stride S and window span SPAN on both axes (compile time); XV:
// bytes per vector window load in the x pass (0: scalar loads).  The y ring
// of the last SPAN x-pass rows is held in registers: a window step computes
// the S new rows (independent FMA chains), forms the R x R outputs and shifts
// the ring by S.  Stage chunks are aligned to window steps: chunk 0 holds the
// SPAN - S rows before the first step, every later chunk CH rows (a multiple
// of S).  Windows reaching outside the input and constant rows take an
// out-of-line path, decided per warp and chunk.
template <int R, int S, int SPAN, int XV, typename Tin, typename Tout>
__global__ void __launch_bounds__(kPskThreads, (PskMinBlocks<R, S, SPAN>::v)) fcfs_psk(const __grid_constant__ PskParams P) {
    static_assert(SPAN > S, "windows overlap");
    constexpr int PRO = SPAN - S;
    constexpr bool WREG = R * SPAN <= 24;   // x weights in registers
    constexpr bool YREG = R * SPAN <= 24;   // y weights in registers
    constexpr int JG = R * R <= 16 ? R : (16 / R > 0 ? 16 / R : 1);
    constexpr int SPANP = (SPAN + 3) / 4 * 4;
    constexpr int WSTRIDE = (R * SPANP + R * SPAN + 3) / 4 * 4;  // floats per warp table (16-byte multiple)
    constexpr int VB = StoreVec<R, Tout>::bytes;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // each consumer warp keeps its own copy of the tables: no barrier between consumer warps
    float* sWx = reinterpret_cast<float*>(smem + P.w_off) + (warp < kPskWarps ? warp : 0) * WSTRIDE;
    float* sWy = sWx + R * SPANP;
    int* flags = reinterpret_cast<int*>(smem + P.flag_off);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + P.bar_off);
    uint64_t* empty = full + P.NS;
    const int es = (int)sizeof(Tin);
    const int stage_bytes = P.CH * P.pitch * es;

    const int per = (P.ntiles + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per, t_end = min(P.ntiles, t_begin + per);
    if (t_begin >= t_end) return;
    if (threadIdx.x == 0) {
        for (int k = 0; k < P.NS; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kPskWarps);
        }
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    volatile int* abort_flag = &s_abort;

    if (warp == kPskWarps) {
        // ---------------- producer: one bulk copy per staged row
        const char* in = static_cast<const char*>(P.in);
        const int H = P.ay.n_in, W = P.ax.n_in;
        long long q = 0;  // chunks issued
        for (int t = t_begin; t < t_end; ++t) {
            const PskTile g = psk_tile<SPAN, SPAN>(P, t);
            const char* plane = in + (long long)g.plane * H * W * es;
            const int ca = max(g.x_al, 0), cb = min(g.x_al + P.pitch, W);
            const uint32_t row_bytes = cb > ca ? (uint32_t)((cb - ca) * es) : 0u;
            const int nch = (PRO > 0 ? 1 : 0) + (g.nwy * S + P.CH - 1) / P.CH;
            for (int ch = 0; ch < nch; ++ch, ++q) {
                const int st = (int)(q % P.NS);
                if (q >= P.NS && !psk_wait(&empty[st], (uint32_t)(((q / P.NS) - 1) & 1), abort_flag)) {
                    if (lane == 0) {
                        s_abort = 1;
                        for (long long d = max(0LL, q - P.NS); d < q; ++d)
                            mbar_wait(&full[d % P.NS], (uint32_t)((d / P.NS) & 1), &g_status_psk);
                    }
                    return;
                }
                // rows of this chunk: the prologue, or window steps
                const int rfirst = (PRO > 0 && ch == 0) ? 0 : PRO + (ch - (PRO > 0 ? 1 : 0)) * P.CH;
                const int rcount = (PRO > 0 && ch == 0) ? PRO : min(P.CH, g.nrows - rfirst);
                const int rr = lane;
                const int row = g.r0 + rfirst + rr;
                bool copy = false;
                int src_row = 0;
                if (rr < rcount) {
                    if (row >= 0 && row < H) {
                        src_row = row;
                        copy = true;
                    } else if (P.pad != FCFS_PAD_CONSTANT) {
                        src_row = ext_index(row, H, P.pad);
                        copy = true;
                    }
                }
                const unsigned cm = __ballot_sync(0xffffffffu, copy && row_bytes > 0);
                const unsigned fm = __ballot_sync(0xffffffffu, rr < rcount && !copy);
                if (lane == 0) flags[st] = (int)fm;  // constant rows of the chunk, one bit per row
                __syncwarp();  // the flags are written before the arrive releases them
                if (lane == 0) {
                    // the arrive (with the byte count) precedes the copies: the phase cannot
                    // complete before every copy of the chunk has landed
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[st])),
                                 "r"((uint32_t)__popc(cm) * row_bytes)
                                 : "memory");
                }
                __syncwarp();
                if ((cm >> lane) & 1u) {
                    unsigned char* dst = smem + st * stage_bytes + (rr * P.pitch + (ca - g.x_al)) * es;
                    fence_proxy_async_smem();
                    bulk_g2s(dst, plane + ((long long)src_row * W + ca) * es, row_bytes, &full[st]);
                }
            }
        }
        return;
    }

    // ---------------- consumers: thread t owns x window wxa + t of the tile
    const int t = threadIdx.x;
    const bool learn = P.learn_x || P.learn_y;
    float wx[WREG ? R : 1][WREG ? SPAN : 1];
    float wy[YREG ? R : 1][YREG ? SPAN : 1];
    int cur_c = -1;
    long long q = 0;  // chunks consumed
    for (int tile = t_begin; tile < t_end; ++tile) {
        const PskTile g = psk_tile<SPAN, SPAN>(P, tile);
        if (cur_c < 0 || (learn && g.c != cur_c)) {
            __syncwarp();  // the warp is done with the previous tables
            psk_stage_wx<R, SPAN, SPANP>(sWx, P, g.c, lane);
            psk_stage_w<R, SPAN>(sWy, P, false, g.c, lane, 32);
            __syncwarp();
#pragma unroll
            for (int j = 0; j < R; ++j)
#pragma unroll
                for (int k = 0; k < SPAN; ++k) {
                    if constexpr (WREG) wx[j][k] = sWx[j * SPANP + k];
                    if constexpr (YREG) wy[j][k] = sWy[j * SPAN + k];
                }
            cur_c = g.c;
        }
        const bool active = t < g.nwx;
        const int wc0 = g.c0 + t * S;  // first input column of this thread's window
        const bool edge = active && (wc0 < 0 || wc0 + SPAN > P.ax.n_in);
        const bool warp_edge = __any_sync(0xffffffffu, edge);
        const int xo = g.xoff + t * S;
        Tout* oplane = static_cast<Tout*>(P.out) + (long long)g.plane * P.ay.n_out * P.ax.n_out;
        const int ox = (g.wxa + t) * R + P.ax.out_off;
        const bool vec_store = ox >= 0 && ox + R <= P.ax.n_out &&
                               (reinterpret_cast<uintptr_t>(oplane + ox) % VB) == 0 &&
                               ((long long)P.ax.n_out * sizeof(Tout)) % VB == 0;
        const bool epi = epi_on(P.epi);
        float ring[SPAN][R];
#pragma unroll
        for (int k = 0; k < SPAN; ++k)
#pragma unroll
            for (int j = 0; j < R; ++j) ring[k][j] = 0.f;
        const int nch = (PRO > 0 ? 1 : 0) + (g.nwy * S + P.CH - 1) / P.CH;
        int wi = 0;  // next y window (relative to the band)
        for (int ch = 0; ch < nch; ++ch, ++q) {
            const int st = (int)(q % P.NS);
            if (!psk_wait(&full[st], (uint32_t)((q / P.NS) & 1), abort_flag)) {
                s_abort = 1;
                return;
            }
            const Tin* sbuf = reinterpret_cast<const Tin*>(smem + st * stage_bytes);
            const unsigned cflags = (unsigned)flags[st];
            const bool fast = !warp_edge && cflags == 0u;  // warp-uniform
            if (PRO > 0 && ch == 0) {
                if (active) {
#pragma unroll
                    for (int k = 0; k < PRO; ++k) {
                        if (fast) {
                            float v[SPAN];
                            load_window<SPAN, XV, Tin>(sbuf + k * P.pitch + xo, v);
#pragma unroll
                            for (int j = 0; j < R; ++j) {
                                float a = 0.f;
#pragma unroll
                                for (int kk = 0; kk < SPAN; ++kk)
                                    a = fmaf(WREG ? wx[WREG ? j : 0][WREG ? kk : 0] : sWx[j * SPANP + kk], v[kk], a);
                                ring[k][j] = a;
                            }
                        } else {
                            psk_xrow_slow<R, SPAN, SPANP, Tin>(sbuf + k * P.pitch, (cflags >> k) & 1u, wc0, g.x_al, P,
                                                               sWx, ring[k]);
                        }
                    }
                }
            } else {
                const int steps = min(P.CH / S, g.nwy - wi);
                for (int sidx = 0; sidx < steps; ++sidx, ++wi) {
                    if (!active) continue;
                    // the S new rows of window wi
                    if (fast) {
#pragma unroll
                        for (int i = 0; i < S; ++i) {
                            float v[SPAN];
                            load_window<SPAN, XV, Tin>(sbuf + (sidx * S + i) * P.pitch + xo, v);
#pragma unroll
                            for (int j = 0; j < R; ++j) {
                                float a = 0.f;
#pragma unroll
                                for (int kk = 0; kk < SPAN; ++kk)
                                    a = fmaf(WREG ? wx[WREG ? j : 0][WREG ? kk : 0] : sWx[j * SPANP + kk], v[kk], a);
                                ring[PRO + i][j] = a;
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < S; ++i) {
                            const int rr = sidx * S + i;
                            psk_xrow_slow<R, SPAN, SPANP, Tin>(sbuf + rr * P.pitch, (cflags >> rr) & 1u, wc0, g.x_al,
                                                               P, sWx, ring[PRO + i]);
                        }
                    }
                    // y pass: rows wi*S .. wi*S + SPAN - 1 are ring[0 .. SPAN - 1]
                    const int oyb = (g.wya + wi) * R + P.ay.out_off;
#pragma unroll
                    for (int jy0 = 0; jy0 < R; jy0 += JG) {
                        float acc[JG][R];
#pragma unroll
                        for (int a = 0; a < JG; ++a)
#pragma unroll
                            for (int jx = 0; jx < R; ++jx) acc[a][jx] = 0.f;
#pragma unroll
                        for (int k = 0; k < SPAN; ++k) {
#pragma unroll
                            for (int a = 0; a < JG; ++a) {
                                if (jy0 + a < R) {
                                    const float wv = YREG ? wy[YREG ? jy0 + a : 0][YREG ? k : 0] : sWy[(jy0 + a) * SPAN + k];
#pragma unroll
                                    for (int jx = 0; jx < R; ++jx) acc[a][jx] = fmaf(wv, ring[k][jx], acc[a][jx]);
                                }
                            }
                        }
#pragma unroll
                        for (int a = 0; a < JG; ++a) {
                            const int oy = oyb + jy0 + a;
                            if (jy0 + a >= R || oy < 0 || oy >= P.ay.n_out) continue;
                            if (epi) {
#pragma unroll
                                for (int jx = 0; jx < R; ++jx) acc[a][jx] = epi_apply(P.epi, g.c, acc[a][jx]);
                            }
                            Tout* rowp = oplane + (long long)oy * P.ax.n_out;
                            if (vec_store) store_row_vec<R, Tout>(rowp + ox, acc[a]);
                            else store_row_checked<R, Tout>(rowp, ox, P.ax.n_out, acc[a]);
                        }
                    }
                    // shift the ring by S rows
#pragma unroll
                    for (int k = 0; k < PRO; ++k)
#pragma unroll
                        for (int j = 0; j < R; ++j) ring[k][j] = ring[k + S][j];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
    }
}

}  // namespace
}  // namespace fcfs

#endif  // FCFS_PSK_KERNELS
