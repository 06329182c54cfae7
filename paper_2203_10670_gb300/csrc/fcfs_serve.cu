// FCFS serving: a persistent request loop on one stream (continuous
// batching).  Requests of mixed image sizes, r/s factors and methods are
// admitted as parameter slots and pool memory free up; every loop step
// launches ONE grouped kernel (K6) over tiles taken round-robin from all
// admitted requests, so work of requests that arrived while others were on
// the GPU overlaps on the device.  Each tile is computed exactly as the
// standalone forward computes it, so a result does not depend on the mix.
#include <chrono>
#include <climits>
#include <string>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <memory>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "fcfs_fwd_tile.cuh"
#include "fcfs_tma.cuh"
#include "fcfs_host.h"
#include "fcfs_sched.h"

namespace fcfs {
namespace {

constexpr int kServeThreads = 256;
// four CTAs per SM (the register limit too); larger budgets (taller tiles, fewer CTAs) measured
// slower: 72 KB 91, 96 KB 72, 144 KB 43 Gpix/s against 98 on the mixed stream
constexpr int kServeMaxSmem = 48 * 1024;
// work items dealt to the CTAs in chunks of four consecutive items (tiles of one request,
// mostly): tile costs differ across requests, and contiguous runs left SMs idle at the end
// of a step (75 -> 97 Gpix/s on the mixed stream)
constexpr int kServeChunk = 4;


struct WorkItem {
    int slot;
    int tile;
};

// Per-request scalars of the tile computation, staged in shared memory when a
// CTA moves to another request, and the per-tile geometry computed once by one
// thread.  Every thread then reads them from shared memory into registers:
// the slot itself lives in global memory, and reading its fields throughout
// the passes would reload them at global latency.
struct ServeReq {
    const void* x;
    void* y;
    int din, nt;
    int H, W, Ho, Wo;
    int rx, sx, ry, sy, lox, loy, spanx, spany;
    int nwinx, nwiny, tiles_x, tiles_y, WX, WY, OX, G, ICp, IR;
    int pad;
    float padv;
};

struct ServeTile {
    int plane, ix0, iy0, nwx, nwy, cols, rows, col0, row0;
};

// Device parameter slot of one admitted request: the compact record the
// kernel reads (scalars, phase taps padded to four, phase offsets), written
// on the host at admission, then the full forward parameters of the plan.
struct ServeSlot {
    ServeReq q;
    float wx[kMaxR * 4], wy[kMaxR * 4];
    short offx[kMaxR], offy[kMaxR];
    FwdParams P;
    int din;  // fcfs_dtype of x
    int nt;   // tap template (1 nearest, 2 bilinear, 4 bicubic)
};

// The compact record of a slot from its forward parameters (y set).
void fill_serve_rec(ServeSlot& S) {
    const AxisP& AX = S.P.ax[2];
    const AxisP& AY = S.P.ax[1];
    ServeReq& q = S.q;
    q.x = S.P.x;
    q.y = S.P.y;
    q.din = S.din;
    q.nt = S.nt;
    q.H = AY.n_in;
    q.W = AX.n_in;
    q.Ho = AY.n_out;
    q.Wo = AX.n_out;
    q.rx = AX.r;
    q.sx = AX.s;
    q.ry = AY.r;
    q.sy = AY.s;
    q.lox = AX.lo;
    q.loy = AY.lo;
    q.spanx = AX.span;
    q.spany = AY.span;
    q.nwinx = AX.n_win;
    q.nwiny = AY.n_win;
    q.tiles_x = S.P.tiles_x;
    q.tiles_y = S.P.tiles_y;
    q.WX = S.P.WX;
    q.WY = S.P.WY;
    q.OX = S.P.OX;
    q.G = S.P.G;
    q.ICp = S.P.ICp;
    q.IR = S.P.IR;
    q.pad = S.P.pad;
    q.padv = S.P.padv;
    for (int e = 0; e < AX.r * 4; ++e) {
        const int j = e >> 2, t = e & 3;
        S.wx[e] = t < AX.nt_src ? AX.wf[j * AX.nt_src + t] : 0.f;
    }
    for (int e = 0; e < AY.r * 4; ++e) {
        const int j = e >> 2, t = e & 3;
        S.wy[e] = t < AY.nt_src ? AY.wf[j * AY.nt_src + t] : 0.f;
    }
    for (int e = 0; e < AX.r; ++e) S.offx[e] = AX.off[e];
    for (int e = 0; e < AY.r; ++e) S.offy[e] = AY.off[e];
}

// Four adjacent outputs of one row: a 16-byte (FP32) or 8-byte (BF16) store
// when aligned and inside the row, else element by element.
__device__ __forceinline__ void store4(float* p, int nvalid, bool vec, const float* a) {
    if (vec) {
        *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
        return;
    }
    for (int i = 0; i < nvalid; ++i) p[i] = a[i];
}
__device__ __forceinline__ void store4(__nv_bfloat16* p, int nvalid, bool vec, const float* a) {
    if (vec) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(a[0], a[1]), hi = __floats2bfloat162_rn(a[2], a[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&lo);
        u.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(p) = u;
        return;
    }
    for (int i = 0; i < nvalid; ++i) p[i] = __float2bfloat16_rn(a[i]);
}

// One tile: stage the padded input (index map), x pass with one window per
// thread (its span samples loaded once for every phase), y pass with four
// adjacent output columns per thread (vector shared-memory loads and stores).
template <int NT, typename Tin, typename Tout>
__device__ __forceinline__ void serve_tile_body(const ServeReq& q, const ServeTile& g, const float* sWx,
                                                const float* sWy, const short* offx, const short* offy, float* sIn) {
    constexpr int MAXSPAN = 24;  // span of a window: phases' taps (fixed methods, r <= 16 here)
    const int OX = q.OX;
    // the intermediate starts on a 16-byte boundary (vector reads in the y pass)
    float* sH = sIn + ((q.IR * q.ICp + 3) & ~3);
    const Tin* xp = static_cast<const Tin*>(q.x) + (long long)g.plane * q.H * q.W;
    load_tile<Tin>(sIn, q.ICp, xp, q.H, q.W, g.row0, g.col0, g.rows, g.cols, q.pad, q.padv);
    __syncthreads();
    // ---- x pass: thread = (window ixl, row group); sH[ry][ixl rx + jx]
    const int rx = q.rx;
    constexpr int RW = NT == 4 ? 5 : 8;  // phases a window-per-thread x pass holds in registers
    if (rx <= RW && q.spanx <= MAXSPAN) {
        const int nthr = g.nwx;
        const int G1 = blockDim.x / nthr;
        const int ixl = threadIdx.x % nthr, grp = threadIdx.x / nthr;
        if (grp < G1) {
            // the phases' taps and offsets in registers (phases beyond rx are never used)
            float w[RW][NT];
            int of[RW];
#pragma unroll
            for (int jx = 0; jx < RW; ++jx) {
                of[jx] = jx < rx ? offx[jx] : 0;
#pragma unroll
                for (int t = 0; t < NT; ++t) w[jx][t] = jx < rx ? sWx[jx * 4 + t] : 0.f;
            }
            const float* row = sIn + grp * q.ICp + ixl * q.sx;
            float* dst = sH + grp * OX + ixl * rx;
            const int rstep = G1 * q.ICp, dstep = G1 * OX;
            for (int ry = grp; ry < g.rows; ry += G1) {
#pragma unroll
                for (int jx = 0; jx < RW; ++jx) {
                    if (jx < rx) {
                        const float* src = row + of[jx];
                        float acc = 0.f;
#pragma unroll
                        for (int t = 0; t < NT; ++t) acc = fmaf(w[jx][t], src[t], acc);
                        dst[jx] = acc;
                    }
                }
                row += rstep;
                dst += dstep;
            }
        }
    } else {
        const int ox = threadIdx.x % OX, grp = threadIdx.x / OX, G = q.G;
        const int jx = ox % rx, ixl = ox / rx;
        if (ixl < g.nwx && grp < G) {
            float w[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) w[t] = sWx[jx * 4 + t];
            const float* base = sIn + ixl * q.sx + offx[jx];
            for (int ry = grp; ry < g.rows; ry += G) {
                const float* row = base + ry * q.ICp;
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t) acc = fmaf(w[t], row[t], acc);
                sH[ry * OX + ox] = acc;
            }
        }
    }
    __syncthreads();
    // ---- y pass: thread = (four output columns, row group); outputs at pixel-shuffled positions
    const int ncolv = g.nwx * rx;          // valid tile columns
    const int nq = (OX + 3) / 4;           // column quads of the tile
    const int G2 = blockDim.x / nq;
    const int cq = threadIdx.x % nq, grp = threadIdx.x / nq;
    const int ox = cq * 4;
    const int gox = g.ix0 * rx + ox;
    if (grp >= G2 || ox >= ncolv || gox >= q.Wo) return;
    const int nvalid = min(4, min(ncolv - ox, q.Wo - gox));
    Tout* yp = static_cast<Tout*>(q.y) + (long long)g.plane * q.Ho * q.Wo + gox;
    const bool vec = nvalid == 4 && (OX % 4) == 0 &&
                     (reinterpret_cast<uintptr_t>(yp) % (4 * sizeof(Tout))) == 0 && (q.Wo % 4) == 0;
    const int nrow = min(g.nwy * q.ry, q.Ho - g.iy0 * q.ry);
    // output row orow of the tile = window iyl, phase jy, walked without division
    const int di = G2 / q.ry, dj = G2 - di * q.ry;
    int iyl = grp / q.ry, jy = grp - iyl * q.ry;
    const bool ox4 = (OX % 4) == 0;
    Tout* yrow = yp + (long long)(g.iy0 * q.ry + grp) * q.Wo;
    const long long ystep = (long long)G2 * q.Wo;
    for (int orow = grp; orow < nrow; orow += G2) {
        const float* col = sH + (iyl * q.sy + offy[jy]) * OX + ox;
        const float4 wy = *reinterpret_cast<const float4*>(sWy + jy * 4);
        const float wt[4] = {wy.x, wy.y, wy.z, wy.w};
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            float h[4];
            if (ox4) {
                const float4 v = *reinterpret_cast<const float4*>(col + t * OX);
                h[0] = v.x, h[1] = v.y, h[2] = v.z, h[3] = v.w;
            } else {
                for (int i = 0; i < 4; ++i) h[i] = ox + i < OX ? col[t * OX + i] : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = fmaf(wt[t], h[i], acc[i]);
        }
        store4(yrow, nvalid, vec, acc);
        yrow += ystep;
        iyl += di;
        jy += dj;
        if (jy >= q.ry) {
            jy -= q.ry;
            ++iyl;
        }
    }
}

template <typename Tin, typename Tout>
__device__ __forceinline__ void serve_tile(const ServeReq& q, const ServeTile& g, const float* sWx, const float* sWy,
                                           const short* offx, const short* offy, float* sIn) {
    if (q.nt == 1) serve_tile_body<1, Tin, Tout>(q, g, sWx, sWy, offx, offy, sIn);
    else if (q.nt == 2) serve_tile_body<2, Tin, Tout>(q, g, sWx, sWy, offx, offy, sIn);
    else serve_tile_body<4, Tin, Tout>(q, g, sWx, sWy, offx, offy, sIn);
}

// K6: a persistent grouped kernel.  The CTAs take chunks of consecutive work
// items round-robin (the items of one request are consecutive, so a request's
// record is staged once per run of its tiles); each item names a request slot
// and one of its tiles.
template <typename Tout>
__global__ void __launch_bounds__(kServeThreads) fcfs_serve_grouped(const ServeSlot* __restrict__ slots,
                                                                     const WorkItem* __restrict__ work, int n_items,
                                                                     int chunk) {
    extern __shared__ __align__(16) float smem[];
    __shared__ ServeReq sq;
    __shared__ __align__(16) float sWx[kMaxR * 4];
    __shared__ __align__(16) float sWy[kMaxR * 4];
    __shared__ short offx[kMaxR], offy[kMaxR];
    const TileDeal deal = deal_tiles(n_items, chunk);
    int last_slot = -1;
    for (int kk = 0; kk < deal.n; ++kk) {
        const WorkItem w = work[deal.tile(kk)];
        __syncthreads();  // the previous tile is done with the staged parameters and buffers
        if (w.slot != last_slot) {
            // the slot's compact record, copied by all threads
            const ServeSlot& S = slots[w.slot];
            const int rx = S.q.rx, ry = S.q.ry;
            static_assert(sizeof(ServeReq) % 4 == 0, "record copied in 4-byte words");
            const int* qsrc = reinterpret_cast<const int*>(&S.q);
            int* qdst = reinterpret_cast<int*>(&sq);
            for (int e = threadIdx.x; e < (int)(sizeof(ServeReq) / 4); e += blockDim.x) qdst[e] = qsrc[e];
            for (int e = threadIdx.x; e < rx * 4; e += blockDim.x) sWx[e] = S.wx[e];
            for (int e = threadIdx.x; e < ry * 4; e += blockDim.x) sWy[e] = S.wy[e];
            for (int e = threadIdx.x; e < rx; e += blockDim.x) offx[e] = S.offx[e];
            for (int e = threadIdx.x; e < ry; e += blockDim.x) offy[e] = S.offy[e];
            last_slot = w.slot;
            __syncthreads();
        }
        const ServeReq q = sq;
        // tile index -> geometry in 32-bit arithmetic (a request has fewer than 2^31 tiles)
        ServeTile g;
        {
            const int txy = q.tiles_x * q.tiles_y;
            g.plane = w.tile / txy;
            const int rem = w.tile - g.plane * txy;
            const int ty = rem / q.tiles_x, tx = rem - ty * q.tiles_x;
            g.ix0 = tx * q.WX;
            g.iy0 = ty * q.WY;
            g.nwx = min(q.WX, q.nwinx - g.ix0);
            g.nwy = min(q.WY, q.nwiny - g.iy0);
            g.cols = (g.nwx - 1) * q.sx + q.spanx;
            g.rows = (g.nwy - 1) * q.sy + q.spany;
            g.col0 = g.ix0 * q.sx + q.lox;
            g.row0 = g.iy0 * q.sy + q.loy;
        }
        if (q.din == FCFS_U8) serve_tile<uint8_t, Tout>(q, g, sWx, sWy, offx, offy, smem);
        else if (q.din == FCFS_F32) serve_tile<float, Tout>(q, g, sWx, sWy, offx, offy, smem);
        else serve_tile<__nv_bfloat16, Tout>(q, g, sWx, sWy, offx, offy, smem);
    }
}

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

struct StepRec {
    sched::Step step;
    cudaEvent_t ev = nullptr;
    WorkItem* host = nullptr;  // pinned staging of the work list
    WorkItem* dev = nullptr;
    size_t cap = 0;
    bool busy = false;
};

struct Server {
    fcfs_serve_config cfg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    unsigned char* pool_base = nullptr;
    ServeSlot* slots_dev = nullptr;
    ServeSlot* slots_host = nullptr;  // pinned, one per slot
    static constexpr int kSteps = 4;  // grouped launches that may be queued on the stream at once
    StepRec steps[kSteps];
    int step_next = 0;
    sched::Scheduler* S = nullptr;
    std::unordered_map<uint64_t, std::unique_ptr<ServeSlot>> pending_params;  // submitted, waiting for a slot
    std::map<uint64_t, std::pair<void*, int>> out_of;  // id -> (y, dtype) for completed pooled outputs
    std::map<uint64_t, std::pair<size_t, size_t>> pooled;  // id -> (pool offset, bytes) kept for the caller
    std::deque<uint64_t> done_ids;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread worker;
    bool stop = false;
    int error = FCFS_OK;
    uint64_t next_id = 1;
    long long steps_launched = 0, rejected = 0;
    double first_arrival = -1, last_done = -1;
    int grid_cap = 1;  // resident CTAs of the grouped kernel (persistent grid)
};

int launch_step(Server& sv, StepRec& R) {
    NvtxRange nv("fcfs serve step");
    const long long n = R.step.tiles;
    if ((size_t)n > R.cap) return FCFS_ERR_NOMEM;
    long long k = 0;
    for (auto& p : R.step.pieces)
        for (long long t = 0; t < p.count; ++t) R.host[k++] = WorkItem{p.slot, (int)(p.first + t)};
    cudaError_t e = cudaMemcpyAsync(R.dev, R.host, n * sizeof(WorkItem), cudaMemcpyHostToDevice, sv.stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve work list copy");
    const unsigned grid = (unsigned)std::min<long long>(n, (long long)sv.grid_cap);
    if (sv.cfg.out_dtype == FCFS_BF16)
        fcfs_serve_grouped<__nv_bfloat16><<<grid, kServeThreads, kServeMaxSmem, sv.stream>>>(sv.slots_dev, R.dev, (int)n, kServeChunk);
    else
        fcfs_serve_grouped<float><<<grid, kServeThreads, kServeMaxSmem, sv.stream>>>(sv.slots_dev, R.dev, (int)n, kServeChunk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "serve grouped launch");
    e = cudaEventRecord(R.ev, sv.stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve event record");
    R.busy = true;
    ++sv.steps_launched;
    return FCFS_OK;
}

void worker_loop(Server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progressed = false;
        // 1. completions
        for (auto& R : sv->steps) {
            if (!R.busy) continue;
            const cudaError_t q = cudaEventQuery(R.ev);
            if (q == cudaErrorNotReady) continue;
            R.busy = false;
            if (q != cudaSuccess) {
                sv->error = cuda_fail(q, "serve step");
                continue;
            }
            const double t = now_s();
            // a canceled request's pool block is returned at once (its output is not read)
            auto done = sv->S->finish(R.step, t, sv->cfg.auto_release != 0);
            for (auto& r : done) {
                sv->done_ids.push_back(r.id);
                if (r.canceled) {
                    if (r.pool_off != SIZE_MAX) sv->S->release_output(r.pool_off, r.out_bytes);
                    sv->out_of.erase(r.id);
                    continue;
                }
                if (r.pool_off != SIZE_MAX) sv->pooled[r.id] = {r.pool_off, r.out_bytes};
                sv->last_done = t;
            }
            progressed = true;
        }
        if (progressed) sv->done_cv.notify_all();
        // 2. admission: the parameter slots of this round are copied with one copy of the slot
        //    range they span, in stream order before any step uses them (slots in between are
        //    either active, copied unchanged, or free and not read by any launched step)
        auto adm = sv->S->admit(now_s());
        int smin = INT_MAX, smax = -1;
        for (auto* r : adm) {
            auto it = sv->pending_params.find(r->id);
            ServeSlot& sl = sv->slots_host[r->slot];
            sl = *it->second;
            sv->pending_params.erase(it);
            if (r->pool_off != SIZE_MAX) {
                sl.P.y = sv->pool_base + r->pool_off;
                // with auto_release the block is reused once the request completes
                if (!sv->cfg.auto_release) sv->out_of[r->id] = {sl.P.y, sv->cfg.out_dtype};
            }
            fill_serve_rec(sl);
            smin = std::min(smin, r->slot);
            smax = std::max(smax, r->slot);
            progressed = true;
        }
        if (smax >= 0) {
            cudaError_t e = cudaMemcpyAsync(sv->slots_dev + smin, sv->slots_host + smin,
                                            sizeof(ServeSlot) * (size_t)(smax - smin + 1), cudaMemcpyHostToDevice,
                                            sv->stream);
            if (e != cudaSuccess) sv->error = cuda_fail(e, "serve slot copy");
        }
        // 3. launch the next step when a step record is free
        StepRec& R = sv->steps[sv->step_next];
        if (!R.busy && sv->S->active() > 0) {
            R.step = sv->S->next_step();
            if (R.step.tiles > 0) {
                const int rc = launch_step(*sv, R);
                if (rc != FCFS_OK) sv->error = rc;
                sv->step_next = (sv->step_next + 1) % Server::kSteps;
                progressed = true;
            }
        }
        if (!progressed) {
            bool busy = false;
            for (auto& R : sv->steps) busy |= R.busy;
            if (busy) {
                // GPU busy: poll again after yielding the processor (a timed sleep would often
                // oversleep the step and leave the GPU idle)
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                // idle: sleep until a submission arrives
                sv->cv.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

// Tile plan for serving: 256-thread CTAs, about 128 output columns and 64
// output rows, shared memory within the grouped kernel's budget.
void plan_serve_tiles(FwdParams& P) {
    int WX = std::max(1, 128 / P.ax[2].r), WY = std::max(1, 64 / P.ax[1].r);
    for (int it = 0; it < 64; ++it) {
        apply_tiles(P, false, WX, WY, 1, 0);
        const int G = std::max(1, kServeThreads / P.OX);
        P.G = G;
        const size_t need = (((size_t)P.IR * P.ICp + 3) / 4 * 4 + (size_t)P.IR * P.OX) * sizeof(float);
        if (P.OX <= kServeThreads && need <= (size_t)kServeMaxSmem) return;
        if (P.OX > kServeThreads && WX > 1) WX = (WX + 1) / 2;
        else if (WY > 1) WY = (WY + 1) / 2;
        else if (WX > 1) WX = (WX + 1) / 2;
        else return;
    }
}

}  // namespace
}  // namespace fcfs

using namespace fcfs;

extern "C" {

double fcfs_serve_clock(void) { return now_s(); }

int fcfs_serve_create(const fcfs_serve_config* cfg, void* stream, void** handle) {
    clear_error();
    if (!cfg || !handle) return fail(FCFS_ERR_ARG, "config and handle are required");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 4096) return fail(FCFS_ERR_ARG, "max_inflight must be 1..4096");
    if (cfg->tile_budget_per_step < 1) return fail(FCFS_ERR_ARG, "tile_budget_per_step must be >= 1");
    if (cfg->out_dtype != FCFS_F32 && cfg->out_dtype != FCFS_BF16) return fail(FCFS_ERR_ARG, "out_dtype must be F32 or BF16");
    *handle = nullptr;
    Server* sv = new Server();
    sv->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e != cudaSuccess) {
        delete sv;
        return cuda_fail(e, "cudaGetDevice");
    }
    auto cleanup = [&](int rc) {
        if (sv->pool_base) cudaFree(sv->pool_base);
        if (sv->slots_dev) cudaFree(sv->slots_dev);
        if (sv->slots_host) cudaFreeHost(sv->slots_host);
        for (auto& R : sv->steps) {
            if (R.dev) cudaFree(R.dev);
            if (R.host) cudaFreeHost(R.host);
            if (R.ev) cudaEventDestroy(R.ev);
        }
        if (sv->own_stream && sv->stream) cudaStreamDestroy(sv->stream);
        delete sv->S;
        delete sv;
        return rc;
    };
    if (stream) {
        sv->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "stream create"));
        sv->own_stream = true;
    }
    if (cfg->hbm_budget_bytes > 0) {
        e = cudaMalloc(&sv->pool_base, cfg->hbm_budget_bytes);
        if (e != cudaSuccess) return cleanup(fail(FCFS_ERR_NOMEM, "pool of %zu bytes: %s", cfg->hbm_budget_bytes,
                                                  cudaGetErrorString(e)));
    }
    e = cudaMalloc(&sv->slots_dev, sizeof(ServeSlot) * cfg->max_inflight);
    if (e == cudaSuccess) e = cudaMallocHost(&sv->slots_host, sizeof(ServeSlot) * cfg->max_inflight);
    for (auto& R : sv->steps) {
        R.cap = (size_t)cfg->tile_budget_per_step;
        if (e == cudaSuccess) e = cudaMalloc(&R.dev, sizeof(WorkItem) * R.cap);
        if (e == cudaSuccess) e = cudaMallocHost(&R.host, sizeof(WorkItem) * R.cap);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
        e = cudaFuncSetAttribute(fcfs_serve_grouped<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kServeMaxSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fcfs_serve_grouped<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kServeMaxSmem);
    }
    if (e == cudaSuccess) {
        int sms = 0, per_sm = 0, dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, cfg->out_dtype == FCFS_BF16 ? (const void*)fcfs_serve_grouped<__nv_bfloat16>
                                                     : (const void*)fcfs_serve_grouped<float>,
                kServeThreads, kServeMaxSmem);
        sv->grid_cap = std::max(1, sms * per_sm);
    }
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "serve buffers"));
    sv->S = new sched::Scheduler(cfg->hbm_budget_bytes, cfg->max_inflight, cfg->tile_budget_per_step);
    sv->worker = std::thread(worker_loop, sv);
    *handle = sv;
    return FCFS_OK;
}

int fcfs_serve_submit(void* h, const fcfs_desc* d, const void* x, void* y, double arrival_s,
                      unsigned long long* req_id) {
    unsigned long long id = 0;
    int n = 0;
    const int rc = fcfs_serve_submit_batch(h, 1, d, &x, &y, &arrival_s, &id, &n);
    if (req_id) *req_id = id;
    return rc;
}

int fcfs_serve_submit_batch(void* h, int count, const fcfs_desc* descs, const void* const* xs, void* const* ys,
                            const double* arrivals, unsigned long long* ids, int* n_submitted) {
    clear_error();
    Server* sv = (Server*)h;
    if (n_submitted) *n_submitted = 0;
    if (!sv) return fail(FCFS_ERR_ARG, "null handle");
    if (count < 0 || (count > 0 && (!descs || !xs || !arrivals))) return fail(FCFS_ERR_ARG, "bad batch arguments");
    // validate and plan every request outside the lock, then queue them in one critical section
    std::vector<std::unique_ptr<ServeSlot>> slots;
    std::vector<sched::Request> reqs;
    slots.reserve(count);
    reqs.reserve(count);
    int status = FCFS_OK;
    for (int k = 0; k < count; ++k) {
        const fcfs_desc* d = descs + k;
        const void* x = xs[k];
        void* y = ys ? ys[k] : nullptr;
        int rc = validate_desc(d, true);
        if (!rc && d->ndim != 2) rc = fail(FCFS_ERR_UNSUPPORTED, "serving takes 2D images");
        if (!rc && d->w2d) rc = fail(FCFS_ERR_UNSUPPORTED, "serving uses separable kernels");
        for (int a = 0; !rc && a < 2; ++a)
            if (d->axis[a].w) rc = fail(FCFS_ERR_UNSUPPORTED, "serving uses the fixed method tables");
        if (!rc && !x) rc = fail(FCFS_ERR_ARG, "x is NULL");
        // every slot of a step is stored by the grouped kernel instantiated for the
        // server's out_dtype, caller-placed outputs included
        if (!rc && d->dtype_out != sv->cfg.out_dtype)
            rc = fail(FCFS_ERR_ARG, "dtype_out %d differs from the server's out_dtype %d", d->dtype_out,
                      sv->cfg.out_dtype);
        if (!rc && (((uintptr_t)x) % dtype_size(d->dtype_in) || (y && ((uintptr_t)y) % dtype_size(d->dtype_out))))
            rc = fail(FCFS_ERR_ARG, "x or y not aligned to its element size");
        auto sl = std::make_unique<ServeSlot>();
        memset(sl.get(), 0, sizeof(ServeSlot));
        int ntk = 1;
        if (!rc) rc = build_forward_params(d, x, y, &sl->P, &ntk);
        if (!rc && ntk != 1 && ntk != 2 && ntk != 4)
            rc = fail(FCFS_ERR_UNSUPPORTED, "serving supports nearest, bilinear, bicubic (no antialiased windows)");
        sched::Request r;
        if (!rc) {
            plan_serve_tiles(sl->P);
            sl->din = d->dtype_in;
            sl->nt = ntk;
            r.tiles = (long long)sl->P.tiles_x * sl->P.tiles_y * sl->P.planes;
            if (r.tiles >= (1LL << 31)) rc = fail(FCFS_ERR_UNSUPPORTED, "request too large");
        }
        if (rc) {
            status = rc;
            break;
        }
        r.out_bytes = y ? 0 : (size_t)numel_out(d) * dtype_size(d->dtype_out);
        r.out_pixels = (double)numel_out(d) / (double)d->c;
        r.bytes = (double)numel_in(d) * dtype_size(d->dtype_in) + (double)numel_out(d) * dtype_size(d->dtype_out);
        r.arrival = arrivals[k];
        reqs.push_back(r);
        slots.push_back(std::move(sl));
    }
    const std::string why = status ? std::string(fcfs_last_error()) : std::string();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->error) return fail(sv->error, "server stopped after an earlier error");
    int done = 0;
    for (size_t k = 0; k < reqs.size(); ++k) {
        sched::Request& r = reqs[k];
        r.id = sv->next_id++;
        if (r.tiles == 0) {  // empty output: complete at once
            sv->done_ids.push_back(r.id);
        } else {
            if (!sv->S->submit(r)) {
                ++sv->rejected;
                sv->next_id--;
                status = fail(FCFS_ERR_NOMEM, "output of %zu bytes exceeds the serving pool", r.out_bytes);
                break;
            }
            sv->pending_params[r.id] = std::move(slots[k]);
            if (sv->first_arrival < 0 || r.arrival < sv->first_arrival) sv->first_arrival = r.arrival;
        }
        if (ids) ids[k] = r.id;
        ++done;
    }
    if (n_submitted) *n_submitted = done;
    if (done > 0) sv->cv.notify_all();
    if (status && status != FCFS_ERR_NOMEM) return fail(status, "%s", why.c_str());
    return status;
}

int fcfs_serve_poll(void* h, unsigned long long* done_ids, int max, int* n_done) {
    clear_error();
    Server* sv = (Server*)h;
    if (!sv || (max > 0 && !done_ids) || !n_done) return fail(FCFS_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    int n = 0;
    while (n < max && !sv->done_ids.empty()) {
        done_ids[n++] = sv->done_ids.front();
        sv->done_ids.pop_front();
    }
    *n_done = n;
    return sv->error;
}

int fcfs_serve_result(void* h, unsigned long long id, void** y) {
    clear_error();
    Server* sv = (Server*)h;
    if (!sv || !y) return fail(FCFS_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->out_of.find(id);
    if (it == sv->out_of.end()) return fail(FCFS_ERR_ARG, "request %llu has no pooled output", id);
    *y = it->second.first;
    return FCFS_OK;
}

int fcfs_serve_release(void* h, unsigned long long id) {
    clear_error();
    Server* sv = (Server*)h;
    if (!sv) return fail(FCFS_ERR_ARG, "null handle");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->pooled.find(id);
    if (it == sv->pooled.end()) return fail(FCFS_ERR_ARG, "request %llu holds no pool memory", id);
    sv->S->release_output(it->second.first, it->second.second);
    sv->pooled.erase(it);
    sv->out_of.erase(id);
    sv->cv.notify_all();
    return FCFS_OK;
}

int fcfs_serve_cancel(void* h, unsigned long long id) {
    clear_error();
    Server* sv = (Server*)h;
    if (!sv) return fail(FCFS_ERR_ARG, "null handle");
    std::lock_guard<std::mutex> lk(sv->mu);
    sched::Request r;
    const int rc = sv->S->cancel(id, true, &r);
    if (rc < 0) return fail(FCFS_ERR_ARG, "request %llu is neither queued nor running", id);
    sv->pending_params.erase(id);
    sv->out_of.erase(id);
    if (rc == 1) {
        sv->done_ids.push_back(id);
        sv->done_cv.notify_all();
    }
    sv->cv.notify_all();
    return FCFS_OK;
}

int fcfs_serve_drain(void* h, int timeout_ms) {
    clear_error();
    Server* sv = (Server*)h;
    if (!sv) return fail(FCFS_ERR_ARG, "null handle");
    if (timeout_ms < 0) timeout_ms = sv->cfg.timeout_ms;
    std::unique_lock<std::mutex> lk(sv->mu);
    const bool ok = sv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                         [&] { return sv->error || sv->S->idle(); });
    if (sv->error) return fail(sv->error, "server error");
    if (!ok) return fail(FCFS_ERR_TIMEOUT, "%zu queued and %zu active requests after %d ms", sv->S->queued(),
                         sv->S->active(), timeout_ms);
    return FCFS_OK;
}

int fcfs_serve_stats(void* h, fcfs_serve_stats_t* out) {
    clear_error();
    Server* sv = (Server*)h;
    if (!sv || !out) return fail(FCFS_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    const auto& L = sv->S->latencies();
    out->submitted = sv->S->submitted();
    out->completed = sv->S->completed();
    out->canceled = sv->S->canceled();
    out->deferred = sv->S->deferred();
    out->rejected = sv->rejected;
    out->steps = sv->steps_launched;
    out->max_inflight_seen = sv->S->max_inflight_seen();
    out->p50_ms = sched::Scheduler::percentile(L, 50) * 1e3;
    out->p90_ms = sched::Scheduler::percentile(L, 90) * 1e3;
    out->p99_ms = sched::Scheduler::percentile(L, 99) * 1e3;
    double sum = 0;
    for (double v : L) sum += v;
    out->mean_ms = L.empty() ? 0 : sum / L.size() * 1e3;
    out->out_pixels = sv->S->out_pixels();
    out->bytes_moved = sv->S->bytes();
    out->wall_s = (sv->first_arrival >= 0 && sv->last_done >= 0) ? sv->last_done - sv->first_arrival : 0;
    out->gpix_s = out->wall_s > 0 ? out->out_pixels / out->wall_s / 1e9 : 0;
    out->gbytes_s = out->wall_s > 0 ? out->bytes_moved / out->wall_s / 1e9 : 0;
    return FCFS_OK;
}

int fcfs_serve_destroy(void* h) {
    clear_error();
    Server* sv = (Server*)h;
    if (!sv) return fail(FCFS_ERR_ARG, "null handle");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    const cudaError_t e = cudaStreamSynchronize(sv->stream);
    if (sv->pool_base) cudaFree(sv->pool_base);
    if (sv->slots_dev) cudaFree(sv->slots_dev);
    if (sv->slots_host) cudaFreeHost(sv->slots_host);
    for (auto& R : sv->steps) {
        if (R.dev) cudaFree(R.dev);
        if (R.host) cudaFreeHost(R.host);
        if (R.ev) cudaEventDestroy(R.ev);
    }
    if (sv->own_stream) cudaStreamDestroy(sv->stream);
    delete sv->S;
    delete sv;
    return e == cudaSuccess ? FCFS_OK : cuda_fail(e, "serve stream synchronize");
}

}  // extern "C"
