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
#include "fcfs_host.h"
#include "fcfs_sched.h"

namespace fcfs {
namespace {

constexpr int kServeThreads = 256;
constexpr int kServeMaxSmem = 64 * 1024;

// Device parameter slot of one admitted request.
struct ServeSlot {
    FwdParams P;
    int din;  // fcfs_dtype of x
    int nt;   // tap template (1 nearest, 2 bilinear, 4 bicubic)
};

struct WorkItem {
    int slot;
    int tile;
};

template <typename Tin, typename Tout>
__device__ __forceinline__ void serve_tile(const FwdParams& P, int nt, long long tile, float* smem) {
    if (nt == 1) fwd2d_tile<1, Tin, Tout>(P, tile, smem);
    else if (nt == 2) fwd2d_tile<2, Tin, Tout>(P, tile, smem);
    else fwd2d_tile<4, Tin, Tout>(P, tile, smem);
}

// K6: one CTA per work item; the item names the request slot and its tile.
template <typename Tout>
__global__ void __launch_bounds__(kServeThreads) fcfs_serve_grouped(const ServeSlot* __restrict__ slots,
                                                                     const WorkItem* __restrict__ work) {
    extern __shared__ float smem[];
    const WorkItem w = work[blockIdx.x];
    const ServeSlot& S = slots[w.slot];
    if (S.din == FCFS_U8) serve_tile<uint8_t, Tout>(S.P, S.nt, w.tile, smem);
    else if (S.din == FCFS_F32) serve_tile<float, Tout>(S.P, S.nt, w.tile, smem);
    else serve_tile<__nv_bfloat16, Tout>(S.P, S.nt, w.tile, smem);
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
    StepRec steps[2];
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
    if (sv.cfg.out_dtype == FCFS_BF16)
        fcfs_serve_grouped<__nv_bfloat16><<<(unsigned)n, kServeThreads, kServeMaxSmem, sv.stream>>>(sv.slots_dev, R.dev);
    else
        fcfs_serve_grouped<float><<<(unsigned)n, kServeThreads, kServeMaxSmem, sv.stream>>>(sv.slots_dev, R.dev);
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
                sv->step_next ^= 1;
                progressed = true;
            }
        }
        if (!progressed) {
            const bool busy = sv->steps[0].busy || sv->steps[1].busy;
            // GPU busy: poll again soon; idle: sleep until a submission arrives
            sv->cv.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(5));
        }
    }
}

// Tile plan for serving: 256-thread CTAs, about 128 output columns, shared
// memory within the grouped kernel's budget.
void plan_serve_tiles(FwdParams& P) {
    int WX = std::max(1, 128 / P.ax[2].r), WY = std::max(1, 32 / P.ax[1].r);
    for (int it = 0; it < 64; ++it) {
        apply_tiles(P, false, WX, WY, 1, 0);
        const int G = std::max(1, kServeThreads / P.OX);
        P.G = G;
        if (P.OX <= kServeThreads && forward_smem_bytes(P, false) <= (size_t)kServeMaxSmem) return;
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
