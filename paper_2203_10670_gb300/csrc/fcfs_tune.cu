// Tile-shape autotuner: times a small candidate set of forward tile shapes
// for one (method, r, s, dtype, ndim) key on the caller's buffers and keeps
// the fastest in the process-wide plan cache that fcfs_forward consults.
#include <climits>
#include <vector>

#include "fcfs_host.h"

using namespace fcfs;

extern "C" int fcfs_tune_forward(const fcfs_desc* d, const void* x, void* y, void* stream, int reps, float* best_ms,
                                 int* n_candidates) {
    NvtxRange nv("fcfs_tune_forward");
    clear_error();
    int rc = validate_desc(d, true);
    if (rc) return rc;
    if (d->w2d) return fail(FCFS_ERR_UNSUPPORTED, "the tile search covers the separable kernels");
    if (reps < 1) reps = 3;
    if (best_ms) *best_ms = 0.f;
    if (n_candidates) *n_candidates = 0;
    if (numel_out(d) == 0) return FCFS_OK;
    if (!x || !y) return fail(FCFS_ERR_ARG, "x and y must be device pointers");
    bool all_nearest = true;
    for (int a = 0; a < d->ndim; ++a) all_nearest &= (d->axis[a].w == nullptr && d->axis[a].method == FCFS_NEAREST);
    if (all_nearest && !tma_eligible(d, x)) return FCFS_OK;  // the nearest gather kernel has no tile choice
    cudaStreamCaptureStatus cs;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(FCFS_ERR_ARG, "tuning cannot run during stream capture");

    FwdParams P0;
    int ntk;
    rc = build_forward_params(d, x, y, &P0, &ntk);
    if (rc) return rc;
    const bool is3d = d->ndim == 3;
    const bool tma = tma_eligible(d, x);
    std::vector<TileChoice> cands;
    TileChoice def = tma ? default_tma_tiles(P0, dtype_size(d->dtype_in), is3d) : default_tiles(P0, is3d);
    def.tma = tma ? 1 : 0;
    def.psk = 0;
    {
        // the polyphase strip kernel, when the descriptor is in its scope
        FwdParams P = P0;
        TileChoice s = def;
        s.psk = 1;
        if (psk_enabled() && psk_forward(d, P, st) == FCFS_OK) cands.push_back(s);
        clear_error();
    }
    cands.push_back(def);
    const int ox_targets[] = {64, 128, 192, 256};
    const int oy_targets[] = {8, 16, 32, 48, 64, 96, 128};
    const int ry = P0.ax[1].r;
    // 3D: depth windows per tile as well (half, same, double the default)
    const int wd_scale[] = {2, 4, 8};
    for (int oxt : ox_targets)
        for (int al = 0; al < 2; ++al)
        for (int oyt : oy_targets)
            for (int gm = 0; gm < 4; ++gm)
                for (int ws : wd_scale) {
                    if (!is3d && ws != 4) continue;
                    // al = 1: the width rounded down to a multiple of 8 outputs (16-byte BF16 stores)
                    int wx = std::max(1, oxt / P0.ax[2].r);
                    if (al) {
                        while (wx > 1 && (wx * P0.ax[2].r) % 8) --wx;
                        if ((wx * P0.ax[2].r) % 8 || wx == std::max(1, oxt / P0.ax[2].r)) continue;
                    }
                    TileChoice t{wx, std::max(1, oyt / ry), std::max(1, def.WD * ws / 4)};
                    t.tma = def.tma;
                    // TMA kernel: the second variant is the 512-thread CTA; gather kernel: thread groups
                    t.G = tma ? 0 : (gm == 0 ? def.G : (def.G == ry ? 1 : ry));
                    t.threads = tma ? ((gm & 1) == 0 ? 256 : 512) : 0;
                    t.rs = gm < 2 ? 1 : 0;
                    t.psk = 0;
                    if (!tma && gm >= 2) continue;
                    FwdParams P = P0;
                    apply_tiles(P, is3d, t.WX, t.WY, t.WD, t.G);
                    if (!tma && P.OX * P.G > 512) continue;
                    if (tma && is3d) {
                        if (t.threads > 256) continue;  // the volume kernels run 256-thread CTAs
                        TmaFwd3Params T;
                        if (prepare_tma3(d, P, &T, t.threads) != FCFS_OK || forward3_tma_smem_bytes(T) > 200 * 1024) {
                            clear_error();
                            continue;
                        }
                    } else if (tma) {
                        TmaFwdParams T;
                        if (prepare_tma(d, P, &T, t.threads) != FCFS_OK || forward_tma_smem_bytes(T) > 200 * 1024) {
                            clear_error();
                            continue;
                        }
                    } else if (forward_smem_bytes(P, is3d) > 200 * 1024) {
                        continue;
                    }
                    t.WX = P.WX;
                    t.WY = P.WY;
                    t.WD = P.WD;
                    t.G = tma ? 0 : P.G;
                    bool dup = false;
                    for (auto& c : cands)
                        dup |= (c.WX == t.WX && c.WY == t.WY && c.WD == t.WD && c.G == t.G && c.tma == t.tma &&
                                c.threads == t.threads && c.rs == t.rs);
                    if (!dup) cands.push_back(t);
                }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(FCFS_ERR_CUDA, "event create failed");
    float best = 1e30f;
    TileChoice pick = def;
    int tried = 0;
    for (auto& t : cands) {
        FwdParams P = P0;
        rc = launch_choice(d, P, ntk, t, st);  // warm-up
        if (rc) continue;
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps; ++k) {
            FwdParams Pk = P0;
            launch_choice(d, Pk, ntk, t, st);
        }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        ++tried;
        if (ms < best) {
            best = ms;
            pick = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tuning launches");
    if (tried == 0) return fail(FCFS_ERR_UNSUPPORTED, "no tile candidate launched");
    set_plan(P0, d->ndim, d->dtype_in, d->dtype_out, pick);
    if (best_ms) *best_ms = best;
    if (n_candidates) *n_candidates = tried;
    return FCFS_OK;
}

extern "C" void fcfs_clear_plans(void) { clear_plans(); }

extern "C" int fcfs_plan_count(void) { return plan_count(); }
