/*
 * libfcfs -- Fully Convolutional Fractional Scaling (FCFS) on GB300 (sm_103a).
 *
 * FCFS (Soloveitchik & Werman, arXiv 2203.10670) scales a signal by a rational
 * factor r/s in one layer: pad the input (Sec. 3), apply a convolution with
 * r output channels and stride s whose kernels are interpolation weights
 * (Sec. 3.1), then pixel-shuffle the r channels into one output axis.  In 2D
 * and 3D (Sec. 4) the convolution has prod(r_a) channels and a per-axis
 * stride, followed by an N-d pixelshuffle.  This library evaluates that layer
 * as one fused polyphase gather: the r-channel hidden layer of Sec. 3.1 is
 * never written to memory, the pixelshuffle is the store index.
 *
 * Conventions used by every entry point:
 *   - Geometry per spatial axis with input length N: output length
 *     No = floor(N r / s); output o = i r + j (window i, phase j) samples the
 *     input at p = o s / r (Sec. 3.1: phase j of window i interpolates at
 *     offset i + j/r in stride units).  A window of T = 2K+1 taps starts at
 *     input index i s - L with L = K - floor(s/2).
 *   - Tensors are contiguous row-major [n][c][spatial...], the last spatial
 *     axis fastest, in DEVICE memory owned by the caller.  Spatial axes are
 *     listed outermost first: (W), (H, W) or (D, H, W).
 *   - Weights W[j][m] multiply x~[i s - L + m] (cross-correlation order; the
 *     true convolution of Sec. 3 is the same kernel reversed).
 *   - Every call returns an fcfs_status; arguments are validated on the host
 *     before anything is enqueued, and nothing is enqueued on error.  Device
 *     work is asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *     stream); FCFS_OK means validated and enqueued.
 *   - The library never allocates device memory on the forward/backward path.
 */
#ifndef FCFS_H
#define FCFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FCFS_OK = 0,
    FCFS_ERR_ARG = -1,              /* malformed argument (shape, pointer, enum, size) */
    FCFS_ERR_KERNEL_TOO_SMALL = -2, /* K below K_min for a fixed method */
    FCFS_ERR_UNSUPPORTED = -3,      /* valid but not implemented combination */
    FCFS_ERR_CUDA = -4,             /* a CUDA runtime call failed */
    FCFS_ERR_NOMEM = -5,            /* workspace or serving budget too small */
    FCFS_ERR_TIMEOUT = -6,          /* a bounded wait ran out */
    FCFS_ERR_BUSY = -7              /* serving: no free slot right now */
} fcfs_status;

/* Interpolation methods of Sec. 5.2.  Bicubic is Keys' cubic convolution with
 * a = -0.5 (the printed kernel's "-4a" constant is +2). */
typedef enum { FCFS_NEAREST = 0, FCFS_BILINEAR = 1, FCFS_BICUBIC = 2 } fcfs_method;

/* Padding of Sec. 3: repetition of edge pixels, a constant c (zeros when
 * c = 0), and reflection about the edge sample (edge not repeated; any
 * distance by periodic mirroring with period 2(N-1)). */
typedef enum { FCFS_PAD_REPLICATE = 0, FCFS_PAD_CONSTANT = 1, FCFS_PAD_REFLECT = 2 } fcfs_pad;

/* Sample alignment of the fixed methods (learnable weights define their own
 * taps and ignore it):
 *   FCFS_ALIGN_PAPER       output o samples p = o s / r (Sec. 3.1: phase j of
 *                          window i at offset i + j/r in stride units); nearest
 *                          takes floor(p + 1/2) (Sec. 5.2.1 examples)
 *   FCFS_ALIGN_HALF_PIXEL  pixel centres: p = (o + 1/2) s / r - 1/2; nearest
 *                          takes floor((o + 1/2) s / r)
 *   FCFS_ALIGN_FLOOR       p = o s / r; nearest takes floor(p)
 * The last two are the conventions of common resize libraries, not the
 * paper's; every one of them is still a period-r polyphase operator. */
typedef enum { FCFS_ALIGN_PAPER = 0, FCFS_ALIGN_HALF_PIXEL = 1, FCFS_ALIGN_FLOOR = 2 } fcfs_align;

/* Element types.  FCFS_U8 is accepted as an input type (converted exactly to
 * FP32 at load).  Arithmetic is FP32 everywhere; BF16 is a storage format
 * only (rounded to nearest-even on store). */
typedef enum { FCFS_F32 = 0, FCFS_BF16 = 1, FCFS_U8 = 2 } fcfs_dtype;

#define FCFS_MAX_R 64      /* largest r per axis for the built-in method tables */
#define FCFS_MAX_TAPS 9    /* largest T = 2K+1 for learnable weights */

/*
 * Weight table of Sec. 5.2 (Sec. 3.1 "kernel_weights").  Writes the r x (2K+1)
 * FP32 table W[j][m] = k(j s / r - (m - L)) to HOST memory w_out (row j =
 * phase), where k is the bilinear hat or the Keys kernel; nearest is one-hot
 * at m = floor((2 j s + r) / (2 r)) + L (round half up, the rounding the
 * Sec. 5.2.1 examples show).  Computed in FP64, rounded once to FP32.
 * K = 0 selects K_min = ceil((s + 2R - 2) / 2) (R = 1 nearest/bilinear,
 * 2 bicubic); *K_out (may be NULL) receives the K used.  w_out may be NULL
 * to query K only.  Errors: FCFS_ERR_ARG (r, s < 1, r > FCFS_MAX_R, unknown
 * method), FCFS_ERR_KERNEL_TOO_SMALL (0 < K < K_min).
 */
int fcfs_make_weights(int method, int r, int s, int K, float* w_out, int* K_out);

/*
 * Geometry of one axis (Sec. 3.1.1 "Description"): for input length n_in,
 * *n_out = floor(n_in r / s), *n_windows = ceil(n_out / r), *left_offset = L.
 * K = 0 selects K_min for `method`.  Any output pointer may be NULL.
 */
int fcfs_geometry(int method, int r, int s, int K, long long n_in, long long* n_out,
                  long long* n_windows, int* left_offset);

/* One spatial axis of the layer. */
typedef struct {
    int r, s;          /* scale factor r/s, both >= 1 (need not be reduced) */
    int K;             /* window half width (T = 2K+1); 0 = K_min for `method` */
    int method;        /* fcfs_method, used when w == NULL */
    const float* w;    /* DEVICE learnable weights [C][r][T] (w_per_channel) or
                          [r][T]; NULL = the fixed table of `method` */
    int w_per_channel; /* 1: one table per channel (depthwise), 0: shared */
} fcfs_axis;

/* The whole layer: depthwise over channels, separable over spatial axes
 * (Sec. 4 with outer-product kernels). */
typedef struct {
    int ndim;                /* spatial dimensions, 1..3 */
    long long n, c;          /* batch and channels */
    long long in_shape[3];   /* spatial input extents, outermost first */
    long long out_shape[3];  /* must equal floor(in_shape * r / s) per axis */
    int dtype_in;            /* fcfs_dtype of x (F32, BF16, U8) */
    int dtype_out;           /* fcfs_dtype of y (F32, BF16) */
    int pad;                 /* fcfs_pad */
    float pad_value;         /* constant for FCFS_PAD_CONSTANT */
    int align;               /* fcfs_align of the fixed methods */
    fcfs_axis axis[3];       /* same order as in_shape */
    float cubic_a;           /* Keys parameter of the fixed bicubic: 0 selects the
                                paper's -0.5 (Sec. 5.2); -0.75 is another common choice */
    const float* w2d;        /* DEVICE non-separable 2D kernels, NULL for the separable
                                layer; see "Non-separable 2D kernels" below */
    int w2d_per_channel;     /* 1: w2d is [C][r_y][r_x][T_y][T_x], 0: [r_y][r_x][T_y][T_x] */
    int antialias;           /* 1: antialiased downscale of the fixed bilinear / bicubic
                                methods; see "Antialiased downscale" below.  0: the paper's kernels */
} fcfs_desc;

/*
 * Antialiased downscale (antialias = 1; not the paper's: its kernels keep their
 * width when s > r, so a downscale samples without a low-pass prefilter).  On
 * every axis with s > r and a fixed bilinear or bicubic method, output o with
 * sample position p (the axis's alignment) takes every input t with
 * |t - p| < R s / r (R = 1 bilinear, 2 bicubic) with weight k((t - p) r / s),
 * the weights divided by their sum, padding as for the plain layer.  It is the
 * prefilter of common resize libraries' antialias mode (their bicubic uses
 * a = -1/2, the paper's constant), still a period-r polyphase operator.  Axes
 * with s <= r, nearest and learnable axes are unchanged.  The widened window
 * may hold at most 9 taps per phase and r x taps <= 256 (bilinear down to
 * 1/4, bicubic down to 1/2); wider ones fail with FCFS_ERR_UNSUPPORTED.
 * fcfs_make_weights keeps the paper's table.
 */

/*
 * Non-separable 2D kernels (w2d != NULL): the 2D convolution of Sec. 4 with a
 * general T_y x T_x kernel per phase pair instead of the outer product of the
 * two axis kernels, so that learning can change the kernel's shape (Sec. 7):
 *   y[n,c, iy r_y + jy, ix r_x + jx] = sum_{my,mx} w2d[c][jy][jx][my][mx]
 *                                      x~[n,c, iy s_y - L_y + my, ix s_x - L_x + mx]
 * Requires ndim == 2 and axis[a].w == NULL; axis[a] gives r, s and K (0 = K_min
 * of axis[a].method), T_a = 2 K_a + 1 <= FCFS_MAX_TAPS, L_a = K_a - floor(s_a/2),
 * and r_y r_x T_y T_x <= 4096.  align and cubic_a do not apply.  fcfs_forward
 * and fcfs_backward take such descriptors (fcfs_backward writes the gradient
 * of w2d, shaped like w2d, to gw[0] and needs gw[1] == NULL); the serving API
 * and fcfs_tune_forward reject them with FCFS_ERR_UNSUPPORTED.
 */

/*
 * Forward FCFS (Sec. 3.1 pseudocode; Sec. 4 for 2D/3D):
 *   y[n,c,o] = sum_m prod_a W_a[c][j_a][m_a] x~[n,c, i_a s_a - L_a + m_a]
 * with o_a = i_a r_a + j_a.  x: DEVICE [n][c][in_shape...] of dtype_in;
 * y: DEVICE [n][c][out_shape...] of dtype_out, fully overwritten.  x and y
 * must not overlap.  Nearest on every axis is an exact copy (bit-exact).
 * Errors: FCFS_ERR_ARG, FCFS_ERR_KERNEL_TOO_SMALL, FCFS_ERR_UNSUPPORTED,
 * FCFS_ERR_CUDA (launch failure).  Empty outputs enqueue nothing.
 */
int fcfs_forward(const fcfs_desc* d, const void* x, void* y, void* stream);

/* Activation of the fused epilogue. */
typedef enum { FCFS_ACT_NONE = 0, FCFS_ACT_RELU = 1, FCFS_ACT_LEAKY_RELU = 2, FCFS_ACT_CLAMP = 3 } fcfs_act;

/* The pointwise layer that follows FCFS in a fully convolutional network. */
typedef struct {
    int c_out;          /* output channels (>= 1) */
    const float* mix;   /* DEVICE [c_out][c] FP32 1x1 convolution, or NULL = identity (c_out == c) */
    const float* bias;  /* DEVICE [c_out] FP32, or NULL */
    int act;            /* fcfs_act */
    float alpha;        /* FCFS_ACT_LEAKY_RELU: slope for negative inputs */
    float lo, hi;       /* FCFS_ACT_CLAMP: bounds (lo <= hi) */
} fcfs_epilogue;

/*
 * FCFS fused with the layer after it (Sec. 1: the resize as one layer of an
 * FCN; Sec. 4 for 2D):
 *   y[n,o,p] = act(sum_c mix[o][c] FCFS(x)[n,c,p] + bias[o])
 * relu max(v, 0); leaky relu v >= 0 ? v : alpha v; clamp min(max(v, lo), hi).
 * The FCFS outputs of all c channels are combined on chip and never written.
 * d: a 2D separable descriptor (fixed or learnable axes, any pad / align;
 * w2d must be NULL; r_y r_x <= 512); x: DEVICE [n][c][H][W] of dtype_in;
 * y: DEVICE [n][c_out][Ho][Wo] of dtype_out, fully overwritten.  FP32
 * arithmetic.  Errors: as fcfs_forward, FCFS_ERR_ARG for a bad epilogue,
 * FCFS_ERR_UNSUPPORTED outside the 2D separable layer.  Gradients:
 * fcfs_backward_fused.
 */
int fcfs_forward_fused(const fcfs_desc* d, const fcfs_epilogue* e, const void* x, void* y, void* stream);

/*
 * Bytes of DEVICE workspace fcfs_backward_fused needs for descriptor d and
 * epilogue e (the recomputed FCFS outputs, the pre-activation gradient, the
 * partial sums of the mix gradient, and fcfs_backward's own workspace); 0 when
 * d or e is invalid (fcfs_last_error says why).
 */
size_t fcfs_backward_fused_workspace(const fcfs_desc* d, const fcfs_epilogue* e);

/*
 * Gradients of the fused layer (Sec. 1: the resize trained as one layer of
 * an FCN; the layer of fcfs_forward_fused).  With z = FCFS(x) and
 * v = mix z + bias recomputed in FP32 and gv = gy act'(v):
 *   gmix[o][c] = sum_{n,p} gv[n,o,p] z[n,c,p]   gbias[o] = sum_{n,p} gv[n,o,p]
 *   gz[n,c,p]  = sum_o mix[o][c] gv[n,o,p]      (gz = gv without a mix)
 * and gx, gw are the FCFS gradients for the upstream gradient gz (as
 * fcfs_backward).  act': relu 1 for v > 0 else 0; leaky relu 1 for v > 0
 * else alpha; clamp 1 for lo <= v <= hi else 0; none 1.
 * d, e: as for the forward (dtype_out is gy's type, FP32 or BF16; dtype_in
 * FP32 or BF16).  x: DEVICE input; gy: DEVICE [n][c_out][Ho][Wo]; gx: DEVICE
 * like x or NULL; gmix: DEVICE FP32 [c_out][c] or NULL (needs a mix); gbias:
 * DEVICE FP32 [c_out] or NULL (needs a bias); gw: as for fcfs_backward (or
 * NULL).  Every requested output is overwritten.  workspace: DEVICE, 256-byte
 * aligned, at least fcfs_backward_fused_workspace(d, e) bytes.  Results are
 * reproducible bit for bit (fixed summation orders).  Errors: as
 * fcfs_backward; FCFS_ERR_ARG for a bad epilogue, a missing or small
 * workspace, or a gradient of a term the layer does not have.
 */
int fcfs_backward_fused(const fcfs_desc* d, const fcfs_epilogue* e, const void* x, const void* gy, void* gx,
                        float* gmix, float* gbias, float* const* gw, void* workspace, size_t ws_bytes, void* stream);

/*
 * Bytes of device workspace fcfs_backward needs for the weight gradients
 * requested by the descriptor (0 when no axis has learnable weights).
 */
size_t fcfs_backward_workspace(const fcfs_desc* d);

/*
 * Backward of the forward map above (the learnable-weights remark of Sec. 7
 * needs both gradients):
 *   gx = adjoint of the polyphase map applied to gy, with the pad adjoint
 *        folded in (replicate sends every virtual index to the edge pixel,
 *        reflect to its mirror, constant drops them);
 *   gw[a][c][j][m] = sum over n and outputs of phase j on axis a of
 *        gy * x~ * (product of the other axes' weights).
 * x (DEVICE, dtype_in) is needed only for gw and may be NULL otherwise;
 * gy: DEVICE, dtype_out, shape of y; gx: DEVICE, dtype_in (F32 or BF16), shape
 * of x, fully overwritten, may be NULL; gw: array of ndim pointers (the array
 * itself may be NULL) to DEVICE FP32 buffers shaped like that axis's w,
 * overwritten; gw[a] must be NULL when axis a has no learnable weights.
 * workspace: DEVICE, at least fcfs_backward_workspace(d) bytes, 256-byte
 * aligned, caller-owned.  Partial sums are reduced in a fixed order, so
 * results are bitwise reproducible run to run.
 * Errors: as fcfs_forward, plus FCFS_ERR_NOMEM when ws_bytes is too small.
 */
int fcfs_backward(const fcfs_desc* d, const void* x, const void* gy, void* gx, float* const* gw,
                  void* workspace, size_t ws_bytes, void* stream);

/*
 * Tile-shape search for the planned forward (the plan/autotune step; the paper
 * has no counterpart: it chooses how the Sec. 3.1 / Sec. 4 layer is tiled on
 * the GPU, not what it computes).  Times the default tile and a candidate set
 * (output columns x rows per tile, CTA size, register-blocked or not; depth
 * windows for 3D) on the caller's x and y, reps launches each, synchronously,
 * and stores the fastest in a process-wide plan cache keyed by (ndim, r, s
 * per axis, taps, tap offsets, dtypes) that later fcfs_forward calls with the
 * same key use.  Every candidate computes the same result; y is overwritten.
 * reps < 1 selects 3.  *best_ms (may be NULL) receives the best time per call,
 * *n_candidates (may be NULL) the number timed.  Must not be called while
 * `stream` is being captured (FCFS_ERR_ARG).  Errors: as fcfs_forward;
 * FCFS_ERR_UNSUPPORTED for non-separable (w2d) descriptors.
 */
int fcfs_tune_forward(const fcfs_desc* d, const void* x, void* y, void* stream, int reps, float* best_ms,
                      int* n_candidates);

/* Forget every plan fcfs_tune_forward stored (later calls use the default tiles).
 * The on-disk cache (below) is left as it is and not read again in this process. */
void fcfs_clear_plans(void);

/*
 * Number of plans in the process-wide cache.  With the environment variable
 * FCFS_TUNE_CACHE naming a file, each plan fcfs_tune_forward chooses is
 * appended to that file (one text line: the device kind it was measured on,
 * the key, the tile), and the first plan lookup of a process loads the lines
 * of the same device kind, so tuned shapes keep their tiles across runs.
 */
int fcfs_plan_count(void);

/*
 * Status word written by the device code: 0 when every bounded wait of the
 * bulk-copy kernels completed, else a bit set (1 = a wait on a copy ran past
 * its iteration limit; the kernel finished without hanging but its output is
 * not trustworthy; 4 = an input-gradient tile broke the vector alignment its
 * plan assumed, output not trustworthy).  Synchronizes the device.  clear != 0
 * resets the word.
 * Returns the word, or FCFS_ERR_CUDA if it could not be read.
 */
int fcfs_device_status(int clear);

/*
 * fcfs_backward without a workspace argument, for callers that must not
 * allocate device memory: code hosted inside a framework or server that owns
 * every device allocation through its own pool, fixed-footprint deployments
 * that reserve all memory up front, and latency-critical loops that cannot
 * afford the synchronization an allocation call may cause.  The paper has no
 * counterpart; it is an interface convenience.
 *
 * Same arguments and results as fcfs_backward minus (workspace, ws_bytes):
 * the caller still provides x, gy, gx and the gw buffers.  The weight-gradient
 * partial sums go to a scratch area compiled into the library: 8 MiB of
 * device memory that every GPU loading libfcfs keeps until the process exits.
 * Descriptors whose weight gradient needs more than that (see
 * fcfs_backward_workspace) fail with FCFS_ERR_NOMEM before anything is
 * enqueued.  No device memory is allocated or freed by this call.
 *
 * The first call on each device performs a one-time set-up (it looks up the
 * device address of the scratch area); make that first call before any stream
 * capture.  All calls share the one scratch area, so calls whose work can
 * overlap on the GPU (different streams, or different host threads, without
 * ordering between them) race and give wrong weight gradients; serialize them.
 * Nothing in the area needs clearing between calls: every partial sum is
 * written before it is read.
 */
int fcfs_backward_noalloc(const fcfs_desc* d, const void* x, const void* gy, void* gx, float* const* gw,
                          void* stream);

/* ------------------------------------------------------------------------
 * Serving: a persistent request loop on one stream with continuous batching.
 * Requests (2D images, fixed methods, mixed sizes and factors) queue on the
 * host; a worker thread admits them while a parameter slot and pool memory
 * are free (admission by HBM footprint), and every loop step launches one
 * grouped kernel over tiles taken round-robin from all admitted requests, so
 * requests that arrive while others are on the GPU join the next step.  Each
 * tile is computed exactly as fcfs_forward computes it alone: results do not
 * depend on the mix.  The library allocates device memory here only, at
 * create: the output pool (hbm_budget_bytes), parameter slots and two
 * work-list buffers.
 * ---------------------------------------------------------------------- */
typedef struct {
    size_t hbm_budget_bytes;  /* pool for outputs the library places (y == NULL at submit) */
    int max_inflight;         /* requests admitted at once (1..4096) */
    int out_dtype;            /* FCFS_F32 or FCFS_BF16 for pooled outputs */
    int tile_budget_per_step; /* tiles per grouped launch; large requests are chunked */
    int timeout_ms;           /* default bound of fcfs_serve_drain when it is passed -1 */
    int auto_release;         /* 1: a pooled output is freed as soon as its request completes */
} fcfs_serve_config;

typedef struct {
    long long submitted, completed, deferred, rejected, steps;
    int max_inflight_seen;
    double p50_ms, p90_ms, p99_ms, mean_ms; /* completion host time - arrival time */
    double out_pixels;                      /* output pixels (channels of a pixel counted once) */
    double bytes_moved;                     /* algorithmic input + output bytes */
    double wall_s;                          /* first arrival to last completion */
    double gpix_s, gbytes_s;
    long long canceled;                     /* requests ended by fcfs_serve_cancel */
} fcfs_serve_stats_t;

/* Seconds on the steady clock the serving loop stamps latencies with. */
double fcfs_serve_clock(void);

/* Start a server on `stream` (NULL: the server creates its own).  Allocates
 * the pool and buffers (FCFS_ERR_NOMEM if the pool does not fit) and starts
 * the worker thread.  *handle receives the server. */
int fcfs_serve_create(const fcfs_serve_config* cfg, void* stream, void** handle);

/* Queue one request: d describes a 2D resize with fixed methods; x is DEVICE
 * input (F32, BF16 or U8), kept valid until the request completes; y is DEVICE
 * output or NULL to place it in the pool.  d->dtype_out must equal the
 * server's out_dtype in both cases (FCFS_ERR_ARG otherwise).  arrival_s (fcfs_serve_clock time) is the time latency
 * is measured from.  *req_id receives the id.  FCFS_ERR_NOMEM when the output
 * could never fit the pool; FCFS_ERR_ARG / FCFS_ERR_UNSUPPORTED for bad
 * descriptors. */
int fcfs_serve_submit(void* h, const fcfs_desc* d, const void* x, void* y, double arrival_s,
                      unsigned long long* req_id);

/* Queue `count` requests at once (the same rules as fcfs_serve_submit for each):
 * descs[k], xs[k], ys[k] (ys may be NULL: every output pooled), arrivals[k];
 * ids[k] (may be NULL) receives each id.  Requests are validated in order and
 * queued in one critical section; the first invalid one stops the batch: the
 * requests before it are queued (*n_submitted of them, may be NULL) and its
 * status is returned.  One call replaces a call per request for callers that
 * receive requests in groups. */
int fcfs_serve_submit_batch(void* h, int count, const fcfs_desc* descs, const void* const* xs, void* const* ys,
                            const double* arrivals, unsigned long long* ids, int* n_submitted);

/* Non-blocking: up to `max` ids of completed requests (each reported once).
 * Returns FCFS_OK, or the error that stopped the server. */
int fcfs_serve_poll(void* h, unsigned long long* done_ids, int max, int* n_done);

/* Device address of a completed request's pooled output (auto_release == 0). */
int fcfs_serve_result(void* h, unsigned long long id, void** y);

/* Return a completed request's pooled output to the pool (auto_release == 0). */
int fcfs_serve_release(void* h, unsigned long long id);

/* Cancel a request (a client that gives up on it).  Queued: it is removed at
 * once.  Running: no further tile of it is launched; it ends when its launched
 * tiles finish.  Either way its id is reported by fcfs_serve_poll like a
 * completion, its output is left incomplete (pooled memory returns to the
 * pool, fcfs_serve_result refuses it), and it is left out of the latency and
 * throughput figures (counted in fcfs_serve_stats_t.canceled).  FCFS_ERR_ARG
 * when the id is neither queued nor running. */
int fcfs_serve_cancel(void* h, unsigned long long id);

/* Wait until every queued request has completed, at most timeout_ms (-1: the
 * configured timeout); FCFS_ERR_TIMEOUT otherwise.  No GPU wait is unbounded. */
int fcfs_serve_drain(void* h, int timeout_ms);

/* Counters, latency percentiles and throughput since create. */
int fcfs_serve_stats(void* h, fcfs_serve_stats_t* out);

/* Stop the worker, wait for the stream, free everything. */
int fcfs_serve_destroy(void* h);

/* Static text for a status code. */
const char* fcfs_status_string(int status);

/* Detail text of the last error returned on the calling thread ("" if none). */
const char* fcfs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FCFS_H */
