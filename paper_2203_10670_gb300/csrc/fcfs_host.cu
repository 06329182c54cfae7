// libfcfs host side: the C ABI entry points, argument validation, the weight
// and geometry tables of Sec. 3.1 / Sec. 5.2, and the tile planner.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <climits>
#include <mutex>
#include <string>
#include <unordered_map>

#include "fcfs_host.h"

namespace fcfs {

static thread_local std::string g_last_error;

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

void clear_error() { g_last_error.clear(); }

int cuda_fail(cudaError_t e, const char* what) {
    return fail(FCFS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Interpolation kernels of Sec. 5.2 evaluated in FP64: the bilinear hat and
// Keys' cubic convolution kernel with a = -1/2.
double kernel_value(int method, double t, double ka) {
    const double a = fabs(t);
    if (method == FCFS_BILINEAR) return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 1.0) return ((ka + 2.0) * a - (ka + 3.0)) * a * a + 1.0;
    if (a < 2.0) return ((ka * a - 5.0 * ka) * a + 8.0 * ka) * a - 4.0 * ka;
    return 0.0;
}

int support_radius(int method) { return method == FCFS_BICUBIC ? 2 : 1; }

// Keys parameter of a descriptor: 0 selects the paper's -0.5
double keys_a(const fcfs_desc* d) { return d->cubic_a != 0.f ? (double)d->cubic_a : -0.5; }

int k_min(int method, int s) { return (s + 2 * support_radius(method) - 2 + 1) / 2; }

static long long floor_div(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

long long out_len(long long n, int r, int s) { return floor_div(n * (long long)r, s); }

// Smallest kernel template width that holds nt taps.
int template_taps(int nt) {
    static const int widths[] = {1, 2, 3, 4, 5, 7, 9};
    for (int w : widths)
        if (w >= nt) return w;
    return -1;
}

// Fixed-method phase table in compact form: for phase j the taps sit at
// i*s + first_j + t relative to window i.  Phase j samples the rational
// position num/den past i*s: j s / r (paper and floor alignment) or
// (2 j s + s - r) / (2 r) (half-pixel centres); the kernel is evaluated at
// (num - q den) / den for tap q.  Nearest rounds the paper's position half up,
// the floor alignment's down, and takes floor((2 j s + s) / (2 r)) for
// half-pixel centres.
//
// Antialiased downscale (aa and s > r): the kernel is stretched by s / r: tap
// q counts when |q den - num| r < R s den (exact integers), with weight
// k((q - p) r / s), and the phase's weights are divided by their sum.
static void fixed_phase(int method, int r, int s, int j, int align, double ka, int aa, int* first, double* w,
                        int* nt) {
    if (method == FCFS_NEAREST) {
        const long long js = (long long)j * s;
        if (align == FCFS_ALIGN_FLOOR) *first = (int)(js / r);
        else if (align == FCFS_ALIGN_HALF_PIXEL) *first = (int)((2 * js + s) / (2LL * r));
        else *first = (int)((2 * js + r) / (2LL * r));
        w[0] = 1.0;
        *nt = 1;
        return;
    }
    long long num = (long long)j * s, den = r;
    if (align == FCFS_ALIGN_HALF_PIXEL) {
        num = 2LL * j * s + s - r;
        den = 2LL * r;
    }
    const long long b = floor_div(num, den);
    const int R = support_radius(method);
    if (aa && s > r) {
        const long long reach = (long long)R * ((s + r - 1) / r) + 1;
        int n = 0;
        double sum = 0.0;
        *first = 0;
        for (long long q = b - reach; q <= b + reach; ++q) {
            const long long dq = q * den - num;
            if ((dq < 0 ? -dq : dq) * (long long)r >= (long long)R * s * den) continue;
            if (n == 0) *first = (int)q;
            if (n < kMaxAATaps) w[n] = kernel_value(method, (double)(dq * r) / (double)(den * s), ka);
            sum += n < kMaxAATaps ? w[n] : 0.0;
            ++n;
        }
        *nt = n;
        for (int t = 0; t < std::min(n, kMaxAATaps); ++t) w[t] /= sum;
        return;
    }
    *first = (int)(b - R + 1);
    *nt = 2 * R;
    for (int t = 0; t < 2 * R; ++t) {
        const long long q = b - R + 1 + t;
        w[t] = kernel_value(method, (double)(num - q * den) / (double)den, ka);
    }
}

int validate_axis(const fcfs_axis& a, int idx) {
    if (a.r < 1 || a.s < 1) return fail(FCFS_ERR_ARG, "axis %d: r and s must be >= 1 (got %d/%d)", idx, a.r, a.s);
    if (a.method < FCFS_NEAREST || a.method > FCFS_BICUBIC) return fail(FCFS_ERR_ARG, "axis %d: unknown method %d", idx, a.method);
    if (a.K < 0) return fail(FCFS_ERR_ARG, "axis %d: K must be >= 0", idx);
    if (a.w == nullptr) {
        if (a.r > kMaxR) return fail(FCFS_ERR_ARG, "axis %d: r=%d exceeds FCFS_MAX_R=%d", idx, a.r, kMaxR);
        if (a.K != 0 && a.K < k_min(a.method, a.s))
            return fail(FCFS_ERR_KERNEL_TOO_SMALL, "axis %d: K=%d below K_min=%d", idx, a.K, k_min(a.method, a.s));
    } else {
        const int T = 2 * (a.K ? a.K : k_min(a.method, a.s)) + 1;
        if (T > FCFS_MAX_TAPS) return fail(FCFS_ERR_UNSUPPORTED, "axis %d: %d learnable taps exceed FCFS_MAX_TAPS", idx, T);
        if (((uintptr_t)a.w) % 4) return fail(FCFS_ERR_ARG, "axis %d: weight pointer not 4-byte aligned", idx);
        if (a.w_per_channel != 0 && a.w_per_channel != 1) return fail(FCFS_ERR_ARG, "axis %d: w_per_channel must be 0 or 1", idx);
    }
    return FCFS_OK;
}

int validate_desc(const fcfs_desc* d, bool output_dtype_check) {
    if (!d) return fail(FCFS_ERR_ARG, "descriptor is NULL");
    if (d->ndim < 1 || d->ndim > 3) return fail(FCFS_ERR_ARG, "ndim must be 1..3 (got %d)", d->ndim);
    if (d->n < 0 || d->c < 0) return fail(FCFS_ERR_ARG, "n and c must be >= 0");
    if (d->dtype_in != FCFS_F32 && d->dtype_in != FCFS_BF16 && d->dtype_in != FCFS_U8)
        return fail(FCFS_ERR_ARG, "unknown dtype_in %d", d->dtype_in);
    if (output_dtype_check && d->dtype_out != FCFS_F32 && d->dtype_out != FCFS_BF16)
        return fail(FCFS_ERR_ARG, "dtype_out must be F32 or BF16 (got %d)", d->dtype_out);
    if (d->pad < FCFS_PAD_REPLICATE || d->pad > FCFS_PAD_REFLECT) return fail(FCFS_ERR_ARG, "unknown pad mode %d", d->pad);
    if (d->align < FCFS_ALIGN_PAPER || d->align > FCFS_ALIGN_FLOOR) return fail(FCFS_ERR_ARG, "unknown alignment %d", d->align);
    if (!std::isfinite(d->cubic_a)) return fail(FCFS_ERR_ARG, "cubic_a must be finite");
    if (d->antialias != 0 && d->antialias != 1) return fail(FCFS_ERR_ARG, "antialias must be 0 or 1");
    if (d->c > INT_MAX) return fail(FCFS_ERR_ARG, "c too large");
    if (d->w2d) {
        if (d->ndim != 2) return fail(FCFS_ERR_ARG, "non-separable kernels (w2d) need ndim == 2 (got %d)", d->ndim);
        if (d->w2d_per_channel != 0 && d->w2d_per_channel != 1)
            return fail(FCFS_ERR_ARG, "w2d_per_channel must be 0 or 1");
    }
    for (int a = 0; a < d->ndim; ++a) {
        fcfs_axis ax = d->axis[a];
        if (d->w2d) {
            // the axis gives r, s and K of the non-separable kernel, checked like learnable weights
            if (ax.w) return fail(FCFS_ERR_ARG, "axis %d: per-axis weights and w2d are exclusive", a);
            ax.w = d->w2d;
            ax.w_per_channel = d->w2d_per_channel;
        }
        int rc = validate_axis(ax, a);
        if (rc) return rc;
        if (d->antialias && !ax.w && !d->w2d && ax.method != FCFS_NEAREST && ax.s > ax.r) {
            const int nt = fixed_taps(ax.method, ax.r, ax.s, d->align, keys_a(d), 1);
            if (nt > FCFS_MAX_TAPS || ax.r * nt > kMaxR * kMaxFixedTaps)
                return fail(FCFS_ERR_UNSUPPORTED, "axis %d: antialiased %d/%d needs %d taps per phase (at most %d)", a,
                            ax.r, ax.s, nt, FCFS_MAX_TAPS);
        }
        if (d->in_shape[a] < 0 || d->in_shape[a] > INT_MAX / 2)
            return fail(FCFS_ERR_ARG, "axis %d: input extent %lld out of range", a, d->in_shape[a]);
        const long long no = out_len(d->in_shape[a], d->axis[a].r, d->axis[a].s);
        if (d->out_shape[a] != no)
            return fail(FCFS_ERR_ARG, "axis %d: out_shape %lld != floor(%lld*%d/%d) = %lld", a, d->out_shape[a],
                        d->in_shape[a], d->axis[a].r, d->axis[a].s, no);
        if (no > INT_MAX / 2) return fail(FCFS_ERR_ARG, "axis %d: output extent too large", a);
    }
    return FCFS_OK;
}

long long numel_in(const fcfs_desc* d) {
    long long v = d->n * d->c;
    for (int a = 0; a < d->ndim; ++a) v *= d->in_shape[a];
    return v;
}

long long numel_out(const fcfs_desc* d) {
    long long v = d->n * d->c;
    for (int a = 0; a < d->ndim; ++a) v *= d->out_shape[a];
    return v;
}

int dtype_size(int dt) { return dt == FCFS_F32 ? 4 : dt == FCFS_BF16 ? 2 : 1; }

// Fill the compact polyphase form of one real axis; nt_kernel is the
// template width every phase is evaluated with (zero-padded taps).
void fill_axis(AxisP* A, const fcfs_axis& a, long long n_in, int C, int nt_kernel, int align, double ka, int aa) {
    memset(A, 0, sizeof(*A));
    A->r = a.r;
    A->s = a.s;
    A->n_in = (int)n_in;
    A->n_out = (int)out_len(n_in, a.r, a.s);
    A->n_win = (int)((A->n_out + a.r - 1) / a.r);
    A->nt = nt_kernel;
    if (a.w) {
        const int K = a.K ? a.K : k_min(a.method, a.s);
        A->learn = 1;
        A->w = a.w;
        A->nt_src = 2 * K + 1;
        A->w_cstride = a.w_per_channel ? (long long)a.r * A->nt_src : 0;
        A->lo = -(K - a.s / 2);
        A->span = nt_kernel;
        (void)C;
        return;
    }
    // phases may differ in tap count (antialias): every phase takes the largest, zero-padded
    int first[kMaxR], cnt[kMaxR];
    double w[kMaxR][kMaxAATaps];
    int lo = INT_MAX, nt = 1;
    for (int j = 0; j < a.r; ++j) {
        fixed_phase(a.method, a.r, a.s, j, align, ka, aa, &first[j], w[j], &cnt[j]);
        lo = std::min(lo, first[j]);
        nt = std::max(nt, cnt[j]);
    }
    for (int j = 0; j < a.r; ++j)
        for (int t = 0; t < nt; ++t) A->wf[j * nt + t] = t < cnt[j] ? (float)w[j][t] : 0.f;
    int span = 0;
    for (int j = 0; j < a.r; ++j) {
        A->off[j] = (short)(first[j] - lo);
        span = std::max(span, first[j] - lo + nt_kernel);
    }
    A->nt_src = nt;
    A->lo = lo;
    A->span = span;
}

// Taps per phase of the fixed table of an axis (the widest phase when antialiased).
int fixed_taps(int method, int r, int s, int align, double ka, int aa) {
    if (method == FCFS_NEAREST) return 1;
    if (!(aa && s > r)) return 2 * support_radius(method);
    int nt = 1;
    for (int j = 0; j < r; ++j) {
        int first, n;
        double w[kMaxAATaps];
        fixed_phase(method, r, s, j, align, ka, aa, &first, w, &n);
        nt = std::max(nt, n);
    }
    return nt;
}

int axis_taps(const fcfs_desc* d, int a) {
    const fcfs_axis& ax = d->axis[a];
    if (ax.w) return 2 * (ax.K ? ax.K : k_min(ax.method, ax.s)) + 1;
    return fixed_taps(ax.method, ax.r, ax.s, d->align, keys_a(d), d->w2d ? 0 : d->antialias);
}

void identity_axis(AxisP* A, int nt_kernel) {
    memset(A, 0, sizeof(*A));
    A->r = A->s = 1;
    A->n_in = A->n_out = A->n_win = 1;
    A->nt = nt_kernel;
    A->nt_src = 1;
    A->wf[0] = 1.f;
    A->span = nt_kernel;
}

// ----------------------------------------------------------- tile planning

struct PlanKey {
    int ndim, r[3], s[3], nt, din, dout, lo[3], span[3];
    bool operator==(const PlanKey& o) const { return memcmp(this, &o, sizeof(PlanKey)) == 0; }
};
struct PlanKeyHash {
    size_t operator()(const PlanKey& k) const {
        size_t h = 1469598103934665603ull;
        const unsigned char* p = (const unsigned char*)&k;
        for (size_t i = 0; i < sizeof(k); ++i) h = (h ^ p[i]) * 1099511628211ull;
        return h;
    }
};
static std::mutex g_plan_mu;
static std::unordered_map<PlanKey, TileChoice, PlanKeyHash> g_plans;

// On-disk plan cache.  When FCFS_TUNE_CACHE names a file, every plan
// fcfs_tune_forward chooses is appended to it as one text line
//   fcfs-plan <device> <16 key integers> <8 tile integers>
// and the first plan lookup of a process loads the lines measured on the same
// kind of device (name, SM count and compute capability folded into <device>),
// so a tuned shape keeps its tiles across processes without timing again.
static std::once_flag g_cache_once;

static unsigned long long device_signature() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return 0;
    unsigned long long h = 1469598103934665603ull;
    for (const char* c = prop.name; *c; ++c) h = (h ^ (unsigned char)*c) * 1099511628211ull;
    h = (h ^ (unsigned long long)prop.multiProcessorCount) * 1099511628211ull;
    h = (h ^ (unsigned long long)(prop.major * 100 + prop.minor)) * 1099511628211ull;
    return h;
}

static void key_ints(const PlanKey& k, int* v) {
    int n = 0;
    v[n++] = k.ndim;
    for (int a = 0; a < 3; ++a) v[n++] = k.r[a];
    for (int a = 0; a < 3; ++a) v[n++] = k.s[a];
    v[n++] = k.nt;
    v[n++] = k.din;
    v[n++] = k.dout;
    for (int a = 0; a < 3; ++a) v[n++] = k.lo[a];
    for (int a = 0; a < 3; ++a) v[n++] = k.span[a];
}

static void load_plan_cache() {
    const char* path = getenv("FCFS_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    const unsigned long long sig = device_signature();
    char line[512];
    while (fgets(line, sizeof line, f)) {
        unsigned long long dsig = 0;
        int v[24], used = 0;
        if (sscanf(line, "fcfs-plan %llu%n", &dsig, &used) != 1 || dsig != sig) continue;
        const char* q = line + used;
        int n = 0;
        while (n < 24) {
            int k = 0;
            if (sscanf(q, "%d%n", &v[n], &k) != 1) break;
            q += k;
            ++n;
        }
        if (n != 24) continue;
        PlanKey key;
        memset(&key, 0, sizeof key);
        int i = 0;
        key.ndim = v[i++];
        for (int a = 0; a < 3; ++a) key.r[a] = v[i++];
        for (int a = 0; a < 3; ++a) key.s[a] = v[i++];
        key.nt = v[i++];
        key.din = v[i++];
        key.dout = v[i++];
        for (int a = 0; a < 3; ++a) key.lo[a] = v[i++];
        for (int a = 0; a < 3; ++a) key.span[a] = v[i++];
        TileChoice t{v[16], v[17], v[18]};
        t.G = v[19];
        t.tma = v[20];
        t.threads = v[21];
        t.rs = v[22];
        t.psk = v[23];
        g_plans[key] = t;
    }
    fclose(f);
}

static void save_plan(const PlanKey& k, const TileChoice& t) {
    const char* path = getenv("FCFS_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    int v[16];
    key_ints(k, v);
    fprintf(f, "fcfs-plan %llu", device_signature());
    for (int i = 0; i < 16; ++i) fprintf(f, " %d", v[i]);
    fprintf(f, " %d %d %d %d %d %d %d %d\n", t.WX, t.WY, t.WD, t.G, t.tma, t.threads, t.rs, t.psk);
    fclose(f);
}

static PlanKey plan_key(const FwdParams& P, int ndim, int din, int dout) {
    PlanKey k;
    memset(&k, 0, sizeof k);
    k.ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        k.r[a] = P.ax[a].r;
        k.s[a] = P.ax[a].s;
    }
    k.nt = P.ax[2].nt;
    k.din = din;
    k.dout = dout;
    for (int a = 0; a < 3; ++a) k.lo[a] = P.ax[a].lo, k.span[a] = P.ax[a].span;  // alignment moves the taps
    return k;
}

void set_plan(const FwdParams& P, int ndim, int din, int dout, TileChoice t) {
    std::call_once(g_cache_once, [] {
        std::lock_guard<std::mutex> g(g_plan_mu);
        load_plan_cache();
    });
    std::lock_guard<std::mutex> g(g_plan_mu);
    const PlanKey k = plan_key(P, ndim, din, dout);
    g_plans[k] = t;
    save_plan(k, t);
}

void clear_plans() {
    std::call_once(g_cache_once, [] {});  // a cleared cache is not reloaded from the file
    std::lock_guard<std::mutex> g(g_plan_mu);
    g_plans.clear();
}

int plan_count() {
    std::call_once(g_cache_once, [] {
        std::lock_guard<std::mutex> g(g_plan_mu);
        load_plan_cache();
    });
    std::lock_guard<std::mutex> g(g_plan_mu);
    return (int)g_plans.size();
}

bool get_plan(const FwdParams& P, int ndim, int din, int dout, TileChoice* t) {
    std::call_once(g_cache_once, [] {
        std::lock_guard<std::mutex> g(g_plan_mu);
        load_plan_cache();
    });
    std::lock_guard<std::mutex> g(g_plan_mu);
    auto it = g_plans.find(plan_key(P, ndim, din, dout));
    if (it == g_plans.end()) return false;
    *t = it->second;
    return true;
}

// Derive the tile sizes of P from a choice of windows per tile.
void apply_tiles(FwdParams& P, bool is3d, int WX, int WY, int WD, int Gforce) {
    const AxisP &AX = P.ax[2], &AY = P.ax[1], &AD = P.ax[0];
    WX = std::max(1, std::min(WX, AX.n_win));
    WY = std::max(1, std::min(WY, AY.n_win));
    P.WX = WX;
    P.WY = WY;
    P.OX = WX * AX.r;
    P.OY = WY * AY.r;
    P.IC = (WX - 1) * AX.s + AX.span;
    P.ICp = P.IC;
    P.IR = (WY - 1) * AY.s + AY.span;
    int G = Gforce > 0 ? Gforce : std::max(1, (256 + P.OX / 2) / P.OX);
    while (P.OX * G > 512 && G > 1) --G;
    P.G = G;
    P.tiles_x = (AX.n_win + WX - 1) / WX;
    P.tiles_y = (AY.n_win + WY - 1) / WY;
    if (is3d) {
        WD = std::max(1, std::min(WD, AD.n_win));
        P.WD = WD;
        P.tiles_d = (AD.n_win + WD - 1) / WD;
        P.ring = AD.span;
    } else {
        P.WD = 1;
        P.tiles_d = 1;
        P.ring = 0;
    }
}

// Heuristic tile: about 128 output columns, as many rows as fit the
// shared-memory budget (several CTAs per SM), depth chunks for enough CTAs.
TileChoice default_tiles(const FwdParams& P0, bool is3d) {
    FwdParams P = P0;
    const AxisP &AX = P.ax[2], &AY = P.ax[1], &AD = P.ax[0];
    int WX = std::max(1, 128 / AX.r);
    int WY = std::max(1, (is3d ? 24 : 48) / AY.r);
    const size_t budget = 60 * 1024;
    for (int it = 0; it < 64; ++it) {
        apply_tiles(P, is3d, WX, WY, 1);
        if (forward_smem_bytes(P, is3d) <= budget) break;
        if (WY > 1 && (P.IR >= P.IC / 2 || WX == 1)) WY = (WY + 1) / 2;
        else if (WX > 1) WX = (WX + 1) / 2;
        else break;
    }
    int WD = 1;
    if (is3d) {
        const long long base = (long long)P.tiles_x * P.tiles_y * P.planes;
        const long long want = 152LL * 6;
        const long long chunks = std::max(1LL, (want + base - 1) / base);
        WD = (int)std::max(1LL, (AD.n_win + chunks - 1) / chunks);
    }
    return TileChoice{WX, WY, WD};
}

}  // namespace fcfs

using namespace fcfs;

extern "C" {

const char* fcfs_status_string(int status) {
    switch (status) {
        case FCFS_OK: return "ok";
        case FCFS_ERR_ARG: return "invalid argument";
        case FCFS_ERR_KERNEL_TOO_SMALL: return "kernel half width K below K_min";
        case FCFS_ERR_UNSUPPORTED: return "unsupported combination";
        case FCFS_ERR_CUDA: return "CUDA error";
        case FCFS_ERR_NOMEM: return "insufficient memory or workspace";
        case FCFS_ERR_TIMEOUT: return "timed out";
        case FCFS_ERR_BUSY: return "busy";
        default: return "unknown status";
    }
}

const char* fcfs_last_error(void) { return g_last_error.c_str(); }

int fcfs_device_status(int clear) {
    clear_error();
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "device synchronize");
    const int v = read_status_fwd_tma(clear), w = read_status_bwd_tma(clear), u = read_status_fused_tc(clear);
    const int p = read_status_psk(clear), q = read_status_psk_bf16(clear);
    if (v < 0 || w < 0 || u < 0 || p < 0 || q < 0) return fail(FCFS_ERR_CUDA, "reading the device status word failed");
    return v | w | u | p | q;
}

int fcfs_make_weights(int method, int r, int s, int K, float* w_out, int* K_out) {
    clear_error();
    if (r < 1 || s < 1 || r > kMaxR) return fail(FCFS_ERR_ARG, "r, s must be >= 1 and r <= %d", kMaxR);
    if (method < FCFS_NEAREST || method > FCFS_BICUBIC) return fail(FCFS_ERR_ARG, "unknown method %d", method);
    const int km = k_min(method, s);
    if (K < 0) return fail(FCFS_ERR_ARG, "K must be >= 0");
    if (K == 0) K = km;
    if (K < km) return fail(FCFS_ERR_KERNEL_TOO_SMALL, "K=%d below K_min=%d", K, km);
    if (K_out) *K_out = K;
    if (!w_out) return FCFS_OK;
    const int T = 2 * K + 1, L = K - s / 2;
    for (int j = 0; j < r; ++j) {
        int first, nt;
        double w[kMaxAATaps];
        fixed_phase(method, r, s, j, FCFS_ALIGN_PAPER, -0.5, 0, &first, w, &nt);
        for (int m = 0; m < T; ++m) w_out[j * T + m] = 0.f;
        for (int t = 0; t < nt; ++t) {
            const int m = first + t + L;  // tap offset first+t from i*s, window origin i*s - L
            if (m >= 0 && m < T) w_out[j * T + m] = (float)w[t];
        }
    }
    return FCFS_OK;
}

int fcfs_geometry(int method, int r, int s, int K, long long n_in, long long* n_out, long long* n_windows,
                  int* left_offset) {
    clear_error();
    if (r < 1 || s < 1) return fail(FCFS_ERR_ARG, "r and s must be >= 1");
    if (method < FCFS_NEAREST || method > FCFS_BICUBIC) return fail(FCFS_ERR_ARG, "unknown method %d", method);
    if (n_in < 0) return fail(FCFS_ERR_ARG, "n_in must be >= 0");
    if (K == 0) K = k_min(method, s);
    const long long no = out_len(n_in, r, s);
    if (n_out) *n_out = no;
    if (n_windows) *n_windows = (no + r - 1) / r;
    if (left_offset) *left_offset = K - s / 2;
    return FCFS_OK;
}

int fcfs_forward(const fcfs_desc* d, const void* x, void* y, void* stream) {
    NvtxRange nv("fcfs_forward");
    clear_error();
    int rc = validate_desc(d, true);
    if (rc) return rc;
    if (numel_out(d) == 0) return FCFS_OK;
    if (!x || !y) return fail(FCFS_ERR_ARG, "x and y must be device pointers");
    if (((uintptr_t)x) % dtype_size(d->dtype_in) || ((uintptr_t)y) % dtype_size(d->dtype_out))
        return fail(FCFS_ERR_ARG, "x or y not aligned to its element size");
    cudaStream_t st = (cudaStream_t)stream;
    if (d->w2d) return full2d_forward(d, x, y, st);

    bool all_nearest = true;
    for (int a = 0; a < d->ndim; ++a) all_nearest &= (d->axis[a].w == nullptr && d->axis[a].method == FCFS_NEAREST);
    if (all_nearest && !(d->ndim <= 2 && tma_eligible(d, x))) {
        NearestParams P;
        memset(&P, 0, sizeof P);
        const int lead = 3 - d->ndim;
        for (int a = 0; a < 3; ++a) {
            if (a < lead) {
                P.r[a] = P.s[a] = P.n_in[a] = P.n_out[a] = 1;
            } else {
                P.r[a] = d->axis[a - lead].r;
                P.s[a] = d->axis[a - lead].s;
                P.n_in[a] = (int)d->in_shape[a - lead];
                P.n_out[a] = (int)d->out_shape[a - lead];
            }
        }
        P.planes = d->n * d->c;
        P.pad = d->pad;
        P.padv = d->pad_value;
        P.align = d->align;
        P.OXT = P.n_out[2] >= 256 ? 256 : P.n_out[2] > 64 ? 128 : P.n_out[2] > 32 ? 64 : 32;
        P.OYT = std::min(64, 2048 / P.OXT);
        P.tiles_x = (P.n_out[2] + P.OXT - 1) / P.OXT;
        P.tiles_y = (P.n_out[1] + P.OYT - 1) / P.OYT;
        P.x = x;
        P.y = y;
        if ((long long)P.tiles_x * P.tiles_y * P.n_out[0] * P.planes > INT_MAX)
            return fail(FCFS_ERR_UNSUPPORTED, "grid too large");
        cudaError_t e = launch_nearest(P, d->dtype_in, d->dtype_out, st);
        return e == cudaSuccess ? FCFS_OK : cuda_fail(e, "nearest launch");
    }

    return forward_planned(d, x, y, nullptr, st);
}

}  // extern "C"

namespace fcfs {

// The planned separable forward (bulk-copy or gather kernels, planner cache),
// with an optional store epilogue (2D only).
int forward_planned(const fcfs_desc* d, const void* x, void* y, const Epi* epi, cudaStream_t st) {
    FwdParams P;
    int ntk;
    int rc = build_forward_params(d, x, y, &P, &ntk);
    if (rc) return rc;
    if (epi) P.epi = *epi;
    TileChoice tc;
    const bool have = get_plan(P, d->ndim, d->dtype_in, d->dtype_out, &tc);
    if ((have && tc.psk == 1) || psk_policy() == 2) {
        rc = psk_forward(d, P, st);
        if (rc != -1) return rc;
        clear_error();
    }
    if (!have) {
        const bool use_tma = tma_eligible(d, x);
        tc = use_tma ? default_tma_tiles(P, dtype_size(d->dtype_in), d->ndim == 3) : default_tiles(P, d->ndim == 3);
        tc.tma = use_tma ? 1 : 0;
    }
    return launch_choice(d, P, ntk, tc, st);
}

// Whether the planned 2D forward of d runs a kernel that applies the store
// epilogue: every 2D path except the gather kernel for nearest on both axes.
bool forward_has_epilogue_path(const fcfs_desc* d, const void* x) {
    if (d->ndim != 2) return false;
    bool all_nearest = true;
    for (int a = 0; a < d->ndim; ++a) all_nearest &= (d->axis[a].w == nullptr && d->axis[a].method == FCFS_NEAREST);
    return !all_nearest || tma_eligible(d, x);
}

int build_forward_params(const fcfs_desc* d, const void* x, void* y, FwdParams* out, int* ntk) {
    int nt = 1;
    for (int a = 0; a < d->ndim; ++a) nt = std::max(nt, axis_taps(d, a));
    const int w = template_taps(nt);
    if (w < 0) return fail(FCFS_ERR_UNSUPPORTED, "%d taps per phase exceed the kernel templates", nt);
    FwdParams& P = *out;
    memset(&P, 0, sizeof P);
    const int lead = 3 - d->ndim;
    for (int a = 0; a < 3; ++a) {
        if (a < lead) identity_axis(&P.ax[a], w);
        else fill_axis(&P.ax[a], d->axis[a - lead], d->in_shape[a - lead], (int)d->c, w, d->align, keys_a(d),
                       d->antialias);
    }
    P.planes = d->n * d->c;
    P.C = (int)d->c;
    P.pad = d->pad;
    P.padv = d->pad_value;
    P.x = x;
    P.y = y;
    *ntk = w;
    return FCFS_OK;
}

int launch_planned(FwdParams& P, int ntk, bool is3d, int din, int dout, cudaStream_t st) {
    const size_t smem = forward_smem_bytes(P, is3d);
    if (smem > 227 * 1024) return fail(FCFS_ERR_UNSUPPORTED, "tile needs %zu bytes of shared memory", smem);
    const long long blocks = (long long)P.tiles_x * P.tiles_y * P.tiles_d * P.planes;
    if (blocks > INT_MAX) return fail(FCFS_ERR_UNSUPPORTED, "grid too large");
    cudaError_t e = is3d ? launch_forward_3d(P, ntk, din, dout, st) : launch_forward_2d(P, ntk, din, dout, st);
    return e == cudaSuccess ? FCFS_OK : cuda_fail(e, "forward launch");
}

}  // namespace fcfs

// ---------------------------------------------------------------- backward

#include <cudaTypedefs.h>

namespace fcfs {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

// Transposed tap table of one axis (see AdjAxis): entry (k, j, t) of residue u
// for every tap with relative offset e = off[j] + t = u + k*s.
int build_adjoint(const AxisP& A, AdjAxis* J) {
    memset(J, 0, sizeof(*J));
    if (A.s > kMaxS) return fail(FCFS_ERR_UNSUPPORTED, "backward supports s <= %d", kMaxS);
    if (A.r * A.nt_src > kMaxAdj) return fail(FCFS_ERR_UNSUPPORTED, "backward table too large");
    int count[kMaxS] = {0};
    int emax = 0;
    for (int j = 0; j < A.r; ++j)
        for (int t = 0; t < A.nt_src; ++t) {
            const int e = A.off[j] + t;
            count[e % A.s]++;
            emax = std::max(emax, e);
        }
    J->ustart[0] = 0;
    for (int u = 0; u < A.s; ++u) J->ustart[u + 1] = J->ustart[u] + count[u];
    int fillp[kMaxS];
    for (int u = 0; u < A.s; ++u) fillp[u] = J->ustart[u];
    for (int j = 0; j < A.r; ++j)
        for (int t = 0; t < A.nt_src; ++t) {
            const int e = A.off[j] + t;
            const int u = e % A.s, k = e / A.s;
            J->ent[fillp[u]++] = (k << 16) | (j << 8) | t;
        }
    J->vmin = A.lo;
    J->vmax = (A.n_win - 1) * A.s + A.lo + emax;
    return FCFS_OK;
}

// Largest g extent (windows * r) any input tile of width Q needs on one axis,
// over the tiles of the real indices [qa, qb) (qb < 0: the whole axis).
static int g_capacity(const AxisP& A, const AdjAxis& J, int pad, int Q, int qa = 0, int qb = -1) {
    if (qb < 0) qb = A.n_in;
    int cap = 0;
    for (int q0 = qa; q0 < qb; q0 += Q) {
        const int q1 = std::min(qb, q0 + Q) - 1;
        const WinRange w = win_range(A, J, pad, q0, q1);
        cap = std::max(cap, (w.ihi - w.ilo + 1) * A.r);
    }
    return std::max(cap, 1);
}

int build_backward_params(const fcfs_desc* d, const void* x, const void* gy, void* gx, BwdParams* out, int* ntk) {
    BwdParams& B = *out;
    memset(&B, 0, sizeof B);
    int rc = build_forward_params(d, x, nullptr, &B.fw, ntk);
    if (rc) return rc;
    for (int a = 0; a < 3; ++a) {
        B.ax[a] = B.fw.ax[a];
        rc = build_adjoint(B.ax[a], &B.adj[a]);
        if (rc) return rc;
    }
    B.planes = B.fw.planes;
    B.C = B.fw.C;
    B.pad = d->pad;
    B.padv = d->pad_value;
    B.x = x;
    B.gy = gy;
    B.gx = gx;
    B.n = d->n;
    return FCFS_OK;
}

void plan_dx(BwdParams& B, bool is3d) {
    const AxisP &AX = B.ax[2], &AY = B.ax[1], &AD = B.ax[0];
    B.QX = AX.n_in >= 128 ? 128 : AX.n_in > 64 ? 128 : AX.n_in > 32 ? 64 : 32;
    B.QY = is3d ? 16 : 32;
    if (is3d && B.QX > 64) B.QX = 64;
    B.QY = std::min(B.QY, std::max(1, AY.n_in));
    B.Gq = std::max(1, 256 / B.QX);
    for (int it = 0; it < 16; ++it) {
        B.GCcap = g_capacity(AX, B.adj[2], B.pad, B.QX);
        B.GRcap = g_capacity(AY, B.adj[1], B.pad, B.QY);
        B.GCp = B.GCcap;
        B.GDcap = is3d ? g_capacity(AD, B.adj[0], B.pad, 1) : 1;
        if (dx_smem_bytes(B, is3d) <= 100 * 1024 || (B.QY == 1 && B.QX == 32)) break;
        if (B.QY > 1) B.QY = (B.QY + 1) / 2;
        else B.QX = std::max(32, B.QX / 2);
    }
    B.qtiles_x = (AX.n_in + B.QX - 1) / B.QX;
    B.qtiles_y = (AY.n_in + B.QY - 1) / B.QY;
    B.rqx0 = 0;
    B.rqx1 = AX.n_in;
    B.rqy0 = 0;
    B.rqy1 = AY.n_in;
    if (is3d) {
        const long long base = (long long)B.qtiles_x * B.qtiles_y * B.planes;
        const long long chunks = std::max(1LL, (152LL * 6 + base - 1) / base);
        B.QD = (int)std::max(1LL, (AD.n_in + chunks - 1) / chunks);
        B.qtiles_d = (AD.n_in + B.QD - 1) / B.QD;
    } else {
        B.QD = 1;
        B.qtiles_d = 1;
    }
}

// Restrict a planned 2D gather input gradient to the real indices
// [x0, x1) x [y0, y1): tile counts and g capacities of that region's tiles.
void plan_dx_region(BwdParams& B, int x0, int x1, int y0, int y1) {
    B.rqx0 = x0;
    B.rqx1 = x1;
    B.rqy0 = y0;
    B.rqy1 = y1;
    B.QX = std::min(B.QX, std::max(32, (x1 - x0 + 31) / 32 * 32));
    B.Gq = std::max(1, 256 / B.QX);
    B.QY = std::min(B.QY, std::max(1, y1 - y0));
    B.GCcap = g_capacity(B.ax[2], B.adj[2], B.pad, B.QX, x0, x1);
    B.GRcap = g_capacity(B.ax[1], B.adj[1], B.pad, B.QY, y0, y1);
    B.GCp = B.GCcap;
    B.qtiles_x = (x1 - x0 + B.QX - 1) / B.QX;
    B.qtiles_y = (y1 - y0 + B.QY - 1) / B.QY;
}

void plan_dw(BwdParams& B) {
    FwdParams& P = B.fw;
    int WX = std::max(1, 128 / P.ax[2].r);
    int WY = std::max(1, 32 / P.ax[1].r);
    for (int it = 0; it < 64; ++it) {
        apply_tiles(P, false, WX, WY, 1);
        if (dw_smem_bytes(B) <= 110 * 1024) break;
        if (WY > 1) WY = (WY + 1) / 2;
        else if (WX > 1) WX = (WX + 1) / 2;
        else break;
    }
    const int nt = P.ax[2].nt;
    B.dw_axis_off[0] = 0;
    B.dw_axis_off[1] = 0;
    B.dw_axis_off[2] = P.ax[1].r * nt;
    B.dw_rec = (P.ax[1].r + P.ax[2].r) * nt;
}

// Adjoint table of one forward axis in the forward-like form of AdjP.
// Returns the tap count the kernel must evaluate, or -1 if it does not fit.
int build_adjp(const AxisP& A, AdjP* J) {
    memset(J, 0, sizeof(*J));
    if (A.s > kMaxS) return -1;
    J->s = A.s;
    J->r = A.r;
    J->lo_out = A.lo;
    J->n_g = A.n_out;
    J->n_x = A.n_in;
    int emin[kMaxS], emax[kMaxS], lo_in = INT_MAX, efmax = 0;
    for (int u = 0; u < A.s; ++u) {
        emin[u] = INT_MAX;
        emax[u] = INT_MIN;
    }
    for (int j = 0; j < A.r; ++j)
        for (int t = 0; t < A.nt_src; ++t) {
            const int e = A.off[j] + t, u = e % A.s, k = e / A.s;
            const int ep = j - k * A.r;
            emin[u] = std::min(emin[u], ep);
            emax[u] = std::max(emax[u], ep);
            lo_in = std::min(lo_in, ep);
            efmax = std::max(efmax, e);
        }
    int nt = 1;
    for (int u = 0; u < A.s; ++u)
        if (emin[u] != INT_MAX) nt = std::max(nt, emax[u] - emin[u] + 1);
    if (nt > kMaxAdjTaps) return -1;
    for (int u = 0; u < A.s; ++u) {
        for (int t = 0; t < kMaxAdjTaps; ++t) J->idx[u * kMaxAdjTaps + t] = -1;
        if (emin[u] == INT_MAX) {
            J->off[u] = 0;
            J->ntu[u] = 0;
            continue;
        }
        J->off[u] = (short)(emin[u] - lo_in);
        J->ntu[u] = (signed char)(emax[u] - emin[u] + 1);
    }
    for (int j = 0; j < A.r; ++j)
        for (int t = 0; t < A.nt_src; ++t) {
            const int e = A.off[j] + t, u = e % A.s, k = e / A.s;
            const int ep = j - k * A.r;
            J->idx[u * kMaxAdjTaps + (ep - emin[u])] = (short)(j * A.nt_src + t);
        }
    J->lo_in = lo_in;
    J->vmin = A.lo;
    J->vmax = (A.n_win - 1) * A.s + A.lo + efmax;
    return nt;
}

static int adj_template_taps(int nt) {
    static const int widths[] = {2, 3, 4, 6, 8, 10, 12, 16};
    for (int w : widths)
        if (w >= nt) return w;
    return -1;
}

// Plan the bulk-copy input-gradient kernel.  Returns FCFS_OK when the path
// applies (1D/2D, same storage type for g and dx, 16-byte row pitch of g,
// tables within limits), with *ntk the tap template.
static int plan_dx_tma(const fcfs_desc* d, const BwdParams& B, const void* gy, void* gx, TmaDxParams* T, int* ntk) {
    if (d->ndim > 2 || d->dtype_in != d->dtype_out || d->dtype_in == FCFS_U8) return -1;
    const int es = dtype_size(d->dtype_out);
    const long long Wo = d->out_shape[d->ndim - 1];
    if (((uintptr_t)gy) % 16 || (Wo * es) % 16) return -1;
    if (d->n * d->c >= (1LL << 31)) return -1;
    long long iplane = 1;
    for (int a = 0; a < d->ndim; ++a) iplane *= d->in_shape[a];
    if (iplane >= (1LL << 31)) return -1;
    memset(T, 0, sizeof(*T));
    int nt = 1;
    for (int a = 0; a < 3; ++a) {
        T->ax[a] = B.ax[a];
        const int n = build_adjp(B.ax[a], &T->aj[a]);
        if (n < 0) return -1;
        nt = std::max(nt, n);
    }
    const int w = adj_template_taps(nt);
    if (w < 0) return -1;
    // padded taps widen the span each adjoint window reads
    for (int a = 1; a < 3; ++a) {
        AdjP& J = T->aj[a];
        J.nt = w;
        int span = 0;
        for (int u = 0; u < J.s; ++u) span = std::max(span, J.off[u] + w);
        J.span = span;
    }
    T->C = (int)d->c;
    T->pad = d->pad;
    T->align = 16 / es;
    T->threads = 256;
    const int Nx = T->aj[2].n_x, Ny = T->aj[1].n_x;
    T->QX = Nx >= 128 ? 128 : Nx > 64 ? 128 : Nx > 32 ? 64 : 32;
    T->QY = std::min(32, std::max(1, Ny));
    // register-blocked variant: one phase count and window span on both axes
    auto true_span = [](const AdjP& J) {
        int sp = 0;
        for (int u = 0; u < J.s; ++u) sp = std::max(sp, J.off[u] + J.ntu[u]);
        return sp;
    };
    bool rs_ok = T->aj[2].s == T->aj[1].s && T->aj[2].r == T->aj[1].r &&
                 true_span(T->aj[2]) == true_span(T->aj[1]) && dx_rs_compiled(T->aj[2].s, true_span(T->aj[2]));
    T->rs_vw = rs_ok ? dx_rs_vector_width(T->aj[2].r, es) : 0;
    // vector loads need every adjoint window to start on a VW boundary of the staged row: the
    // window starts are a r + lo_in with r = VW and the row starts on a 16-byte boundary
    if (T->rs_vw > 1 && ((T->aj[2].lo_in % T->rs_vw) + T->rs_vw) % T->rs_vw != 0) T->rs_vw = 0;
    rs_ok = rs_ok && T->rs_vw > 0;
    T->rs_span = rs_ok ? true_span(T->aj[2]) : 0;
    // the register-blocked kernel starts from tall tiles (fixed per-tile latency spread over more
    // rows; 2/3 downscale gradient 0.21 -> 0.165 ms at 16x3x1080p) and shrinks them to its budget
    if (rs_ok) T->QY = std::min(128, std::max(1, Ny));
    // the x pass reads the span rounded up to VW samples (at least a pair) from each window start
    const int vp = std::max(T->rs_vw, 2);
    const int spanx = rs_ok ? (T->rs_span + vp - 1) / vp * vp : 0;
    for (int it = 0; it < 24; ++it) {
        // capacities over every tile position of each axis
        int vx = 1, vy = 1, gw = 1, gh = 1, wa = 1, fxp = 1;
        for (int q0 = 0; q0 < Nx; q0 += T->QX) {
            const AxRange R = ax_range(T->aj[2], d->pad, q0, std::min(Nx, q0 + T->QX) - 1);
            vx = std::max(vx, R.vhi - R.vlo + 1);
            if (R.ahi >= R.alo) {
                gw = std::max(gw, (R.ahi - R.alo) * T->aj[2].r + std::max(T->aj[2].span, spanx));
                wa = std::max(wa, R.ahi - R.alo + 1);
                // register-blocked layout: the windows' outputs start up to 3 columns in, and the
                // y pass reads the tile's QX columns from its first real column
                const int fxw = R.alo * T->aj[2].s + T->aj[2].lo_out;
                fxp = std::max(fxp, 3 + (R.ahi - R.alo + 1) * T->aj[2].s);
                fxp = std::max(fxp, 3 + q0 - fxw + T->QX);
            }
        }
        T->WAcap = wa;
        T->FXP = rs_ok ? (std::max(vx, fxp) + 3) / 4 * 4 : std::max(vx, wa * T->aj[2].s);
        for (int q0 = 0; q0 < Ny; q0 += T->QY) {
            const AxRange R = ax_range(T->aj[1], d->pad, q0, std::min(Ny, q0 + T->QY) - 1);
            vy = std::max(vy, R.vhi - R.vlo + 1);
            if (R.ahi >= R.alo) gh = std::max(gh, (R.ahi - R.alo) * T->aj[1].r + T->aj[1].span);
        }
        T->VXcap = vx;
        T->VYcap = vy;
        T->GBW = (gw + T->align - 1 + T->align - 1) / T->align * T->align;
        T->GBH = gh;
        const size_t gbytes = (size_t)T->GBW * T->GBH * es;
        const size_t obytes = (size_t)T->VYcap * T->QX * 4;
        T->buf_bytes = (int)((std::max(gbytes, obytes) + 127) / 128 * 128);
        T->stages = T->buf_bytes <= 12 * 1024 ? 3 : 2;
        T->fx_off = T->stages * T->buf_bytes;
        T->w_off = T->fx_off + T->GBH * T->FXP * 4;
        T->tab_off = T->w_off + (T->aj[2].s + T->aj[1].s) * w * 4;
        T->bar_off = (T->tab_off + (T->VXcap + T->VYcap) * 4 + 15) / 16 * 16;
        // the register-blocked kernel runs at most four CTAs per SM (registers) and gains from
        // taller tiles (less halo per output row); the per-output kernel from more resident CTAs
        const size_t budget = rs_ok ? 110 * 1024 : 56 * 1024;
        if (T->GBW <= 256 && T->GBH <= 256 && T->bar_off + 8 * T->stages <= budget) break;
        if (T->QX > 64 && T->QX >= 4 * T->QY) T->QX /= 2;
        else if (rs_ok && T->QY > 32) T->QY -= 8;  // tall tiles shrink in steps of 8 rows to the budget
        else if (T->QY > 8) T->QY /= 2;
        else if (T->QX > 32) T->QX /= 2;
        else break;
    }
    if (T->GBW > 256 || T->GBH > 256 || T->bar_off + 8 * T->stages > 200 * 1024) return -1;
    T->qtiles_x = (Nx + T->QX - 1) / T->QX;
    T->qtiles_y = (Ny + T->QY - 1) / T->QY;
    T->ntiles = (long long)T->qtiles_x * T->qtiles_y * d->n * d->c;
    // tiles dealt one at a time round-robin (balanced edge tiles, shared halos in L2); one run per
    // CTA for per-channel weights, which are restaged at every change of channel
    T->chunk = B.ax[1].learn || B.ax[2].learn ? 0 : 1;
    if (T->ntiles >= (1LL << 31)) return -1;
    T->gy = gy;
    T->gx = gx;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return -1;
    const cuuint64_t Wg = (cuuint64_t)T->aj[2].n_g, Hg = (cuuint64_t)T->aj[1].n_g;
    cuuint64_t dims[3] = {Wg, Hg, (cuuint64_t)(d->n * d->c)};
    cuuint64_t strides[2] = {Wg * es, Wg * Hg * es};
    cuuint32_t box[3] = {(cuuint32_t)T->GBW, (cuuint32_t)T->GBH, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (enc(&T->tmap, dt, 3, const_cast<void*>(gy), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return -1;
    *ntk = w;
    return FCFS_OK;
}

// Plan the bulk-copy 3D input-gradient kernel (same storage type for g and
// dx, 16-byte row pitch of g, adjoint taps within the kernel templates).
// Tiles of up to 128 x 32 real (x, y) indices (a g plane's fixed costs spread
// over many outputs; two CTAs per SM) and a depth chunk sized so the
// persistent grid gets several tiles per CTA.
static int plan_dx3_tma(const fcfs_desc* d, const BwdParams& B, const void* gy, void* gx, TmaDx3Params* T,
                        int* ntk) {
    if (d->ndim != 3 || d->dtype_in != d->dtype_out || d->dtype_in == FCFS_U8) return -1;
    const int es = dtype_size(d->dtype_out);
    const long long Wo = d->out_shape[2];
    if (((uintptr_t)gy) % 16 || (Wo * es) % 16) return -1;
    if (d->n * d->c >= (1LL << 31)) return -1;
    memset(T, 0, sizeof(*T));
    int nt = 1;
    for (int a = 0; a < 3; ++a) {
        T->ax[a] = B.ax[a];
        const int n = build_adjp(B.ax[a], &T->aj[a]);
        if (n < 0) return -1;
        nt = std::max(nt, n);
    }
    const int w = adj_template_taps(nt);
    if (w < 0 || w > 8) return -1;
    for (int a = 0; a < 3; ++a) {
        AdjP& J = T->aj[a];
        J.nt = w;
        int span = 0;
        for (int u = 0; u < J.s; ++u) span = std::max(span, J.off[u] + w);
        J.span = span;
    }
    T->C = (int)d->c;
    T->pad = d->pad;
    T->align = 16 / es;
    T->threads = 256;
    // depth indices that receive folded padding contributions
    const AdjP& JD = T->aj[0];
    const int Nd = JD.n_x, Ny = T->aj[1].n_x, Nx = T->aj[2].n_x;
    T->nL = T->nR = 0;
    if (d->pad != FCFS_PAD_CONSTANT) {
        for (int v = JD.vmin; v < 0; ++v) T->nL = std::max(T->nL, ext_index(v, Nd, d->pad) + 1);
        int tmin = Nd;
        for (int v = Nd; v <= JD.vmax; ++v) tmin = std::min(tmin, ext_index(v, Nd, d->pad));
        T->nR = Nd - tmin;
        if (T->nL + T->nR > Nd) {
            T->nL = Nd;
            T->nR = 0;
        }
    }
    T->QX = Nx > 64 ? 128 : Nx > 32 ? 64 : 32;
    T->QY = std::min(32, std::max(1, Ny));
    const int nfold = T->nL + T->nR;
    for (int it = 0; it < 8; ++it) {
        int vx = 1, vy = 1, gwid = 1, gh = 1;
        for (int q0 = 0; q0 < Nx; q0 += T->QX) {
            const AxRange R = ax_range(T->aj[2], d->pad, q0, std::min(Nx, q0 + T->QX) - 1);
            vx = std::max(vx, R.vhi - R.vlo + 1);
            if (R.ahi >= R.alo) gwid = std::max(gwid, (R.ahi - R.alo) * T->aj[2].r + T->aj[2].span);
        }
        for (int q0 = 0; q0 < Ny; q0 += T->QY) {
            const AxRange R = ax_range(T->aj[1], d->pad, q0, std::min(Ny, q0 + T->QY) - 1);
            vy = std::max(vy, R.vhi - R.vlo + 1);
            if (R.ahi >= R.alo) gh = std::max(gh, (R.ahi - R.alo) * T->aj[1].r + T->aj[1].span);
        }
        T->VXcap = vx;
        T->VYcap = vy;
        T->GBW = (gwid + T->align - 1 + T->align - 1) / T->align * T->align;
        T->GBH = gh;
        const size_t gbytes = (size_t)T->GBW * T->GBH * es;
        const size_t obytes = (size_t)T->VYcap * T->QX * 4;
        T->buf_bytes = (int)((std::max(gbytes, obytes) + 127) / 128 * 128);
        T->stages = T->buf_bytes <= 8 * 1024 ? 4 : T->buf_bytes <= 16 * 1024 ? 3 : 2;
        const size_t plane = (size_t)T->QY * T->QX * 4;
        size_t off = (size_t)T->stages * T->buf_bytes;
        T->fx_off = (int)off;
        off += (size_t)T->GBH * T->VXcap * 4;
        T->ring_off = (int)off;
        off += (size_t)JD.span * plane;
        T->facc_off = (int)off;
        off += (size_t)nfold * plane;
        T->w_off = (int)off;
        off += (size_t)(T->aj[0].s + T->aj[1].s + T->aj[2].s) * w * 4;
        T->tab_off = (int)off;
        off += (size_t)(T->VXcap + T->VYcap) * 4;
        T->bar_off = (int)((off + 15) / 16 * 16);
        if (T->GBW <= 256 && T->GBH <= 256 && T->bar_off + 8 * T->stages <= 110 * 1024) break;
        if (T->QY > 8) T->QY /= 2;
        else if (T->QX > 32) T->QX /= 2;
        else break;
    }
    if (T->GBW > 256 || T->GBH > 256 || T->bar_off + 8 * T->stages > 200 * 1024) return -1;
    T->qtiles_x = (Nx + T->QX - 1) / T->QX;
    T->qtiles_y = (Ny + T->QY - 1) / T->QY;
    const long long base = (long long)T->qtiles_x * T->qtiles_y * d->n * d->c;
    const long long want = 152LL * 2 * 4;
    const long long chunks = std::max(1LL, std::min<long long>(Nd, (want + base - 1) / base));
    T->QD = (int)((Nd + chunks - 1) / chunks);
    T->qtiles_d = (Nd + T->QD - 1) / T->QD;
    const long long ntiles = base * T->qtiles_d;
    if (ntiles >= (1LL << 31)) return -1;
    T->ntiles = (int)ntiles;
    T->chunk = 0;  // contiguous runs: measured faster for the volume kernels than dealt tiles
    T->gy = gy;
    T->gx = gx;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return -1;
    const cuuint64_t Wg = (cuuint64_t)T->aj[2].n_g, Hg = (cuuint64_t)T->aj[1].n_g, Dg = (cuuint64_t)JD.n_g;
    cuuint64_t dims[4] = {Wg, Hg, Dg, (cuuint64_t)(d->n * d->c)};
    cuuint64_t strides[3] = {Wg * es, Wg * Hg * es, Wg * Hg * Dg * es};
    cuuint32_t box[4] = {(cuuint32_t)T->GBW, (cuuint32_t)T->GBH, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (enc(&T->tmap, dt, 4, const_cast<void*>(gy), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return -1;
    *ntk = w;
    return FCFS_OK;
}

// Plan the bulk-copy weight-gradient kernel (1D/2D, x and gy in the same
// storage type, 16-byte row pitches).  The grid is fixed by the tile's
// shared-memory footprint on a 152-SM GB300, so the workspace size and the
// summation order depend on the descriptor only.
static int plan_dw_tma(const fcfs_desc* d, const FwdParams& P0, const void* x, const void* gy, TmaDwParams* T,
                       int* ntk, bool encode) {
    if (d->ndim > 2 || d->dtype_in != d->dtype_out || d->dtype_in == FCFS_U8) return -1;
    const int es = dtype_size(d->dtype_in);
    const long long W = d->in_shape[d->ndim - 1], Wo = d->out_shape[d->ndim - 1];
    if ((W * es) % 16 || (Wo * es) % 16) return -1;
    if (encode && (((uintptr_t)x) % 16 || ((uintptr_t)gy) % 16)) return -1;
    if (d->n * d->c >= (1LL << 31)) return -1;
    memset(T, 0, sizeof(*T));
    T->P = P0;
    FwdParams& P = T->P;
    const int nt = P.ax[2].nt;
    const int align = 16 / es;
    T->align = align;
    T->threads = 256;
    // register-blocked kernel: learnable taps on both axes, one phase count and tap count
    const AxisP &AXx = P.ax[2], &AXy = P.ax[1];
    T->rb = 0;
    if (d->ndim == 2 && AXx.learn && AXy.learn && AXx.r == AXy.r && AXx.nt_src == nt && AXy.nt_src == nt &&
        dw_rb_compiled(AXx.r, nt)) {
        const int R = AXx.r;
        int WX = std::max(1, 120 / R), WY = std::max(1, 60 / R);
        for (int it = 0; it < 64; ++it) {
            apply_tiles(P, false, WX, WY, 1, 0);
            T->BWx = (P.IC + align - 1 + align - 1) / align * align;
            T->BHx = P.IR;
            T->BWg = (P.OX + align - 1 + align - 1) / align * align;
            T->BHg = P.OY;
            T->ICp = P.IC;
            T->xbuf_bytes = (T->BWx * T->BHx * es + 127) / 128 * 128;
            T->gbuf_bytes = (T->BWg * T->BHg * es + 127) / 128 * 128;
            T->sh_off = 2 * T->xbuf_bytes + 2 * T->gbuf_bytes;
            T->sv_off = T->sh_off + P.IR * P.OX * 4;
            T->w_off = T->sv_off + P.OY * T->ICp * 4;
            T->red_off = T->w_off;
            T->bar_off = (T->red_off + (T->threads / 32) * 2 * R * nt * 4 + 15) / 16 * 16;
            const bool fits = T->BWx <= 256 && T->BHx <= 256 && T->BWg <= 256 && T->BHg <= 256 &&
                              P.OX <= T->threads && P.IC <= T->threads && P.WX <= T->threads &&
                              T->bar_off + 16 <= 110 * 1024;
            if (fits) {
                T->rb = R;
                break;
            }
            if ((P.OX > T->threads || P.IC > T->threads || T->BWx > 256) && WX > 1) WX = std::max(1, WX * 3 / 4);
            else if (WY > 1) WY = (WY + 1) / 2;
            else if (WX > 1) WX = (WX + 1) / 2;
            else break;
        }
    }
    int WX = std::max(1, 128 / P.ax[2].r), WY = std::max(1, 32 / P.ax[1].r);
    for (int it = 0; it < 64 && !T->rb; ++it) {
        apply_tiles(P, false, WX, WY, 1, 0);
        const int npair = P.OX * P.ax[1].r;
        T->BWx = (P.IC + align - 1 + align - 1) / align * align;
        T->BHx = P.IR;
        T->BWg = (P.OX + align - 1 + align - 1) / align * align;
        T->BHg = P.OY;
        T->ICp = P.IC;
        T->xbuf_bytes = (T->BWx * T->BHx * es + 127) / 128 * 128;
        T->gbuf_bytes = (T->BWg * T->BHg * es + 127) / 128 * 128;
        T->sh_off = 2 * T->xbuf_bytes + 2 * T->gbuf_bytes;
        T->sv_off = T->sh_off + P.IR * P.OX * 4;
        T->w_off = T->sv_off + P.OY * T->ICp * 4;
        T->red_off = T->w_off + (P.ax[2].r + P.ax[1].r) * nt * 4;
        T->bar_off = (T->red_off + (T->threads + npair) * nt * 4 + 15) / 16 * 16;
        const bool fits = T->BWx <= 256 && T->BHx <= 256 && T->BWg <= 256 && T->BHg <= 256 &&
                          npair <= 2 * T->threads && P.OX <= T->threads && T->bar_off + 16 <= 64 * 1024;
        if (fits) break;
        if (npair > 2 * T->threads && WX > 1) WX = std::max(1, WX * 3 / 4);
        else if (WY > 1) WY = (WY + 1) / 2;
        else if (WX > 1) WX = (WX + 1) / 2;
        else return -1;
    }
    const int npair = P.OX * P.ax[1].r;
    if (!T->rb && (npair > 2 * T->threads || P.OX > T->threads)) return -1;
    if (T->bar_off + 16 > 227 * 1024) return -1;
    const long long ntiles = (long long)P.tiles_x * P.tiles_y * P.planes;
    if (ntiles >= (1LL << 31)) return -1;
    T->ntiles = (int)ntiles;
    // CTAs per SM by shared memory (the register-blocked kernel is built for two)
    const int per_sm = std::max(1, std::min(T->rb ? 2 : 8, (int)(227 * 1024 / (T->bar_off + 16))));
    T->grid = (int)std::min<long long>(ntiles, 152LL * per_sm);
    const int per = (T->ntiles + T->grid - 1) / T->grid;
    const int tpp = P.tiles_x * P.tiles_y;
    T->maxseg = (per + tpp - 1) / tpp + 1;
    T->rec = (P.ax[1].r + P.ax[2].r) * nt;
    T->n = d->n;
    *ntk = nt;
    if (!encode) return FCFS_OK;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return -1;
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint32_t estr[3] = {1, 1, 1};
    {
        const cuuint64_t Wx = (cuuint64_t)P.ax[2].n_in, Hx = (cuuint64_t)P.ax[1].n_in;
        cuuint64_t dims[3] = {Wx, Hx, (cuuint64_t)P.planes};
        cuuint64_t strides[2] = {Wx * es, Wx * Hx * es};
        cuuint32_t box[3] = {(cuuint32_t)T->BWx, (cuuint32_t)T->BHx, 1};
        if (enc(&T->tmap_x, dt, 3, const_cast<void*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
    }
    {
        const cuuint64_t Wg = (cuuint64_t)P.ax[2].n_out, Hg = (cuuint64_t)P.ax[1].n_out;
        cuuint64_t dims[3] = {Wg, Hg, (cuuint64_t)P.planes};
        cuuint64_t strides[2] = {Wg * es, Wg * Hg * es};
        cuuint32_t box[3] = {(cuuint32_t)T->BWg, (cuuint32_t)T->BHg, 1};
        if (enc(&T->tmap_g, dt, 3, const_cast<void*>(gy), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
    }
    return FCFS_OK;
}

static size_t dw_tma_workspace(const TmaDwParams& T) {
    const long long nrec = (long long)T.grid * T.maxseg;
    return (size_t)((nrec * (T.rec + 1) * sizeof(float) + 255) / 256 * 256);
}

static size_t dw_workspace(const BwdParams& B) {
    const long long recs = (long long)B.fw.tiles_x * B.fw.tiles_y * B.planes;
    return (size_t)(((recs * B.dw_rec * sizeof(float)) + 255) / 256 * 256);
}

// Backward of the non-separable 2D layer: gw[0] (if given) receives the
// gradient of w2d, gw[1] must be NULL.
static int backward_full2d(const fcfs_desc* d, const void* x, const void* gy, void* gx, float* const* gw, void* ws,
                           size_t ws_bytes, cudaStream_t st) {
    float* gw2d = gw ? gw[0] : nullptr;
    if (gw && gw[1]) return fail(FCFS_ERR_ARG, "gw[1] must be NULL with w2d (gw[0] receives its gradient)");
    if (gw2d && ((uintptr_t)gw2d) % 4) return fail(FCFS_ERR_ARG, "gw[0] not 4-byte aligned");
    if (!gx && !gw2d) return FCFS_OK;
    if (numel_in(d) == 0) return FCFS_OK;
    if (gy && ((uintptr_t)gy) % dtype_size(d->dtype_out)) return fail(FCFS_ERR_ARG, "gy misaligned");
    if (gx && ((uintptr_t)gx) % dtype_size(d->dtype_in)) return fail(FCFS_ERR_ARG, "gx misaligned");
    if (numel_out(d) == 0) {
        if (gx) {
            cudaError_t e = cudaMemsetAsync(gx, 0, (size_t)numel_in(d) * dtype_size(d->dtype_in), st);
            if (e != cudaSuccess) return cuda_fail(e, "memset gx");
        }
        if (gw2d) {
            size_t n = (size_t)(d->w2d_per_channel ? d->c : 1) * d->axis[0].r * d->axis[1].r;
            for (int a = 0; a < 2; ++a) n *= 2 * (d->axis[a].K ? d->axis[a].K : k_min(d->axis[a].method, d->axis[a].s)) + 1;
            cudaError_t e = cudaMemsetAsync(gw2d, 0, n * sizeof(float), st);
            if (e != cudaSuccess) return cuda_fail(e, "memset gw");
        }
        return FCFS_OK;
    }
    if (!gy) return fail(FCFS_ERR_ARG, "gy is NULL");
    if (gw2d) {
        if (!x) return fail(FCFS_ERR_ARG, "x is required for weight gradients");
        if (((uintptr_t)x) % dtype_size(d->dtype_in)) return fail(FCFS_ERR_ARG, "x misaligned");
        if (((uintptr_t)ws) % 256) return fail(FCFS_ERR_ARG, "workspace not 256-byte aligned");
    }
    return full2d_backward(d, x, gy, gx, gw2d, ws, ws_bytes, st);
}

static bool any_learnable(const fcfs_desc* d) {
    for (int a = 0; a < d->ndim; ++a)
        if (d->axis[a].w) return true;
    return false;
}

}  // namespace fcfs

extern "C" {

size_t fcfs_backward_workspace(const fcfs_desc* d) {
    clear_error();
    if (validate_desc(d, true) != FCFS_OK) return 0;
    if (d->w2d) return numel_out(d) == 0 ? 0 : full2d_workspace(d);
    if (!any_learnable(d) || d->ndim == 3 || numel_out(d) == 0) return 0;
    BwdParams B;
    int ntk;
    if (build_backward_params(d, nullptr, nullptr, nullptr, &B, &ntk) != FCFS_OK) return 0;
    TmaDwParams T;
    int ntw = 0;
    const size_t fast = plan_dw_tma(d, B.fw, nullptr, nullptr, &T, &ntw, false) == FCFS_OK ? dw_tma_workspace(T) : 0;
    clear_error();
    plan_dw(B);
    return std::max(fast, dw_workspace(B));
}

int fcfs_backward(const fcfs_desc* d, const void* x, const void* gy, void* gx, float* const* gw, void* workspace,
                  size_t ws_bytes, void* stream) {
    NvtxRange nv("fcfs_backward");
    clear_error();
    int rc = validate_desc(d, true);
    if (rc) return rc;
    if (d->dtype_in == FCFS_U8) return fail(FCFS_ERR_UNSUPPORTED, "no gradient for uint8 inputs");
    bool want_w = false;
    if (d->w2d) return backward_full2d(d, x, gy, gx, gw, workspace, ws_bytes, (cudaStream_t)stream);
    for (int a = 0; a < d->ndim && gw; ++a) {
        if (!gw[a]) continue;
        if (!d->axis[a].w) return fail(FCFS_ERR_ARG, "gw[%d] given but axis %d has no learnable weights", a, a);
        if (((uintptr_t)gw[a]) % 4) return fail(FCFS_ERR_ARG, "gw[%d] not 4-byte aligned", a);
        want_w = true;
    }
    if (want_w && d->ndim == 3) return fail(FCFS_ERR_UNSUPPORTED, "weight gradients are implemented for 1D/2D");
    if (!gx && !want_w) return FCFS_OK;
    if (numel_in(d) == 0) return FCFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const bool empty_out = numel_out(d) == 0;
    if (!empty_out && !gy) return fail(FCFS_ERR_ARG, "gy is NULL");
    if (gy && ((uintptr_t)gy) % dtype_size(d->dtype_out)) return fail(FCFS_ERR_ARG, "gy misaligned");
    if (gx && ((uintptr_t)gx) % dtype_size(d->dtype_in)) return fail(FCFS_ERR_ARG, "gx misaligned");
    if (empty_out) {
        // no output depends on x: the gradients are zero
        if (gx) {
            cudaError_t e = cudaMemsetAsync(gx, 0, (size_t)numel_in(d) * dtype_size(d->dtype_in), st);
            if (e != cudaSuccess) return cuda_fail(e, "memset gx");
        }
        for (int a = 0; a < d->ndim && gw; ++a) {
            if (!gw[a]) continue;
            const int K = d->axis[a].K ? d->axis[a].K : k_min(d->axis[a].method, d->axis[a].s);
            const size_t n = (size_t)(d->axis[a].w_per_channel ? d->c : 1) * d->axis[a].r * (2 * K + 1);
            cudaError_t e = cudaMemsetAsync(gw[a], 0, n * sizeof(float), st);
            if (e != cudaSuccess) return cuda_fail(e, "memset gw");
        }
        return FCFS_OK;
    }
    BwdParams B;
    int ntk;
    rc = build_backward_params(d, x, gy, gx, &B, &ntk);
    if (rc) return rc;
    const bool is3d = d->ndim == 3;
    if (want_w) {
        if (!x) return fail(FCFS_ERR_ARG, "x is required for weight gradients");
        if (((uintptr_t)x) % dtype_size(d->dtype_in)) return fail(FCFS_ERR_ARG, "x misaligned");
        plan_dw(B);
        const size_t need = dw_workspace(B);
        if (!workspace || ws_bytes < need)
            return fail(FCFS_ERR_NOMEM, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
        if (((uintptr_t)workspace) % 256) return fail(FCFS_ERR_ARG, "workspace not 256-byte aligned");
        B.ws = (float*)workspace;
        const int lead = 3 - d->ndim;
        for (int a = 0; a < d->ndim; ++a) B.gw[lead + a] = gw[a];
        const long long blocks = (long long)B.fw.tiles_x * B.fw.tiles_y * B.planes;
        if (blocks > INT_MAX || dw_smem_bytes(B) > 227 * 1024) return fail(FCFS_ERR_UNSUPPORTED, "weight-gradient tile too large");
    }
    if (gx && !is3d) {
        TmaDxParams T;
        int ntd = 0;
        const bool tile_ok = plan_dx_tma(d, B, gy, gx, &T, &ntd) == FCFS_OK;
        clear_error();
        // the strip kernel on the interior and the gather kernel on the border bands, where the
        // tile path has no register-blocked kernel for this window shape (or when asked for)
        if (psk_policy() == 2 || (psk_policy() == 1 && !(tile_ok && T.rs_span > 0))) {
            rc = psk_input_gradient(d, B, gy, gx, ntk, st);
            if (rc == FCFS_OK) gx = nullptr;
            else if (rc != -1) return rc;
            clear_error();
        }
        if (gx && tile_ok) {
            cudaError_t e = cudaErrorInvalidValue;
            if (T.rs_span > 0) e = launch_dx_rs(T, d->dtype_out, st);
            if (e == cudaErrorInvalidValue) e = launch_dx_tma(T, ntd, d->dtype_out, d->dtype_in, st);
            if (e != cudaSuccess) return cuda_fail(e, "input-gradient (bulk-copy) launch");
            gx = nullptr;  // done
        }
        clear_error();
    }
    if (gx && is3d) {
        TmaDx3Params T;
        int ntd = 0;
        if (plan_dx3_tma(d, B, gy, gx, &T, &ntd) == FCFS_OK) {
            cudaError_t e = launch_dx3d_tma(T, ntd, d->dtype_out, st);
            if (e != cudaSuccess) return cuda_fail(e, "3D input-gradient (bulk-copy) launch");
            gx = nullptr;  // done
        }
        clear_error();
    }
    if (gx) {
        plan_dx(B, is3d);
        if (is3d && B.GDcap > 256) return fail(FCFS_ERR_UNSUPPORTED, "depth ratio needs more than 256 gradient planes per tile");
        const long long blocks = (long long)B.qtiles_x * B.qtiles_y * B.qtiles_d * B.planes;
        if (blocks > INT_MAX || dx_smem_bytes(B, is3d) > 227 * 1024)
            return fail(FCFS_ERR_UNSUPPORTED, "input-gradient tile too large");
        cudaError_t e = launch_dx(B, ntk, d->dtype_out, d->dtype_in, is3d, st);
        if (e != cudaSuccess) return cuda_fail(e, "input-gradient launch");
    }
    if (want_w) {
        TmaDwParams T;
        int ntw = 0;
        BwdParams B2;
        int ntk2;
        build_backward_params(d, x, gy, gx, &B2, &ntk2);
        if (plan_dw_tma(d, B2.fw, x, gy, &T, &ntw, true) == FCFS_OK && dw_tma_workspace(T) <= ws_bytes) {
            T.ws = (float*)workspace;
            const int lead = 3 - d->ndim;
            for (int a = 0; a < d->ndim; ++a) T.gw[lead + a] = gw[a];
            cudaError_t e = launch_dw_tma(T, ntw, d->dtype_in, st, x);
            if (e != cudaSuccess) return cuda_fail(e, "weight-gradient (bulk-copy) launch");
        } else {
            clear_error();
            cudaError_t e = launch_dw(B, ntk, d->dtype_in, d->dtype_out, st);
            if (e != cudaSuccess) return cuda_fail(e, "weight-gradient launch");
            e = launch_dw_reduce(B, st);
            if (e != cudaSuccess) return cuda_fail(e, "weight-gradient reduce launch");
        }
    }
    return FCFS_OK;
}

}  // extern "C"

// ------------------------------------------------------------- TMA path

namespace fcfs {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// The bulk-tensor path needs a 16-byte aligned base, rows whose byte pitch is
// a multiple of 16, and extents a tensor map can describe.
bool tma_eligible(const fcfs_desc* d, const void* x) {
    const int es = dtype_size(d->dtype_in);
    const long long W = d->in_shape[d->ndim - 1];
    const long long H = d->ndim >= 2 ? d->in_shape[d->ndim - 2] : 1;
    const long long D = d->ndim == 3 ? d->in_shape[0] : 1;
    if (((uintptr_t)x) % 16) return false;
    if ((W * es) % 16) return false;
    if (W >= (1LL << 31) || H >= (1LL << 31) || D >= (1LL << 31) || d->n * d->c >= (1LL << 31)) return false;
    if (d->ndim == 3 && d->dtype_in != d->dtype_out) return false;
    if (d->ndim == 3 && d->dtype_in == FCFS_U8) return false;
    long long oplane = 1;
    for (int a = 0; a < d->ndim; ++a) oplane *= d->out_shape[a];
    if (oplane >= (1LL << 31)) return false;  // 32-bit offsets within an output plane
    return encode_fn() != nullptr;
}

static int box_width(int IC, int align) { return (IC + align - 1 + align - 1) / align * align; }

static void tma_sizes(const FwdParams& P, int es, int* BW, int* BH, int* buf_bytes, int* bar_off) {
    const int align = 16 / es;
    *BW = box_width(P.IC, align);
    *BH = P.IR;
    *buf_bytes = ((*BW) * (*BH) * es + 127) / 128 * 128;
    size_t off = 2 * (size_t)(*buf_bytes) + (size_t)P.IR * P.OX * 4 + (size_t)(P.ax[2].r + P.ax[1].r) * P.ax[2].nt * 4;
    *bar_off = (int)((off + 15) / 16 * 16);
}

// 256-thread CTAs; output columns ~128 (an even count), rows as the
// shared-memory budget allows (3+ CTAs per SM, tiles of ~16-32 outputs per
// thread so per-tile work amortizes).
TileChoice default_tma3_tiles(const FwdParams& P0, int es);

TileChoice default_tma_tiles(const FwdParams& P0, int es, bool is3d) {
    if (is3d) return default_tma3_tiles(P0, es);
    FwdParams P = P0;
    const int rx = P.ax[2].r, ry = P.ax[1].r;
    int WX = std::max(1, 128 / rx);
    // tile widths a multiple of 8 outputs where possible (16-byte vector stores of BF16 rows)
    int wx8 = WX;
    while (wx8 > 1 && (wx8 * rx) % 8) --wx8;
    if ((wx8 * rx) % 8 == 0 && 4 * wx8 >= 3 * WX) WX = wx8;
    if ((WX * rx) % 2 && WX > 1) WX -= 1;
    // two-byte inputs: twice the rows in the same staging bytes (shrunk below when the budget says so)
    int WY = std::max(1, (es <= 2 ? 128 : 64) / ry);
    for (int it = 0; it < 64; ++it) {
        apply_tiles(P, false, WX, WY, 1, 0);
        int BW, BH, bb, bo;
        tma_sizes(P, es, &BW, &BH, &bb, &bo);
        if (BW <= 256 && BH <= 256 && bo + 16 <= 72 * 1024) break;
        if (BW > 256 && WX > 1) WX = std::max(1, WX * 3 / 4);
        else if (WY > 1) WY = std::max(1, WY * 3 / 4);
        else if (WX > 1) WX = std::max(1, WX * 3 / 4);
        else break;
    }
    TileChoice t{WX, WY, 1};
    t.G = 0;
    t.tma = 1;
    return t;
}

int prepare_tma(const fcfs_desc* d, const FwdParams& P, TmaFwdParams* T, int threads) {
    memset(T, 0, sizeof(*T));
    T->P = P;
    const int es = dtype_size(d->dtype_in);
    T->align = 16 / es;
    tma_sizes(P, es, &T->BW, &T->BH, &T->buf_bytes, &T->bar_off);
    if (T->BW > 256 || T->BH > 256) return fail(FCFS_ERR_UNSUPPORTED, "tile too large for one bulk copy");
    if (P.OX > 256) return fail(FCFS_ERR_UNSUPPORTED, "tile wider than the CTA");
    T->ntiles = (long long)P.tiles_x * P.tiles_y * P.planes;
    if (T->ntiles >= (1LL << 31)) return fail(FCFS_ERR_UNSUPPORTED, "too many tiles");
    T->chunk = P.ax[1].learn || P.ax[2].learn ? 0 : 1;
    T->threads = threads > 0 ? threads : 256;
    if (P.OX > T->threads) return fail(FCFS_ERR_UNSUPPORTED, "tile wider than the CTA");
    const cuuint64_t W = (cuuint64_t)P.ax[2].n_in, H = (cuuint64_t)P.ax[1].n_in;
    cuuint64_t dims[3] = {W, H, (cuuint64_t)P.planes};
    cuuint64_t strides[2] = {W * es, W * H * es};
    cuuint32_t box[3] = {(cuuint32_t)T->BW, (cuuint32_t)T->BH, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = d->dtype_in == FCFS_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : d->dtype_in == FCFS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                              : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUresult r = encode_fn()(&T->tmap, dt, 3, const_cast<void*>(P.x), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FCFS_ERR_UNSUPPORTED, "tensor map encode failed (%d)", (int)r);
    return FCFS_OK;
}

// 3D bulk-copy forward: staging box, plane buffers, the x-pass intermediate,
// the ring of span_d y-interpolated planes and the weights, in that order.
static void tma3_sizes(const FwdParams& P, int es, TmaFwd3Params* T) {
    T->align = 16 / es;
    T->BW = box_width(P.IC, T->align);
    T->BH = P.IR;
    T->buf_bytes = (T->BW * T->BH * es + 127) / 128 * 128;
    // plane copies in flight: a plane is small next to the latency of one copy
    T->stages = T->buf_bytes <= 12 * 1024 ? 4 : T->buf_bytes <= 24 * 1024 ? 3 : 2;
    size_t off = (size_t)T->stages * T->buf_bytes;
    T->sh_off = (int)off;
    off += (size_t)P.IR * P.OX * 4;
    T->ring_off = (int)off;
    off += (size_t)P.ring * P.OY * P.OX * 4;
    T->w_off = (int)off;
    off += (size_t)(P.ax[0].r + P.ax[1].r + P.ax[2].r) * P.ax[2].nt * 4;
    T->bar_off = (int)((off + 15) / 16 * 16);
}

size_t forward3_tma_smem_bytes(const TmaFwd3Params& T) { return (size_t)T.bar_off + 8 * T.stages; }

// Tiles of ~128 output columns and 16-32 output rows (the ring of span_d
// planes dominates shared memory; 3 CTAs per SM), depth chunks so that every
// CTA of the persistent grid gets several tiles.
TileChoice default_tma3_tiles(const FwdParams& P0, int es) {
    FwdParams P = P0;
    const int rx = P.ax[2].r, ry = P.ax[1].r;
    int WX = std::max(1, 128 / rx);
    while (WX > 1 && (WX * rx) % 4) --WX;  // 4-wide column groups in the register-blocked kernel
    int WY = std::max(1, 24 / ry);
    for (int it = 0; it < 64; ++it) {
        apply_tiles(P, true, WX, WY, 1, 0);
        TmaFwd3Params T;
        tma3_sizes(P, es, &T);
        if (T.BW <= 256 && T.BH <= 256 && forward3_tma_smem_bytes(T) <= 72 * 1024) break;
        if (T.BW > 256 && WX > 1) WX = std::max(1, WX * 3 / 4);
        else if (WY > 1) WY = std::max(1, WY * 3 / 4);
        else if (WX > 1) WX = std::max(1, WX * 3 / 4);
        else break;
    }
    // same number of tiles, spread evenly (no thin last tile)
    {
        const int nx = P.ax[2].n_win, ny = P.ax[1].n_win;
        const int tx = (nx + WX - 1) / WX, ty = (ny + WY - 1) / WY;
        int wx = (nx + tx - 1) / tx;
        while ((wx * rx) % 4 && wx < WX) ++wx;
        if ((wx * rx) % 4 == 0 || wx == WX) WX = wx;
        WY = (ny + ty - 1) / ty;
        apply_tiles(P, true, WX, WY, 1, 0);
    }
    const long long base = (long long)P.tiles_x * P.tiles_y * P.planes;
    const long long want = 152LL * 3 * 6;
    const long long chunks = std::max(1LL, (want + base - 1) / base);
    const int WD = (int)std::max(1LL, (P.ax[0].n_win + chunks - 1) / chunks);
    TileChoice t{WX, WY, std::max(WD, 2)};
    t.G = 0;
    t.tma = 1;
    return t;
}

int prepare_tma3(const fcfs_desc* d, const FwdParams& P, TmaFwd3Params* T, int threads) {
    memset(T, 0, sizeof(*T));
    T->P = P;
    const int es = dtype_size(d->dtype_in);
    tma3_sizes(P, es, T);
    if (T->BW > 256 || T->BH > 256) return fail(FCFS_ERR_UNSUPPORTED, "tile too large for one bulk copy");
    T->threads = threads > 0 ? threads : 256;
    if (T->threads > 256) return fail(FCFS_ERR_UNSUPPORTED, "the volume kernels run 256-thread CTAs");
    if (P.OX > T->threads) return fail(FCFS_ERR_UNSUPPORTED, "tile wider than the CTA");
    if (P.ax[2].nt > 5) return fail(FCFS_ERR_UNSUPPORTED, "3D bulk-copy path takes at most 5 taps per phase");
    const long long nt = (long long)P.tiles_x * P.tiles_y * P.tiles_d * P.planes;
    if (nt >= (1LL << 31)) return fail(FCFS_ERR_UNSUPPORTED, "too many tiles");
    T->ntiles = (int)nt;
    T->chunk = 0;  // contiguous runs: measured faster for the volume kernels than dealt tiles
    const cuuint64_t W = (cuuint64_t)P.ax[2].n_in, H = (cuuint64_t)P.ax[1].n_in, D = (cuuint64_t)P.ax[0].n_in;
    cuuint64_t dims[4] = {W, H, D, (cuuint64_t)P.planes};
    cuuint64_t strides[3] = {W * es, W * H * es, W * H * D * es};
    cuuint32_t box[4] = {(cuuint32_t)T->BW, (cuuint32_t)T->BH, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt =
        d->dtype_in == FCFS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = encode_fn()(&T->tmap, dt, 4, const_cast<void*>(P.x), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FCFS_ERR_UNSUPPORTED, "tensor map encode failed (%d)", (int)r);
    return FCFS_OK;
}

// Launch the forward with a tile choice: the TMA-staged persistent kernel
// when the choice asks for it and the layout allows, else the gather kernel.
int launch_choice(const fcfs_desc* d, FwdParams& P, int ntk, const TileChoice& t, cudaStream_t st) {
    const bool is3d = d->ndim == 3;
    if (t.psk == 1) {
        const int rc = psk_forward(d, P, st);
        if (rc != -1) return rc;
        clear_error();
    }
    if (t.tma == 1 && is3d && tma_eligible(d, P.x)) {
        apply_tiles(P, true, t.WX, t.WY, t.WD, 0);
        TmaFwd3Params T;
        int rc = prepare_tma3(d, P, &T, t.threads);
        if (rc == FCFS_OK && forward3_tma_smem_bytes(T) <= 200 * 1024) {
            if (t.rs != 0) {
                cudaError_t e = launch_forward3d_rs(T, d->dtype_in, d->dtype_out, st);
                if (e == cudaSuccess) return FCFS_OK;
                if (e != cudaErrorInvalidValue) return cuda_fail(e, "3D forward (register-blocked) launch");
            }
            cudaError_t e = launch_forward3d_tma(T, ntk, d->dtype_in, d->dtype_out, st);
            return e == cudaSuccess ? FCFS_OK : cuda_fail(e, "3D forward (bulk-copy) launch");
        }
        clear_error();
    }
    if (t.tma == 1 && !is3d && tma_eligible(d, P.x)) {
        apply_tiles(P, false, t.WX, t.WY, 1, t.G);
        TmaFwdParams T;
        int rc = prepare_tma(d, P, &T, t.threads);
        if (rc == FCFS_OK && forward_tma_smem_bytes(T) <= 200 * 1024) {
            if (t.rs != 0 && forward_rs_available(T, d->dtype_in, d->dtype_out)) {
                cudaError_t e = launch_forward_rs(T, d->dtype_in, st);
                if (e == cudaSuccess) return FCFS_OK;
                if (e != cudaErrorInvalidValue) return cuda_fail(e, "forward (register-blocked) launch");
            }
            cudaError_t e = launch_forward_tma(T, ntk, d->dtype_in, d->dtype_out, st);
            return e == cudaSuccess ? FCFS_OK : cuda_fail(e, "forward (bulk-copy) launch");
        }
        clear_error();
    }
    TileChoice g = t;
    if (t.tma == 1) g = default_tiles(P, is3d);
    apply_tiles(P, is3d, g.WX, g.WY, g.WD, t.tma == 1 ? 0 : t.G);
    return launch_planned(P, ntk, is3d, d->dtype_in, d->dtype_out, st);
}

}  // namespace fcfs
