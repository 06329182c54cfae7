/*
 * FP64 CPU oracle for Fully Convolutional Fractional Scaling (FCFS,
 * Soloveitchik & Werman, arXiv 2203.10670).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the library never does, and it
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything is double precision, loops are written out, nothing is blocked,
 * fused or reordered.  OpenMP only splits independent (n, c) planes (or
 * channels, for the weight gradient) across threads.
 *
 * Tensor layout: [n][c][e0][e1][e2], row-major, last axis fastest.  Fewer than
 * three spatial axes are handled by prepending identity axes of extent 1
 * (r = s = 1, one tap of weight 1), which leaves every sum unchanged.
 *
 * What is computed (per spatial axis, readings of the paper in brackets):
 *   - output length No = floor(N r / s)                     [Sec. 3.1.1 "Description"; floor reading]
 *   - output o samples the input at p = o s / r             [Sec. 3.1: phase j of window i at i + j/r, stride units]
 *   - direct formula: y(p) = sum_t k(p - t) x~[t]           [Sec. 5.2, bilinear and Keys kernels]
 *     nearest: x~[floor(p + 1/2)] in exact integers         [Sec. 5.2.1 examples: rounding, ties upward]
 *   - sample-alignment variants (not the paper's; the conventions of common
 *     resize libraries), fixed methods only:
 *       half-pixel centres p = (o + 1/2) s / r - 1/2, nearest x~[floor((o + 1/2) s / r)]
 *       floor nearest x~[floor(o s / r)] (linear/cubic as the paper's p)
 *     and the Keys parameter a (the paper's kernel has a = -1/2).
 *   - antialiased downscale (not the paper's: the paper's kernels keep their
 *     width when s > r), fixed bilinear / bicubic only, when s > r: output o
 *     with sample position p takes every input t with |t - p| < R s / r
 *     (R = 1 bilinear, 2 bicubic) with weight k((t - p) r / s), the weights
 *     divided by their sum.  The kernel stretched by s / r is the low-pass
 *     prefilter of common resize libraries' antialias mode.
 *   - polyphase form with explicit weights W[j][m]:
 *     y[i r + j] = sum_m W[j][m] x~[i s - L + m]            [Sec. 3.1 pseudocode: pad, conv(stride s, r outputs), pixelshuffle]
 *     window half width K >= K_min, T = 2K + 1, L = K - floor(s/2)
 *   - x~ is the padded (extended) signal: replicate, constant, reflect [Sec. 3 "Stride, Padding & Pixelshuffle"]
 *   - ND: tensor product of the per-axis weights, ND extension  [Sec. 4, ND FCFS]
 *   - adjoint (input gradient) and weight gradient of the polyphase form
 *     (the paper's Sec. 7 "learn the weights" remark needs both).
 *
 * Parity notes: the printed bicubic 3x3 matrices of Sec. 5.2.3 are not
 * reproduced by any Keys weight vector; they are not used (parity unpinned
 * for those printed values only).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_NEAREST = 0, ORC_BILINEAR = 1, ORC_BICUBIC = 2 };
enum { ORC_PAD_REPLICATE = 0, ORC_PAD_CONSTANT = 1, ORC_PAD_REFLECT = 2 };
enum { ORC_ALIGN_PAPER = 0, ORC_ALIGN_HALF_PIXEL = 1, ORC_ALIGN_FLOOR = 2 };

typedef struct {
    int r, s;         /* scale factor r/s on this axis */
    int method;       /* ORC_NEAREST / ORC_BILINEAR / ORC_BICUBIC */
    int K;            /* polyphase half width, T = 2K+1; 0 -> K_min(method, s) */
    const double* w;  /* polyphase weights [C or 1][r][T]; NULL -> the method's table */
    int w_per_channel;
    int align;        /* ORC_ALIGN_*: sample positions of the fixed methods */
    double cubic_a;   /* Keys parameter of bicubic; 0 -> -1/2 */
    int antialias;    /* 1: widened, renormalised kernel when s > r (bilinear / bicubic) */
} orc_axis;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- kernels */

/* Interpolation kernel of Sec. 5.2.  Bilinear: the hat max(0, 1-|t|).
 * Bicubic: Keys' cubic convolution kernel with a = -0.5, whose constant term
 * -4a on 1<|t|<2 is +2. Nearest has no continuous kernel here (NAN). */
double orc_kernel_a(int method, double t, double ka) {
    double a = fabs(t);
    if (method == ORC_BILINEAR) return a < 1.0 ? 1.0 - a : 0.0;
    if (method == ORC_BICUBIC) {
        if (a <= 1.0) return (ka + 2.0) * a * a * a - (ka + 3.0) * a * a + 1.0;
        if (a < 2.0) return ka * a * a * a - 5.0 * ka * a * a + 8.0 * ka * a - 4.0 * ka;
        return 0.0;
    }
    return NAN;
}

double orc_kernel(int method, double t) { return orc_kernel_a(method, t, -0.5); }

/* support radius R: the kernel is zero for |t| >= R (nearest picks one of 2 taps) */
int orc_support(int method) { return method == ORC_BICUBIC ? 2 : 1; }

long long orc_floor_div(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* output length along one axis: floor(N r / s) */
long long orc_out_len(long long n, int r, int s) { return orc_floor_div(n * (long long)r, s); }

/* smallest K whose window [i s - L, i s - L + 2K] holds every tap any phase uses */
int orc_kmin(int method, int s) {
    int R = orc_support(method);
    return (int)orc_floor_div(s + 2 * R - 2 + 1, 2); /* ceil((s + 2R - 2) / 2) */
}

int orc_left_offset(int K, int s) { return K - s / 2; }

long long orc_num_windows(long long n_out, int r) { return orc_floor_div(n_out + r - 1, r); }

/* Extension rule (padding) on one axis: index into [0, n) or -1 for the constant value. */
long long orc_ext_index(long long q, long long n, int pad) {
    if (q >= 0 && q < n) return q;
    if (pad == ORC_PAD_CONSTANT) return -1;
    if (pad == ORC_PAD_REPLICATE) return q < 0 ? 0 : n - 1;
    /* reflect without repeating the edge sample: period 2(n-1) */
    if (n == 1) return 0;
    long long p = 2 * (n - 1);
    long long m = q % p;
    if (m < 0) m += p;
    return m < n ? m : p - m;
}

/* a1: dense table W[j][m] = k(j s / r - (m - L)), j < r, m < 2K+1.
 * Nearest: one-hot at m = floor((2 j s + r) / (2 r)) + L.  Returns -1 if K < K_min. */
int orc_make_weights(int method, int r, int s, int K, double* w) {
    if (K == 0) K = orc_kmin(method, s);
    if (K < orc_kmin(method, s)) return -1;
    int T = 2 * K + 1, L = orc_left_offset(K, s);
    for (int j = 0; j < r; ++j)
        for (int m = 0; m < T; ++m) {
            double v;
            if (method == ORC_NEAREST) {
                long long near = orc_floor_div(2LL * j * s + r, 2LL * r);
                v = (m == near + L) ? 1.0 : 0.0;
            } else {
                /* distance between the sample j s / r and the tap m - L, in input pixels */
                double delta = (double)((long long)j * s - (long long)(m - L) * r) / (double)r;
                v = orc_kernel(method, delta);
            }
            w[j * T + m] = v;
        }
    return K;
}

/* ------------------------------------------------------------- geometry */

typedef struct {
    long long n_in, n_out, n_win;
    int r, s, method, K, T, L, per_channel;
    int align;       /* ORC_ALIGN_* (fixed methods) */
    double cubic_a;  /* Keys parameter */
    int antialias;   /* the widened kernel applies (s > r, bilinear or bicubic) */
    const double* w; /* polyphase weights (may be the method table) */
} axis_t;

/* the fixed-method table of this axis describes it exactly (paper alignment, a = -1/2, no antialias) */
static int table_exact(const axis_t* A) {
    return A->align == ORC_ALIGN_PAPER && A->cubic_a == -0.5 && !A->antialias;
}

#define MAXTAP 256

static int setup_axes(int ndim, const long long* in_shape, const orc_axis* ax, axis_t out[3],
                      double* tables[3]) {
    int lead = 3 - ndim;
    for (int a = 0; a < 3; ++a) tables[a] = NULL;
    if (ndim < 1 || ndim > 3) return -1;
    for (int a = 0; a < 3; ++a) {
        axis_t* A = &out[a];
        if (a < lead) { /* identity axis of extent 1 */
            A->n_in = 1; A->r = 1; A->s = 1; A->method = ORC_NEAREST;
            A->K = 0; A->T = 1; A->L = 0; A->per_channel = 0;
            A->align = ORC_ALIGN_PAPER; A->cubic_a = -0.5; A->antialias = 0;
            tables[a] = (double*)malloc(sizeof(double));
            tables[a][0] = 1.0;
            A->w = tables[a];
        } else {
            const orc_axis* g = &ax[a - lead];
            A->n_in = in_shape[a - lead];
            A->r = g->r; A->s = g->s; A->method = g->method;
            A->K = g->K ? g->K : orc_kmin(g->method, g->s);
            A->T = 2 * A->K + 1;
            if (A->T > MAXTAP) return -1;
            A->L = orc_left_offset(A->K, A->s);
            A->per_channel = g->w ? g->w_per_channel : 0;
            if (g->align < ORC_ALIGN_PAPER || g->align > ORC_ALIGN_FLOOR) return -1;
            A->align = g->align;
            A->cubic_a = g->cubic_a != 0.0 ? g->cubic_a : -0.5;
            if (g->antialias != 0 && g->antialias != 1) return -1;
            A->antialias = g->antialias && !g->w && g->method != ORC_NEAREST && g->s > g->r;
            /* taps of a widened window: fewer than 2 R (s / r + 1) + 3 */
            if (A->antialias && 2LL * orc_support(g->method) * (g->s / g->r + 1) + 3 > MAXTAP) return -1;
            if (g->w) {
                A->w = g->w;
            } else {
                tables[a] = (double*)malloc(sizeof(double) * (size_t)A->r * A->T);
                if (orc_make_weights(A->method, A->r, A->s, A->K, tables[a]) < 0) return -1;
                A->w = tables[a];
            }
        }
        A->n_out = orc_out_len(A->n_in, A->r, A->s);
        A->n_win = orc_num_windows(A->n_out, A->r);
    }
    return 0;
}

static void free_tables(double* tables[3]) {
    for (int a = 0; a < 3; ++a) free(tables[a]);
}

/* taps of the direct formula at output o.  The sample position is the exact
 * rational p = num / den:
 *   paper (and floor)  p = o s / r                 num = o s,           den = r
 *   half-pixel         p = (o + 1/2) s / r - 1/2   num = 2 o s + s - r,  den = 2 r
 * nearest: paper floor(p + 1/2), floor floor(o s / r), half-pixel floor((o + 1/2) s / r) */
static int taps_direct(const axis_t* A, long long o, long long* t, double* w) {
    long long os = o * (long long)A->s;
    if (A->method == ORC_NEAREST) {
        if (A->align == ORC_ALIGN_FLOOR) t[0] = orc_floor_div(os, A->r);
        else if (A->align == ORC_ALIGN_HALF_PIXEL) t[0] = orc_floor_div(2 * os + A->s, 2LL * A->r);
        else t[0] = orc_floor_div(2 * os + A->r, 2LL * A->r); /* floor(p + 1/2) */
        w[0] = 1.0;
        return 1;
    }
    long long num = os, den = A->r;
    if (A->align == ORC_ALIGN_HALF_PIXEL) {
        num = 2 * os + A->s - A->r;
        den = 2LL * A->r;
    }
    int R = orc_support(A->method);
    long long b = orc_floor_div(num, den); /* floor(p) */
    int n = 0;
    if (A->antialias) {
        /* every q with |q - p| < R s / r, i.e. |q den - num| r < R s den (exact integers);
         * weight k((q - p) r / s), then divided by the sum of the weights */
        long long reach = (long long)R * ((A->s + A->r - 1) / A->r) + 1;
        double sum = 0.0;
        for (long long q = b - reach; q <= b + reach; ++q) {
            long long d = q * den - num;
            if ((d < 0 ? -d : d) * (long long)A->r >= (long long)R * A->s * den) continue;
            t[n] = q;
            w[n] = orc_kernel_a(A->method, (double)(d * A->r) / (double)(den * A->s), A->cubic_a);
            sum += w[n];
            ++n;
        }
        for (int k = 0; k < n; ++k) w[k] /= sum;
        return n;
    }
    for (long long q = b - R + 1; q <= b + R; ++q) {
        t[n] = q;
        w[n] = orc_kernel_a(A->method, (double)(num - q * den) / (double)den, A->cubic_a); /* k(p - q) */
        ++n;
    }
    return n;
}

/* taps of the polyphase form at output o = i r + j: window origin i s - L */
static int taps_poly(const axis_t* A, long long o, long long c, long long* t, double* w) {
    long long i = o / A->r;
    int j = (int)(o % A->r);
    const double* W = A->w + (A->per_channel ? c * (long long)A->r * A->T : 0) + (long long)j * A->T;
    for (int m = 0; m < A->T; ++m) {
        t[m] = i * A->s - A->L + m;
        w[m] = W[m];
    }
    return A->T;
}

/* ND sum over the tensor product of per-axis taps, with the ND extension */
static double nd_sum(const axis_t ax[3], const double* plane, int pad, double pad_value,
                     int n0, const long long* t0, const double* w0,
                     int n1, const long long* t1, const double* w1,
                     int n2, const long long* t2, const double* w2) {
    double acc = 0.0;
    for (int a = 0; a < n0; ++a) {
        long long q0 = orc_ext_index(t0[a], ax[0].n_in, pad);
        for (int b = 0; b < n1; ++b) {
            long long q1 = orc_ext_index(t1[b], ax[1].n_in, pad);
            for (int c = 0; c < n2; ++c) {
                long long q2 = orc_ext_index(t2[c], ax[2].n_in, pad);
                double v;
                if (q0 < 0 || q1 < 0 || q2 < 0) v = pad_value;
                else v = plane[(q0 * ax[1].n_in + q1) * ax[2].n_in + q2];
                acc += w0[a] * w1[b] * w2[c] * v;
            }
        }
    }
    return acc;
}

static double eval_one(const axis_t ax[3], int poly, const double* plane, long long c, int pad,
                       double pad_value, long long o0, long long o1, long long o2) {
    long long t0[MAXTAP], t1[MAXTAP], t2[MAXTAP];
    double w0[MAXTAP], w1[MAXTAP], w2[MAXTAP];
    int n0, n1, n2;
    if (poly) {
        n0 = taps_poly(&ax[0], o0, c, t0, w0);
        n1 = taps_poly(&ax[1], o1, c, t1, w1);
        n2 = taps_poly(&ax[2], o2, c, t2, w2);
    } else {
        n0 = taps_direct(&ax[0], o0, t0, w0);
        n1 = taps_direct(&ax[1], o1, t1, w1);
        n2 = taps_direct(&ax[2], o2, t2, w2);
    }
    return nd_sum(ax, plane, pad, pad_value, n0, t0, w0, n1, t1, w1, n2, t2, w2);
}

/* -------------------------------------------------------------- forward */

static int resize(int poly, int ndim, long long n, long long c, const long long* in_shape,
                  const orc_axis* axes, int pad, double pad_value, const double* x, double* y) {
    axis_t ax[3];
    double* tables[3];
    if (setup_axes(ndim, in_shape, axes, ax, tables) != 0) {
        free_tables(tables);
        return -1;
    }
    for (int a = 0; poly && a < 3; ++a)
        if (tables[a] && !table_exact(&ax[a])) { /* the method table is the paper's */
            free_tables(tables);
            return -1;
        }
    long long in_plane = ax[0].n_in * ax[1].n_in * ax[2].n_in;
    long long out_plane = ax[0].n_out * ax[1].n_out * ax[2].n_out;
    long long planes = n * c;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < planes; ++p) {
        const double* plane = x + p * in_plane;
        double* out = y + p * out_plane;
        long long ch = p % c;
        for (long long o0 = 0; o0 < ax[0].n_out; ++o0)
            for (long long o1 = 0; o1 < ax[1].n_out; ++o1)
                for (long long o2 = 0; o2 < ax[2].n_out; ++o2)
                    out[(o0 * ax[1].n_out + o1) * ax[2].n_out + o2] =
                        eval_one(ax, poly, plane, ch, pad, pad_value, o0, o1, o2);
    }
    free_tables(tables);
    return 0;
}

/* Fixed methods evaluated by the direct interpolation formula at p = o s / r. */
int orc_resize_direct(int ndim, long long n, long long c, const long long* in_shape,
                      const orc_axis* axes, int pad, double pad_value, const double* x, double* y) {
    return resize(0, ndim, n, c, in_shape, axes, pad, pad_value, x, y);
}

/* Pad -> strided conv with r phase kernels -> pixelshuffle, written as the polyphase sum. */
int orc_resize_polyphase(int ndim, long long n, long long c, const long long* in_shape,
                         const orc_axis* axes, int pad, double pad_value, const double* x, double* y) {
    return resize(1, ndim, n, c, in_shape, axes, pad, pad_value, x, y);
}

/* Evaluate chosen outputs only: idx holds flat output indices into [n][c][out...]. */
int orc_resize_at(int poly, int ndim, long long n, long long c, const long long* in_shape,
                  const orc_axis* axes, int pad, double pad_value, const double* x,
                  const long long* idx, long long count, double* out) {
    axis_t ax[3];
    double* tables[3];
    if (setup_axes(ndim, in_shape, axes, ax, tables) != 0) {
        free_tables(tables);
        return -1;
    }
    long long in_plane = ax[0].n_in * ax[1].n_in * ax[2].n_in;
    long long out_plane = ax[0].n_out * ax[1].n_out * ax[2].n_out;
    (void)n;
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < count; ++k) {
        long long f = idx[k];
        long long p = f / out_plane, r = f % out_plane;
        long long o2 = r % ax[2].n_out;
        long long o1 = (r / ax[2].n_out) % ax[1].n_out;
        long long o0 = r / (ax[2].n_out * ax[1].n_out);
        out[k] = eval_one(ax, poly, x + p * in_plane, p % c, pad, pad_value, o0, o1, o2);
    }
    free_tables(tables);
    return 0;
}

/* ------------------------------------------------------------- adjoints */

/* Input gradient of the polyphase form: the explicit transposed sum.  Every
 * output o and tap combination sends W-product * g[o] to the real input pixel
 * its extended index maps to (replicate/reflect fold; constant drops). */
int orc_adjoint_dx(int ndim, long long n, long long c, const long long* in_shape,
                   const orc_axis* axes, int pad, const double* g, double* dx) {
    axis_t ax[3];
    double* tables[3];
    if (setup_axes(ndim, in_shape, axes, ax, tables) != 0) {
        free_tables(tables);
        return -1;
    }
    int direct[3];
    for (int a = 0; a < 3; ++a) direct[a] = tables[a] != NULL && !table_exact(&ax[a]);
    long long in_plane = ax[0].n_in * ax[1].n_in * ax[2].n_in;
    long long out_plane = ax[0].n_out * ax[1].n_out * ax[2].n_out;
    long long planes = n * c;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < planes; ++p) {
        long long t0[MAXTAP], t1[MAXTAP], t2[MAXTAP];
        double w0[MAXTAP], w1[MAXTAP], w2[MAXTAP];
        double* d = dx + p * in_plane;
        const double* gp = g + p * out_plane;
        long long ch = p % c;
        for (long long k = 0; k < in_plane; ++k) d[k] = 0.0;
        for (long long o0 = 0; o0 < ax[0].n_out; ++o0)
            for (long long o1 = 0; o1 < ax[1].n_out; ++o1)
                for (long long o2 = 0; o2 < ax[2].n_out; ++o2) {
                    double gv = gp[(o0 * ax[1].n_out + o1) * ax[2].n_out + o2];
                    /* the polyphase taps, or the direct ones where a fixed method's
                     * alignment / Keys parameter is not its table's */
                    int n0 = direct[0] ? taps_direct(&ax[0], o0, t0, w0) : taps_poly(&ax[0], o0, ch, t0, w0);
                    int n1 = direct[1] ? taps_direct(&ax[1], o1, t1, w1) : taps_poly(&ax[1], o1, ch, t1, w1);
                    int n2 = direct[2] ? taps_direct(&ax[2], o2, t2, w2) : taps_poly(&ax[2], o2, ch, t2, w2);
                    for (int a = 0; a < n0; ++a) {
                        long long q0 = orc_ext_index(t0[a], ax[0].n_in, pad);
                        if (q0 < 0) continue;
                        for (int b = 0; b < n1; ++b) {
                            long long q1 = orc_ext_index(t1[b], ax[1].n_in, pad);
                            if (q1 < 0) continue;
                            for (int e = 0; e < n2; ++e) {
                                long long q2 = orc_ext_index(t2[e], ax[2].n_in, pad);
                                if (q2 < 0) continue;
                                d[(q0 * ax[1].n_in + q1) * ax[2].n_in + q2] += w0[a] * w1[b] * w2[e] * gv;
                            }
                        }
                    }
                }
    }
    free_tables(tables);
    return 0;
}

/* Per-axis list of (output index, weight) pairs that reach real input index q:
 * every extended index v with ext(v) == q, every window i whose taps cover v
 * (m = v + L - i s in [0, T)), every phase j with i r + j < No. */
static int adjoint_list(const axis_t* A, long long ch, int pad, long long q, long long* o, double* w,
                        int cap) {
    int n = 0;
    long long vmin = -A->L;
    long long vmax = (A->n_win - 1) * A->s - A->L + A->T - 1;
    for (long long v = vmin; v <= vmax; ++v) {
        if (orc_ext_index(v, A->n_in, pad) != q) continue;
        /* windows whose taps i s - L + m, m in [0, T), reach v */
        long long ilo = orc_floor_div(v + A->L - A->T + 1 + A->s - 1, A->s);
        long long ihi = orc_floor_div(v + A->L, A->s);
        if (ilo < 0) ilo = 0;
        if (ihi > A->n_win - 1) ihi = A->n_win - 1;
        for (long long i = ilo; i <= ihi; ++i) {
            long long m = v + A->L - i * A->s;
            if (m < 0 || m >= A->T) continue;
            for (int j = 0; j < A->r; ++j) {
                long long oo = i * A->r + j;
                if (oo >= A->n_out) continue;
                if (n >= cap) return -1;
                o[n] = oo;
                w[n] = A->w[(A->per_channel ? ch * (long long)A->r * A->T : 0) + (long long)j * A->T + m];
                ++n;
            }
        }
    }
    return n;
}

/* Gather form of the input gradient at chosen input pixels (flat indices into
 * [n][c][in...]).  Written independently of the scatter form above. */
int orc_adjoint_dx_at(int ndim, long long n, long long c, const long long* in_shape,
                      const orc_axis* axes, int pad, const double* g, const long long* idx,
                      long long count, double* out) {
    axis_t ax[3];
    double* tables[3];
    if (setup_axes(ndim, in_shape, axes, ax, tables) != 0) {
        free_tables(tables);
        return -1;
    }
    for (int a = 0; a < 3; ++a)
        if (tables[a] && !table_exact(&ax[a])) { /* gathered from the paper's tables only */
            free_tables(tables);
            return -1;
        }
    long long in_plane = ax[0].n_in * ax[1].n_in * ax[2].n_in;
    long long out_plane = ax[0].n_out * ax[1].n_out * ax[2].n_out;
    int bad = 0;
    (void)n;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long long k = 0; k < count; ++k) {
        enum { CAP = 4096 };
        long long *oa = (long long*)malloc(sizeof(long long) * 3 * CAP);
        double* wa = (double*)malloc(sizeof(double) * 3 * CAP);
        long long f = idx[k];
        long long p = f / in_plane, r = f % in_plane;
        long long q2 = r % ax[2].n_in;
        long long q1 = (r / ax[2].n_in) % ax[1].n_in;
        long long q0 = r / (ax[2].n_in * ax[1].n_in);
        long long ch = p % c;
        int n0 = adjoint_list(&ax[0], ch, pad, q0, oa, wa, CAP);
        int n1 = adjoint_list(&ax[1], ch, pad, q1, oa + CAP, wa + CAP, CAP);
        int n2 = adjoint_list(&ax[2], ch, pad, q2, oa + 2 * CAP, wa + 2 * CAP, CAP);
        double acc = 0.0;
        if (n0 < 0 || n1 < 0 || n2 < 0) {
            bad = 1;
        } else {
            const double* gp = g + p * out_plane;
            for (int a = 0; a < n0; ++a)
                for (int b = 0; b < n1; ++b)
                    for (int e = 0; e < n2; ++e)
                        acc += wa[a] * wa[CAP + b] * wa[2 * CAP + e] *
                               gp[(oa[a] * ax[1].n_out + oa[CAP + b]) * ax[2].n_out + oa[2 * CAP + e]];
        }
        out[k] = acc;
        free(oa);
        free(wa);
    }
    free_tables(tables);
    return bad ? -1 : 0;
}

/* Weight gradient of the polyphase form.  dw[a] (for the ndim real axes, in
 * order) receives [C or 1][r][T]:
 *   dW_a[c][j][m] = sum over n, outputs o with phase j on axis a, taps of the
 *                   other axes: g[o] * x~[taps] * prod_{b != a} W_b
 * Extended samples of the constant pad carry pad_value and contribute too. */
int orc_weight_grad(int ndim, long long n, long long c, const long long* in_shape,
                    const orc_axis* axes, int pad, double pad_value, const double* x,
                    const double* g, double** dw) {
    axis_t ax[3];
    double* tables[3];
    if (setup_axes(ndim, in_shape, axes, ax, tables) != 0) {
        free_tables(tables);
        return -1;
    }
    int lead = 3 - ndim;
    long long in_plane = ax[0].n_in * ax[1].n_in * ax[2].n_in;
    long long out_plane = ax[0].n_out * ax[1].n_out * ax[2].n_out;
    /* per-channel partial sums first (sum over n), then fold shared weights in channel order */
    size_t per_ch[3];
    double* part[3];
    for (int a = 0; a < 3; ++a) {
        per_ch[a] = (size_t)ax[a].r * ax[a].T;
        part[a] = (double*)calloc((size_t)c * per_ch[a], sizeof(double));
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (long long ch = 0; ch < c; ++ch) {
        long long t0[MAXTAP], t1[MAXTAP], t2[MAXTAP];
        double w0[MAXTAP], w1[MAXTAP], w2[MAXTAP];
        double* P0 = part[0] + ch * per_ch[0];
        double* P1 = part[1] + ch * per_ch[1];
        double* P2 = part[2] + ch * per_ch[2];
        for (long long b = 0; b < n; ++b) {
            long long p = b * c + ch;
            const double* plane = x + p * in_plane;
            const double* gp = g + p * out_plane;
            for (long long o0 = 0; o0 < ax[0].n_out; ++o0)
                for (long long o1 = 0; o1 < ax[1].n_out; ++o1)
                    for (long long o2 = 0; o2 < ax[2].n_out; ++o2) {
                        double gv = gp[(o0 * ax[1].n_out + o1) * ax[2].n_out + o2];
                        int j0 = (int)(o0 % ax[0].r), j1 = (int)(o1 % ax[1].r), j2 = (int)(o2 % ax[2].r);
                        int n0 = taps_poly(&ax[0], o0, ch, t0, w0);
                        int n1 = taps_poly(&ax[1], o1, ch, t1, w1);
                        int n2 = taps_poly(&ax[2], o2, ch, t2, w2);
                        for (int a0 = 0; a0 < n0; ++a0) {
                            long long q0 = orc_ext_index(t0[a0], ax[0].n_in, pad);
                            for (int a1 = 0; a1 < n1; ++a1) {
                                long long q1 = orc_ext_index(t1[a1], ax[1].n_in, pad);
                                for (int a2 = 0; a2 < n2; ++a2) {
                                    long long q2 = orc_ext_index(t2[a2], ax[2].n_in, pad);
                                    double v;
                                    if (q0 < 0 || q1 < 0 || q2 < 0) v = pad_value;
                                    else v = plane[(q0 * ax[1].n_in + q1) * ax[2].n_in + q2];
                                    double gx = gv * v;
                                    P0[j0 * ax[0].T + a0] += gx * w1[a1] * w2[a2];
                                    P1[j1 * ax[1].T + a1] += gx * w0[a0] * w2[a2];
                                    P2[j2 * ax[2].T + a2] += gx * w0[a0] * w1[a1];
                                }
                            }
                        }
                    }
        }
    }
    for (int a = lead; a < 3; ++a) {
        double* out = dw[a - lead];
        if (!out) continue;
        if (ax[a].per_channel) {
            memcpy(out, part[a], sizeof(double) * (size_t)c * per_ch[a]);
        } else {
            for (size_t k = 0; k < per_ch[a]; ++k) out[k] = 0.0;
            for (long long ch = 0; ch < c; ++ch)
                for (size_t k = 0; k < per_ch[a]; ++k) out[k] += part[a][ch * per_ch[a] + k];
        }
    }
    for (int a = 0; a < 3; ++a) free(part[a]);
    free_tables(tables);
    return 0;
}

/* ------------------------------------------------- non-separable 2D kernels */

/* Full (non-separable) 2D kernels, the ND convolution of Sec. 4 with one
 * learnable T_y x T_x kernel per phase pair instead of an outer product:
 *   y[n,c, iy r_y + jy, ix r_x + jx] = sum_{my, mx} W[c][jy][jx][my][mx]
 *                                      x~[n,c, iy s_y - L_y + my, ix s_x - L_x + mx]
 * W is [C][r_y][r_x][T_y][T_x] (per_channel) or [r_y][r_x][T_y][T_x];
 * T_a = 2 K_a + 1, L_a = K_a - floor(s_a / 2), K_a from the axis (0 -> K_min of
 * its method).  x~ is the padded input (constant pad samples carry pad_value). */
typedef struct {
    long long n_in, n_out;
    int r, s, K, T, L;
} full_axis_t;

static int full_axes(const long long* in_shape, const orc_axis* axes, full_axis_t f[2]) {
    for (int a = 0; a < 2; ++a) {
        const orc_axis* g = &axes[a];
        if (g->r < 1 || g->s < 1) return -1;
        f[a].n_in = in_shape[a];
        f[a].r = g->r;
        f[a].s = g->s;
        f[a].K = g->K ? g->K : orc_kmin(g->method, g->s);
        f[a].T = 2 * f[a].K + 1;
        f[a].L = orc_left_offset(f[a].K, f[a].s);
        f[a].n_out = orc_out_len(f[a].n_in, f[a].r, f[a].s);
    }
    return 0;
}

static double full_weight(const full_axis_t f[2], const double* w, int per_channel, long long ch, int jy, int jx,
                          int my, int mx) {
    long long per = (long long)f[0].r * f[1].r * f[0].T * f[1].T;
    return w[(per_channel ? ch * per : 0) + (((long long)jy * f[1].r + jx) * f[0].T + my) * f[1].T + mx];
}

int orc_resize_full2d(long long n, long long c, const long long* in_shape, const orc_axis* axes, const double* w,
                      int per_channel, int pad, double pad_value, const double* x, double* y) {
    full_axis_t f[2];
    if (full_axes(in_shape, axes, f) != 0) return -1;
    long long in_plane = f[0].n_in * f[1].n_in, out_plane = f[0].n_out * f[1].n_out;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < n * c; ++p) {
        long long ch = p % c;
        const double* plane = x + p * in_plane;
        for (long long oy = 0; oy < f[0].n_out; ++oy)
            for (long long ox = 0; ox < f[1].n_out; ++ox) {
                long long iy = oy / f[0].r, ix = ox / f[1].r;
                int jy = (int)(oy % f[0].r), jx = (int)(ox % f[1].r);
                double acc = 0.0;
                for (int my = 0; my < f[0].T; ++my) {
                    long long qy = orc_ext_index(iy * f[0].s - f[0].L + my, f[0].n_in, pad);
                    for (int mx = 0; mx < f[1].T; ++mx) {
                        long long qx = orc_ext_index(ix * f[1].s - f[1].L + mx, f[1].n_in, pad);
                        double v = (qy < 0 || qx < 0) ? pad_value : plane[qy * f[1].n_in + qx];
                        acc += full_weight(f, w, per_channel, ch, jy, jx, my, mx) * v;
                    }
                }
                y[p * out_plane + oy * f[1].n_out + ox] = acc;
            }
    }
    return 0;
}

/* Input gradient: the transposed sum, every output sending W * g to the real
 * pixel its extended tap maps to (replicate / reflect fold, constant drops). */
int orc_adjoint_full2d(long long n, long long c, const long long* in_shape, const orc_axis* axes, const double* w,
                       int per_channel, int pad, const double* g, double* dx) {
    full_axis_t f[2];
    if (full_axes(in_shape, axes, f) != 0) return -1;
    long long in_plane = f[0].n_in * f[1].n_in, out_plane = f[0].n_out * f[1].n_out;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < n * c; ++p) {
        long long ch = p % c;
        double* d = dx + p * in_plane;
        for (long long k = 0; k < in_plane; ++k) d[k] = 0.0;
        for (long long oy = 0; oy < f[0].n_out; ++oy)
            for (long long ox = 0; ox < f[1].n_out; ++ox) {
                long long iy = oy / f[0].r, ix = ox / f[1].r;
                int jy = (int)(oy % f[0].r), jx = (int)(ox % f[1].r);
                double gv = g[p * out_plane + oy * f[1].n_out + ox];
                for (int my = 0; my < f[0].T; ++my) {
                    long long qy = orc_ext_index(iy * f[0].s - f[0].L + my, f[0].n_in, pad);
                    if (qy < 0) continue;
                    for (int mx = 0; mx < f[1].T; ++mx) {
                        long long qx = orc_ext_index(ix * f[1].s - f[1].L + mx, f[1].n_in, pad);
                        if (qx < 0) continue;
                        d[qy * f[1].n_in + qx] += full_weight(f, w, per_channel, ch, jy, jx, my, mx) * gv;
                    }
                }
            }
    }
    return 0;
}

/* Weight gradient: dW[c][jy][jx][my][mx] = sum over n and windows of
 * g[iy r_y + jy][ix r_x + jx] x~[iy s_y - L_y + my][ix s_x - L_x + mx]
 * (summed over channels, in channel order, when the kernel is shared). */
int orc_weight_grad_full2d(long long n, long long c, const long long* in_shape, const orc_axis* axes, int per_channel,
                           int pad, double pad_value, const double* x, const double* g, double* dw) {
    full_axis_t f[2];
    if (full_axes(in_shape, axes, f) != 0) return -1;
    long long in_plane = f[0].n_in * f[1].n_in, out_plane = f[0].n_out * f[1].n_out;
    long long per = (long long)f[0].r * f[1].r * f[0].T * f[1].T;
    double* part = (double*)calloc((size_t)(c * per), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (long long ch = 0; ch < c; ++ch) {
        double* P = part + ch * per;
        for (long long b = 0; b < n; ++b) {
            long long p = b * c + ch;
            const double* plane = x + p * in_plane;
            for (long long oy = 0; oy < f[0].n_out; ++oy)
                for (long long ox = 0; ox < f[1].n_out; ++ox) {
                    long long iy = oy / f[0].r, ix = ox / f[1].r;
                    int jy = (int)(oy % f[0].r), jx = (int)(ox % f[1].r);
                    double gv = g[p * out_plane + oy * f[1].n_out + ox];
                    for (int my = 0; my < f[0].T; ++my) {
                        long long qy = orc_ext_index(iy * f[0].s - f[0].L + my, f[0].n_in, pad);
                        for (int mx = 0; mx < f[1].T; ++mx) {
                            long long qx = orc_ext_index(ix * f[1].s - f[1].L + mx, f[1].n_in, pad);
                            double v = (qy < 0 || qx < 0) ? pad_value : plane[qy * f[1].n_in + qx];
                            P[(((long long)jy * f[1].r + jx) * f[0].T + my) * f[1].T + mx] += gv * v;
                        }
                    }
                }
        }
    }
    if (per_channel) {
        memcpy(dw, part, sizeof(double) * (size_t)(c * per));
    } else {
        for (long long e = 0; e < per; ++e) {
            double s = 0.0;
            for (long long ch = 0; ch < c; ++ch) s += part[ch * per + e];
            dw[e] = s;
        }
    }
    free(part);
    return 0;
}
