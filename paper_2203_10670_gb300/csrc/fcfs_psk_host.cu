// Host planning of the polyphase strip kernels (fcfs_psk.cuh): the 2D
// forward of Sec. 3.1 / Sec. 4 and the interior of its input gradient.
//
// Forward: the layer's own tables, every output.  Input gradient: the adjoint
// of each axis in its polyphase form (window a has s phases u, outputs
// v = a s + lo_out + u, phase u reads g at a r + lo_in + off[u] + t) run on the
// upstream gradient g, for the adjoint windows whose outputs are real indices
// that receive no folded padding contribution; the border bands around that
// interior (a few rows and columns per edge) go to the gather kernel, which
// folds the padding adjoint.
#include <climits>
#include <cstdlib>
#include <cstring>

#include <algorithm>

#include "fcfs_host.h"
#include "fcfs_psk.cuh"

namespace fcfs {

cudaError_t launch_psk_f32(const PskParams& P, int R, int S, int span, size_t smem, cudaStream_t st);
cudaError_t launch_psk_bf16(const PskParams& P, int R, int S, int span, size_t smem, cudaStream_t st);
bool psk_compiled(int R, int S, int span);

// Policy of the strip kernels, from FCFS_STRIP_KERNELS: unset = default (the
// input gradient where no register-blocked tile kernel is compiled for the
// adjoint's window shape, and a candidate of the forward tile search);
// 0 = never; 1 = wherever a descriptor is in their scope (used by the tests
// to cover every compiled shape).
int psk_policy() {
    static const int v = [] {
        const char* e = getenv("FCFS_STRIP_KERNELS");
        if (e && e[0] == '0') return 0;
        if (e && e[0] == '1') return 2;
        return 1;
    }();
    return v;
}

bool psk_enabled() { return psk_policy() != 0; }

namespace {

constexpr int kNS = 4;  // stages

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

// Tiling, shared-memory layout and launch of a strip pass whose axes and
// weights are set.  Returns -1 when the shape is outside the kernels' scope.
int psk_launch(PskParams& P, int R, int span, int dt, cudaStream_t st) {
    const int es = dt == FCFS_F32 ? 4 : 2;
    const int NTH = kPskWarps * 32;
    const int S = P.ax.s;
    if (P.ay.s != S || span <= S) return -1;
    const long long nwx = (long long)P.ax.w1 - P.ax.w0, nwy = (long long)P.ay.w1 - P.ay.w0;
    if (nwx < 1 || nwy < 1) return -1;
    P.al = 16 / es;
    // stage chunks: whole window steps, about six rows; the first chunk holds the span - s
    // rows before the first step
    P.CH = S * std::max(1, (6 + S - 1) / S);
    if (span - S > P.CH || P.CH > 32) return -1;
    P.NS = kNS;
    // vector window loads when a window stride spans 8 or 16 bytes and windows start on them
    P.xvec = 0;
    for (int vb : {16, 8}) {
        const int sb = S * es, lb = ((P.ax.lo * es) % vb + vb) % vb;
        if (sb % vb == 0 && lb == 0) {
            P.xvec = vb;
            break;
        }
    }
    const int E = P.xvec ? P.xvec / es : 1;
    const int spanv = (span + E - 1) / E * E;
    P.strip_w = NTH;
    P.nstrips = (int)((nwx + P.strip_w - 1) / P.strip_w);
    const int need = (P.al - 1) + (P.strip_w - 1) * S + spanv;
    P.pitch = (need + P.al - 1) / P.al * P.al;
    // columns outside the input are read through the padding rule: their targets must be staged
    if (P.pad != FCFS_PAD_CONSTANT) {
        const int W = P.ax.n_in;
        for (int sidx = 0; sidx < P.nstrips; ++sidx) {
            const int wxa = P.ax.w0 + sidx * P.strip_w;
            const int nw = std::min(P.strip_w, P.ax.w1 - wxa);
            const int c0 = wxa * S + P.ax.lo;
            const int x_al = c0 >= 0 ? c0 / P.al * P.al : -((-c0 + P.al - 1) / P.al) * P.al;
            const int ca = std::max(x_al, 0), cb = std::min(x_al + P.pitch, W);
            if (c0 >= 0 && c0 + (nw - 1) * S + span <= W) continue;
            for (int c = c0; c < c0 + (nw - 1) * S + span; ++c) {
                const int m = (c >= 0 && c < W) ? c : ext_index(c, W, P.pad);
                if (m < ca || m >= cb) return -1;
            }
        }
    }
    const int spxp = (span + 3) / 4 * 4;
    const size_t stage = (size_t)P.CH * P.pitch * es;
    size_t off = (size_t)kNS * stage;
    P.w_off = (int)off;
    off += (size_t)kPskWarps * ((R * spxp + R * span + 3) / 4 * 4) * 4;
    P.flag_off = (int)off;
    off += (size_t)kNS * P.CH * 4;
    off = (off + 15) / 16 * 16;
    P.bar_off = (int)off;
    const size_t smem = off + 2 * kNS * 8;
    if (smem > 200 * 1024) return -1;
    // bands: the persistent grid's time is (tiles per CTA) x (rows per band), and a grid with fewer
    // tiles than resident CTA slots leaves the rest of the machine idle (the kernel is latency-bound
    // per CTA), so a short tile list is charged for its empty slots
    const int regs_ctas = (R * span <= 12 && R <= 3) ? 4 : 3;
    const int smem_ctas = (int)std::max<size_t>(1, (227 * 1024) / (smem + 1024));
    const long long cap = (long long)sm_count() * std::min(regs_ctas, smem_ctas);
    const long long base = P.planes * P.nstrips;
    long long best = LLONG_MAX;
    int best_h = (int)nwy;
    for (long long nb = 1; nb <= std::min<long long>(nwy, 256); ++nb) {
        const long long h = (nwy + nb - 1) / nb;
        const long long nbe = (nwy + h - 1) / h;
        const long long tiles = base * nbe;
        const long long per = (tiles + cap - 1) / cap;
        long long cost = per * ((h - 1) * S + span);
        if (tiles < cap) cost = cost * cap / tiles;
        if (cost < best) {
            best = cost;
            best_h = (int)h;
        }
    }
    P.band_h = best_h;
    P.nbands = (int)((nwy + best_h - 1) / best_h);
    const long long ntiles = base * P.nbands;
    if (ntiles >= INT_MAX) return -1;
    P.ntiles = (int)ntiles;
    cudaError_t e =
        dt == FCFS_F32 ? launch_psk_f32(P, R, S, span, smem, st) : launch_psk_bf16(P, R, S, span, smem, st);
    if (e == cudaErrorInvalidValue) return -1;
    return e == cudaSuccess ? FCFS_OK : cuda_fail(e, "strip kernel launch");
}

// Span-form table of one forward axis: entry (j, k) is the weight of input
// position k of the window for phase j.
void forward_span_table(const AxisP& A, int span, float* wf, short* wi) {
    for (int j = 0; j < A.r; ++j)
        for (int k = 0; k < span; ++k) {
            const int t = k - A.off[j];
            const bool in = t >= 0 && t < A.nt_src;
            wf[j * span + k] = in && !A.learn ? A.wf[j * A.nt_src + t] : 0.f;
            wi[j * span + k] = in ? (short)(j * A.nt_src + t) : (short)-1;
        }
}

// Span-form table of one adjoint axis: entry (u, k) is the forward weight
// that g position k of the adjoint window carries into phase u.
void adjoint_span_table(const AxisP& A, const AdjP& J, int span, float* wf, short* wi) {
    for (int u = 0; u < J.s; ++u)
        for (int k = 0; k < span; ++k) {
            const int t = k - J.off[u];
            int f = -1;
            if (t >= 0 && t < J.ntu[u]) f = J.idx[u * kMaxAdjTaps + t];
            wf[u * span + k] = f >= 0 && !A.learn ? A.wf[f] : 0.f;
            wi[u * span + k] = (short)f;
        }
}

int true_adj_span(const AdjP& J) {
    int sp = 0;
    for (int u = 0; u < J.s; ++u) sp = std::max(sp, J.off[u] + J.ntu[u]);
    return sp;
}

}  // namespace

int psk_forward(const fcfs_desc* d, const FwdParams& F, cudaStream_t st) {
    if (!psk_enabled() || d->ndim != 2 || d->dtype_in != d->dtype_out) return -1;
    if (d->dtype_in != FCFS_F32 && d->dtype_in != FCFS_BF16) return -1;
    const AxisP &AX = F.ax[2], &AY = F.ax[1];
    if (AX.r != AY.r || AX.s != AY.s || AX.span != AY.span || !psk_compiled(AX.r, AX.s, AX.span)) return -1;
    if (AX.r * AX.span > kPskMaxW) return -1;
    if (!AX.learn && !AY.learn && AX.nt_src == 1 && AY.nt_src == 1) return -1;  // one-tap copy: own kernel
    const int es = dtype_size(d->dtype_in);
    if (((uintptr_t)F.x) % 16 || ((long long)AX.n_in * es) % 16) return -1;
    PskParams P;
    memset(&P, 0, sizeof P);
    P.ay = PskAxis{AY.s, AY.lo, AY.n_in, AY.n_out, 0, 0, AY.n_win};
    P.ax = PskAxis{AX.s, AX.lo, AX.n_in, AX.n_out, 0, 0, AX.n_win};
    P.planes = F.planes;
    P.C = F.C;
    P.pad = F.pad;
    P.padv = F.padv;
    P.in = F.x;
    P.out = F.y;
    P.learn_x = AX.learn;
    P.learn_y = AY.learn;
    P.wl_x = AX.w;
    P.wl_y = AY.w;
    P.wcs_x = AX.w_cstride;
    P.wcs_y = AY.w_cstride;
    forward_span_table(AX, AX.span, P.wf_x, P.wi_x);
    forward_span_table(AY, AY.span, P.wf_y, P.wi_y);
    P.epi = F.epi;
    return psk_launch(P, AX.r, AX.span, d->dtype_in, st);
}

int psk_input_gradient(const fcfs_desc* d, const BwdParams& B, const void* gy, void* gx, int ntk, cudaStream_t st) {
    if (!psk_enabled() || d->ndim != 2 || d->dtype_in != d->dtype_out) return -1;
    if (d->dtype_in != FCFS_F32 && d->dtype_in != FCFS_BF16) return -1;
    const int es = dtype_size(d->dtype_out);
    const AxisP &AX = B.ax[2], &AY = B.ax[1];
    if (((uintptr_t)gy) % 16 || ((long long)AX.n_out * es) % 16) return -1;
    AdjP JX, JY;
    if (build_adjp(AX, &JX) < 0 || build_adjp(AY, &JY) < 0) return -1;
    const int span = true_adj_span(JX);
    if (JX.s != JY.s || JX.r != JY.r || true_adj_span(JY) != span || !psk_compiled(JX.s, JX.r, span)) return -1;
    if (JX.s * span > kPskMaxW) return -1;
    // interior adjoint windows of one axis: every output a real index that no folded
    // padding contribution reaches
    auto interior = [&](const AdjP& J, int* a0, int* a1) {
        const int N = J.n_x, S = J.s;
        int fl = 0, fr = 0;
        if (d->pad != FCFS_PAD_CONSTANT) {
            if (J.vmin < 0) fl = d->pad == FCFS_PAD_REPLICATE ? 1 : -J.vmin + 1;
            if (J.vmax >= N) fr = d->pad == FCFS_PAD_REPLICATE ? 1 : J.vmax - N + 2;
        }
        // reflection farther than one period is left to the gather kernel
        if (d->pad == FCFS_PAD_REFLECT && (-J.vmin >= N - 1 || J.vmax - N + 1 >= N - 1)) return false;
        const int lo = fl - J.lo_out, hi = N - fr - J.lo_out - S;  // a S >= lo and a S <= hi
        *a0 = lo <= 0 ? -((-lo) / S) : (lo + S - 1) / S;
        *a1 = (hi >= 0 ? hi / S : -((-hi + S - 1) / S)) + 1;
        return *a1 - *a0 >= 1;
    };
    int ax0, ax1, ay0, ay1;
    if (!interior(JX, &ax0, &ax1) || !interior(JY, &ay0, &ay1)) return -1;
    PskParams P;
    memset(&P, 0, sizeof P);
    P.ax = PskAxis{JX.r, JX.lo_in, JX.n_g, JX.n_x, JX.lo_out, ax0, ax1};
    P.ay = PskAxis{JY.r, JY.lo_in, JY.n_g, JY.n_x, JY.lo_out, ay0, ay1};
    P.planes = B.planes;
    P.C = B.C;
    P.pad = FCFS_PAD_CONSTANT;  // g is zero outside the forward output
    P.padv = 0.f;
    P.in = gy;
    P.out = gx;
    P.learn_x = AX.learn;
    P.learn_y = AY.learn;
    P.wl_x = AX.w;
    P.wl_y = AY.w;
    P.wcs_x = AX.w_cstride;
    P.wcs_y = AY.w_cstride;
    adjoint_span_table(AX, JX, span, P.wf_x, P.wi_x);
    adjoint_span_table(AY, JY, span, P.wf_y, P.wi_y);
    int rc = psk_launch(P, JX.s, span, d->dtype_in, st);
    if (rc) return rc;
    // the border bands around the interior, with the padding adjoint folded in
    const int qx0 = ax0 * JX.s + JX.lo_out, qx1 = ax1 * JX.s + JX.lo_out;
    const int qy0 = ay0 * JY.s + JY.lo_out, qy1 = ay1 * JY.s + JY.lo_out;
    const int Nx = JX.n_x, Ny = JY.n_x;
    const int bands[4][4] = {{0, Nx, 0, qy0}, {0, Nx, qy1, Ny}, {0, qx0, qy0, qy1}, {qx1, Nx, qy0, qy1}};
    for (const auto& b : bands) {
        if (b[1] <= b[0] || b[3] <= b[2]) continue;
        BwdParams G = B;
        G.gy = gy;
        G.gx = gx;
        plan_dx(G, false);
        plan_dx_region(G, b[0], b[1], b[2], b[3]);
        const long long blocks = (long long)G.qtiles_x * G.qtiles_y * G.planes;
        if (blocks > INT_MAX || dx_smem_bytes(G, false) > 227 * 1024)
            return fail(FCFS_ERR_UNSUPPORTED, "input-gradient border tile too large");
        cudaError_t e = launch_dx(G, ntk, d->dtype_out, d->dtype_in, false, st);
        if (e != cudaSuccess) return cuda_fail(e, "input-gradient border launch");
    }
    return FCFS_OK;
}

}  // namespace fcfs
