// Dispatch of the bulk-copy forward over its per-input-type translation units.
#include "fcfs_internal.cuh"

namespace fcfs {

cudaError_t launch_forward_tma_f32(const TmaFwdParams& T, int nt, int din, int dout, cudaStream_t st);
cudaError_t launch_forward_tma_bf16(const TmaFwdParams& T, int nt, int din, int dout, cudaStream_t st);
cudaError_t launch_forward_tma_u8(const TmaFwdParams& T, int nt, int din, int dout, cudaStream_t st);
cudaError_t launch_forward_rs_f32(const TmaFwdParams& T, int R, int span, cudaStream_t st);
cudaError_t launch_forward_rs_bf16(const TmaFwdParams& T, int R, int span, cudaStream_t st);
int read_status_fwd_tma_f32(int clear);
int read_status_fwd_tma_bf16(int clear);
int read_status_fwd_tma_u8(int clear);
int read_status_fwd3d(int clear);
int read_status_fwd3d_rs(int clear);

cudaError_t launch_forward_tma(const TmaFwdParams& T, int nt, int din, int dout, cudaStream_t st) {
    if (din == FCFS_F32) return launch_forward_tma_f32(T, nt, din, dout, st);
    if (din == FCFS_BF16) return launch_forward_tma_bf16(T, nt, din, dout, st);
    if (din == FCFS_U8) return launch_forward_tma_u8(T, nt, din, dout, st);
    return cudaErrorInvalidValue;
}

// Register-blocked variant: same phase count and window span on both axes,
// interpolating taps (not the one-tap nearest copy), FP32 or BF16 storage.
bool forward_rs_available(const TmaFwdParams& T, int din, int dout) {
    const AxisP &AX = T.P.ax[2], &AY = T.P.ax[1];
    if (din != dout || (din != FCFS_F32 && din != FCFS_BF16)) return false;
    if (AX.r != AY.r || AX.span != AY.span || AX.nt_src < 2 || AY.nt_src < 2) return false;
    if (T.P.OX % 2 || AX.n_out % 2) return false;
    static const int pairs[][2] = {{2, 5}, {4, 6}, {3, 5}, {3, 3}, {5, 5}, {7, 8}};
    for (auto& pr : pairs)
        if (pr[0] == AX.r && pr[1] == AX.span) return true;
    return false;
}

cudaError_t launch_forward_rs(const TmaFwdParams& T, int din, cudaStream_t st) {
    const int R = T.P.ax[2].r, span = T.P.ax[2].span;
    return din == FCFS_F32 ? launch_forward_rs_f32(T, R, span, st) : launch_forward_rs_bf16(T, R, span, st);
}

size_t forward_tma_smem_bytes(const TmaFwdParams& T) { return (size_t)T.bar_off + 16; /* two mbarriers */ }

// status words of the bulk-copy forward translation units, or -1 if one cannot be read
int read_status_fwd_tma(int clear) {
    const int a = read_status_fwd_tma_f32(clear), b = read_status_fwd_tma_bf16(clear), c = read_status_fwd_tma_u8(clear);
    const int e = read_status_fwd3d(clear), f = read_status_fwd3d_rs(clear);
    if (a < 0 || b < 0 || c < 0 || e < 0 || f < 0) return -1;
    return a | b | c | e | f;
}

}  // namespace fcfs
