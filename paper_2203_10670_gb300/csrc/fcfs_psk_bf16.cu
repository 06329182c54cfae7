// Polyphase strip kernels (fcfs_psk.cuh) for __nv_bfloat16 input and output.
#define FCFS_PSK_KERNELS
#include "fcfs_psk.cuh"

namespace fcfs {

namespace {

template <int R, int S, int SPAN, int XV>
cudaError_t run_psk(const PskParams& P, size_t smem, cudaStream_t st) {
    auto k = fcfs_psk<R, S, SPAN, XV, __nv_bfloat16, __nv_bfloat16>;
    int sms = 0, per_sm = 0;
    cudaError_t e = resident_ctas((const void*)k, kPskThreads, smem, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(P.ntiles, (long long)sms * per_sm);
    k<<<(unsigned)grid, kPskThreads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

// (phases, stride, span) compiled, the same on both axes, with the x-pass vector load width
// (bytes, 0 = scalar) for FP32 and for BF16 storage: the forward of bicubic 2/3, 4/3, 3/2, 7/5,
// bilinear 3/2 and 5/4 (also learnable 5-tap 5/4); the input-gradient interiors (adjoint: s phases,
// stride r) of bicubic 2/3, 4/3, 3/2, 7/5, bilinear 3/2, 5/4 and learnable 5/4 (K = 2)
#define FCFS_PSK_CASES(X)                                                                                   \
    X(2, 3, 5, 0, 0) X(4, 3, 6, 0, 0) X(3, 2, 3, 8, 0) X(3, 2, 5, 0, 0) X(5, 4, 5, 16, 8) X(7, 5, 8, 0, 0) \
    X(3, 2, 4, 8, 0) X(3, 4, 8, 16, 8) X(2, 3, 4, 0, 0) X(2, 3, 7, 0, 0) X(4, 5, 10, 0, 0) X(5, 7, 11, 0, 0) \
    X(4, 5, 6, 0, 0)

cudaError_t launch_psk_bf16(const PskParams& P, int R, int S, int span, size_t smem, cudaStream_t st) {
#define CASE(a, b, c, d, e) \
    if (R == a && S == b && span == c && P.xvec == e) return run_psk<a, b, c, e>(P, smem, st);
    FCFS_PSK_CASES(CASE)
#undef CASE
    return cudaErrorInvalidValue;
}

int read_status_psk_bf16(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_psk, sizeof(int)) != cudaSuccess) return -1;
    if (clear) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_psk, &z, sizeof(int));
    }
    return v;
}

}  // namespace fcfs
