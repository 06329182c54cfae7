// Instantiations of the bulk-copy forward (fcfs_fwd_tma.cuh) for u8 inputs.
#include "fcfs_fwd_tma.cuh"

namespace fcfs {

#define FCFS_NT_CASES(X) X(1) X(2) X(3) X(4) X(5) X(7) X(9)

cudaError_t launch_forward_tma_u8(const TmaFwdParams& T, int nt, int din, int dout, cudaStream_t st) {
    const size_t smem = (size_t)T.bar_off + 16;
    if (din == FCFS_U8 && dout == FCFS_F32) {
        switch (nt) {
#define CASE(N) \
    case N: return run<N, uint8_t, float>(T, smem, st);
            FCFS_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    }
    if (din == FCFS_U8 && dout == FCFS_BF16) {
        switch (nt) {
#define CASE(N) \
    case N: return run<N, uint8_t, __nv_bfloat16>(T, smem, st);
            FCFS_NT_CASES(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

int read_status_fwd_tma_u8(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_fwd_tma, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_status_fwd_tma, &z, sizeof(int));
    }
    return v;
}

}  // namespace fcfs
