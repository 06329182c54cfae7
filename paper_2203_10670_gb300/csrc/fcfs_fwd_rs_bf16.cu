// Register-blocked forward (fcfs_fwd_rs.cuh) for bf16 input and output.
#include "fcfs_fwd_rs.cuh"

namespace fcfs {

// Launch when (R, SPAN) is one of the compiled pairs; cudaErrorInvalidValue otherwise.
cudaError_t launch_forward_rs_bf16(const TmaFwdParams& T, int R, int span, cudaStream_t st) {
    if (R == 2 && span == 5) return run_rs<2, 5, __nv_bfloat16, __nv_bfloat16>(T, st);
    if (R == 4 && span == 6) return run_rs<4, 6, __nv_bfloat16, __nv_bfloat16>(T, st);
    if (R == 3 && span == 5) return run_rs<3, 5, __nv_bfloat16, __nv_bfloat16>(T, st);
    if (R == 3 && span == 3) return run_rs<3, 3, __nv_bfloat16, __nv_bfloat16>(T, st);
    if (R == 5 && span == 5) return run_rs<5, 5, __nv_bfloat16, __nv_bfloat16>(T, st);
    if (R == 7 && span == 8) return run_rs<7, 8, __nv_bfloat16, __nv_bfloat16>(T, st);
    return cudaErrorInvalidValue;
}

}  // namespace fcfs
