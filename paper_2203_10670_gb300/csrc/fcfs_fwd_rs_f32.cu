// Register-blocked forward (fcfs_fwd_rs.cuh) for f32 input and output.
#include "fcfs_fwd_rs.cuh"

namespace fcfs {

// Launch when (R, SPAN) is one of the compiled pairs; cudaErrorInvalidValue otherwise.
cudaError_t launch_forward_rs_f32(const TmaFwdParams& T, int R, int span, cudaStream_t st) {
    if (R == 2 && span == 5) return run_rs<2, 5, float, float>(T, st);
    if (R == 4 && span == 6) return run_rs<4, 6, float, float>(T, st);
    if (R == 3 && span == 5) return run_rs<3, 5, float, float>(T, st);
    if (R == 3 && span == 3) return run_rs<3, 3, float, float>(T, st);
    if (R == 5 && span == 5) return run_rs<5, 5, float, float>(T, st);
    if (R == 7 && span == 8) return run_rs<7, 8, float, float>(T, st);
    return cudaErrorInvalidValue;
}

}  // namespace fcfs
