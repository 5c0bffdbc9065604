// FP32 plane stages with thread-private transforms of compile-time length
// (passes A and C) and their launcher.
#include "psatd_regfft.cuh"

namespace psatd {

// stage 0: pass A, stage 1: pass B, stage 2: pass C (see stage_item)
cudaError_t launch_stage_reg(int stage, const LaunchCommon& c, int64_t item0, int64_t nitems, int smem, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const Args<float> a = make_args<float>(c, item0, nitems);
    if (stage == 0) return launch_kernel<float>(k_pass_a_reg, a, smem, st, kRegThreads);
    if (stage == 2) return launch_kernel<float>(k_pass_c_reg, a, smem, st, kRegThreads);
    if (stage == 1) return launch_kernel<float>(k_pass_b_reg, a, smem, st, kRegThreads);
    return cudaErrorInvalidValue;
}

}  // namespace psatd
