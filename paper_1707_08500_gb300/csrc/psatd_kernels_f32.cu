// FP32 instantiations of the stage kernels and their launchers.
#include "psatd_kernels.cuh"

namespace psatd {

template <int I>
using GeoF32 = GeoFix<kFixedF32[I].L, kFixedF32[I].ng, kFixedF32[I].M, 8>;

cudaError_t launch_stage_f32(int stage, const LaunchCommon& c, int64_t item0, int64_t nitems, int smem, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const Args<float> a = make_args<float>(c, item0, nitems);
    if (stage >= 3) return launch_geo<float, GeoDyn>(stage, a, smem, st);
    switch (c.variant) {
        case 0: return launch_geo<float, GeoF32<0>>(stage, a, smem, st);
        case 1: return launch_geo<float, GeoF32<1>>(stage, a, smem, st);
        case 2: return launch_geo<float, GeoF32<2>>(stage, a, smem, st);
        case 3: return launch_geo<float, GeoF32<3>>(stage, a, smem, st);
        case 4: return launch_geo<float, GeoF32<4>>(stage, a, smem, st);
        case -2: return launch_geo<float, GeoDynM<8>>(stage, a, smem, st);
        default: return launch_geo<float, GeoDyn>(stage, a, smem, st);
    }
}

cudaError_t launch_gauss_reduce(const void* subs, int nsub, const double* part, double* out, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (nsub * 32 + threads - 1) / threads;
    k_gauss_reduce<<<blocks, threads, 0, st>>>(static_cast<const SubDesc*>(subs), nsub, part, out);
    return cudaPeekAtLastError();
}

}  // namespace psatd
