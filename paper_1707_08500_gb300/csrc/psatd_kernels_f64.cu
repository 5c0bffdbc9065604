// FP64 instantiations of the stage kernels and their launchers.
#include "psatd_kernels.cuh"

namespace psatd {

template <int I>
using GeoF64 = GeoFix<kFixedF64[I].L, kFixedF64[I].ng, kFixedF64[I].M, 16>;

cudaError_t launch_stage_f64(int stage, const LaunchCommon& c, int64_t item0, int64_t nitems, int smem, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const Args<double> a = make_args<double>(c, item0, nitems);
    if (stage >= 3) return launch_geo<double, GeoDyn>(stage, a, smem, st);
    switch (c.variant) {
        case 0: return launch_geo<double, GeoF64<0>>(stage, a, smem, st);
        case 1: return launch_geo<double, GeoF64<1>>(stage, a, smem, st);
        case 2: return launch_geo<double, GeoF64<2>>(stage, a, smem, st);
        case -2: return launch_geo<double, GeoDynM<4>>(stage, a, smem, st);
        default: return launch_geo<double, GeoDyn>(stage, a, smem, st);
    }
}

}  // namespace psatd
