// Device descriptors of the global-array <-> arena copies (psatd_io.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace psatd {

// One subdomain, as the copy kernels see it.
struct IoDesc {
    int64_t field_off;      // element offset of the padded box in every arena
    int64_t zstart_local;   // first plane of this box among all boxes' local planes
    int64_t zstart_valid;   // first plane among all boxes' valid planes
    int L[3];               // local (padded) extents x, y, z
    int org[3];             // global index of local cell (0, 0, 0): lo - guards (may be negative)
    int lo[3], n[3];        // valid box: first global index and extents
    int g[3];               // guard widths x, y, z
    int pad;
};

constexpr int kIoMaxFields = 10;

struct IoArgs {
    const IoDesc* desc;
    const int* plane_sub_local;   // subdomain of every local plane (all boxes in order)
    const int* plane_sub_valid;   // subdomain of every valid plane
    int nsub, nfields;
    int gn[3];                    // global grid (x, y, z)
    int64_t planes_local, planes_valid;
    const void* in[kIoMaxFields];
    void* out[kIoMaxFields];
};

cudaError_t launch_io(bool scatter, bool f64, const IoArgs& a, cudaStream_t st);

}  // namespace psatd
