// Moves between global arrays and the padded-box arenas of a plan (the data
// layout of Sec. 3.2 / Fig. 2a of arXiv:1707.08500): scatter fills every
// local cell of every box -- valid cells and guard images -- from the
// periodic global grid; gather writes each box's valid cells back to it.
// Pure copies, one CTA per (field, subdomain, z plane), x fastest across the
// threads of a warp so that both sides are read and written in rows.
#include <cuda_runtime.h>

#include <cstdint>

#include "psatd_io.h"

namespace psatd {

namespace {

constexpr int kIoThreads = 256;

// 16-byte vector of T
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

template <typename T>
__global__ void __launch_bounds__(kIoThreads) k_scatter(IoArgs a) {
    const int64_t item = blockIdx.x;
    const int f = int(item / a.planes_local);
    const int64_t p = item - int64_t(f) * a.planes_local;
    const int s = __ldg(a.plane_sub_local + p);
    const IoDesc& d = a.desc[s];
    const int z = int(p - d.zstart_local);
    const int Lx = d.L[0], Ly = d.L[1];
    const int gz = wrap(d.org[2] + z, a.gn[2]);
    const T* __restrict__ in = static_cast<const T*>(a.in[f]) + int64_t(gz) * a.gn[1] * a.gn[0];
    T* __restrict__ out = static_cast<T*>(a.out[f]) + d.field_off + int64_t(z) * Ly * Lx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // rows that do not wrap and start on 16-byte boundaries on both sides move
    // as 16-byte vectors
    constexpr int V = 16 / int(sizeof(T));
    using V16 = typename Vec16<T>::type;
    if (d.org[0] >= 0 && d.org[0] + Lx <= a.gn[0] && d.org[0] % V == 0 && a.gn[0] % V == 0 && Lx % V == 0 &&
        aligned16(in) && aligned16(out)) {
        const int nv = Lx / V;
        for (int y = warp; y < Ly; y += kIoThreads / 32) {
            const V16* row = reinterpret_cast<const V16*>(in + int64_t(wrap(d.org[1] + y, a.gn[1])) * a.gn[0] + d.org[0]);
            V16* orow = reinterpret_cast<V16*>(out + int64_t(y) * Lx);
            for (int x = lane; x < nv; x += 32) orow[x] = __ldg(row + x);
        }
        return;
    }
    const int gx0 = wrap(d.org[0] + lane, a.gn[0]);
    for (int y = warp; y < Ly; y += kIoThreads / 32) {
        const T* row = in + int64_t(wrap(d.org[1] + y, a.gn[1])) * a.gn[0];
        T* orow = out + int64_t(y) * Lx;
        int gx = gx0;
        for (int x = lane; x < Lx; x += 32) {
            orow[x] = __ldg(row + gx);
            gx += 32;
            while (gx >= a.gn[0]) gx -= a.gn[0];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kIoThreads) k_gather(IoArgs a) {
    const int64_t item = blockIdx.x;
    const int f = int(item / a.planes_valid);
    const int64_t p = item - int64_t(f) * a.planes_valid;
    const int s = __ldg(a.plane_sub_valid + p);
    const IoDesc& d = a.desc[s];
    const int zv = int(p - d.zstart_valid);
    const int Lx = d.L[0], Ly = d.L[1];
    const T* __restrict__ in = static_cast<const T*>(a.in[f]) + d.field_off +
                               (int64_t(zv + d.g[2]) * Ly + d.g[1]) * Lx + d.g[0];
    T* __restrict__ out = static_cast<T*>(a.out[f]) +
                          (int64_t(d.lo[2] + zv) * a.gn[1] + d.lo[1]) * a.gn[0] + d.lo[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int V = 16 / int(sizeof(T));
    using V16 = typename Vec16<T>::type;
    if (d.n[0] % V == 0 && Lx % V == 0 && a.gn[0] % V == 0 && aligned16(in) && aligned16(out)) {
        const int nv = d.n[0] / V;
        for (int y = warp; y < d.n[1]; y += kIoThreads / 32) {
            const V16* row = reinterpret_cast<const V16*>(in + int64_t(y) * Lx);
            V16* orow = reinterpret_cast<V16*>(out + int64_t(y) * a.gn[0]);
            for (int x = lane; x < nv; x += 32) orow[x] = __ldg(row + x);
        }
        return;
    }
    for (int y = warp; y < d.n[1]; y += kIoThreads / 32) {
        const T* row = in + int64_t(y) * Lx;
        T* orow = out + int64_t(y) * a.gn[0];
        for (int x = lane; x < d.n[0]; x += 32) orow[x] = __ldg(row + x);
    }
}

}  // namespace

cudaError_t launch_io(bool scatter, bool f64, const IoArgs& a, cudaStream_t st) {
    const int64_t items = int64_t(a.nfields) * (scatter ? a.planes_local : a.planes_valid);
    if (items <= 0) return cudaSuccess;
    if (items > 2147483647) return cudaErrorInvalidConfiguration;
    const unsigned grid = unsigned(items);
    if (scatter) {
        if (f64) k_scatter<double><<<grid, kIoThreads, 0, st>>>(a);
        else k_scatter<float><<<grid, kIoThreads, 0, st>>>(a);
    } else {
        if (f64) k_gather<double><<<grid, kIoThreads, 0, st>>>(a);
        else k_gather<float><<<grid, kIoThreads, 0, st>>>(a);
    }
    return cudaPeekAtLastError();
}

}  // namespace psatd
