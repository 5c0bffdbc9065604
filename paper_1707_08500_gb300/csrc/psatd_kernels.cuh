#pragma once
// CUDA kernels of the local-FFT PSATD push for sm_103a.
//
// One step of one padded subdomain (Sec. 3.2 of arXiv:1707.08500) is split
// into three streaming stages over HBM:
//
//   pass A  per (subdomain, field, z plane): real x-FFT of the plane (as a
//           half-length complex FFT of packed pairs plus the split step),
//           then the y-FFT of every column; writes the plane's half spectrum.
//   pass B  per (subdomain, chunk of M (ky,kx) modes): z-FFT of all fields,
//           Eq. 1a/1b on every mode (Sec. 3.1), inverse z-FFT of E and B;
//           writes back only the valid z planes.
//   pass C  per (subdomain, E/B component, valid z plane): inverse y-FFT,
//           inverse real x-FFT of the valid rows, then the guard replacement
//           of Fig. 3 step 3 fused into the store: every valid cell is
//           written to its own box and to every guard cell that images it.
//
// Every 1D transform of length n = f1*f2 runs in shared memory as two
// in-place register stages (f1-point DFTs at stride f2, twiddle, f2-point
// DFTs on contiguous blocks).  Forward transforms leave frequency k1 + f1*k2
// at position k1*f2 + k2; the inverse consumes that order and returns natural
// order, so spectra never need reordering: the host builds the per-mode
// tables in the same position order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "psatd_internal.h"
#include "small_dft.cuh"

#include <mutex>

// Minimum resident CTAs per SM requested from the compiler for each stage
// kernel (FP32; FP64 uses 2), which caps its registers per thread.
#ifndef PSATD_MINB_A
#define PSATD_MINB_A 5
#endif
#ifndef PSATD_MINB_A_FIXED
#define PSATD_MINB_A_FIXED 6    // compile-time geometry: fewer registers live, one more CTA fits
#endif
#ifndef PSATD_MINB_B
#define PSATD_MINB_B 3    // ten fields of 8 modes x 96 z fill a third of shared memory
#endif
#ifndef PSATD_MINB_C
#define PSATD_MINB_C 5
#endif

namespace psatd {

// A table twiddle as an FP32 hi + lo pair (lo = 0 in FP64).
template <typename T>
struct alignas(4 * sizeof(T)) twd { cpx<T> hi, lo; };

// FP32 table twiddles: the hi part alone (PSATD_TW_HILO 0, the default),
// which the host rounds so that each twiddle's magnitude is as close to 1 as
// neighbouring FP32 values allow (the transform then stays closer to
// unitary; the phase error this trades in cancels between a forward
// transform and its inverse), or hi + lo pairs (PSATD_TW_HILO 1, FP64-exact
// twiddles at twice the multiply cost).  Measured over 100 FP32 steps
// against the FP64 oracle: 5.1e-6 (hi alone) and 3.8e-6 (hi + lo).
#ifndef PSATD_TW_HILO
#define PSATD_TW_HILO 0
#endif

template <typename T>
__device__ __forceinline__ twd<T> ld_tw(const twd<T>* p) {
    twd<T> t;
    if constexpr (sizeof(T) == 4 && !PSATD_TW_HILO) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        t.hi = mk(v.x, v.y);
        t.lo = mk(0.f, 0.f);
    } else if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        t.hi = mk(v.x, v.y);
        t.lo = mk(v.z, v.w);
    } else {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        t.hi = mk(v.x, v.y);
        t.lo = mk(0.0, 0.0);
    }
    return t;
}
template <typename T>   // v * w
__device__ __forceinline__ cpx<T> mul_tw(cpx<T> v, const twd<T>& w) {
    if constexpr (sizeof(T) == 4 && !PSATD_TW_HILO) return cmul(v, w.hi);
    else return cmul_const(v, w.hi.x, w.lo.x, w.hi.y, w.lo.y);
}
template <typename T>   // v * conj(w)
__device__ __forceinline__ cpx<T> mul_tw_conj(cpx<T> v, const twd<T>& w) {
    if constexpr (sizeof(T) == 4 && !PSATD_TW_HILO) return cmulc(v, w.hi);
    else return cmul_const(v, w.hi.x, w.lo.x, -w.hi.y, -w.lo.y);
}

template <typename T>
struct Args {
    const SubDesc* subs;
    const Segment* segs;
    const twd<T>* tw;       // twiddle pool (hi/lo pairs)
    const T* tab;           // real tables (coefficients, wavenumbers)
    const cpx<T>* tabc;     // complex tables (stagger phases)
    cpx<T>* spec;           // spectra
    T* eb[6];               // Ex Ey Ez Bx By Bz
    const T* jr[4];         // Jx Jy Jz rho
    double* gauss_part;     // 2 per pass-B item
    unsigned long long* work;   // work-item ticket counter of this launch (zero at its start)
    unsigned int* err;          // device error word: bit 0 item outside its subdomain, bit 1 ticket out of range
    int persistent;         // 1: CTAs draw items from `work`; 0: CTA b does item item0 + b
    int64_t item0, nitems;  // items handled by this launch
    int64_t per_sub[5];     // items per subdomain of each stage when uniform, else 0
    int nsub, nseg;
    int nf;                 // fields transformed forward (9, or 10 with rho; heat: 1, or 2 with a source)
    int nout;               // fields written back (6; heat: 1)
    int staggered;
    int own_only;           // pass C writes only the own valid box
};



template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T>
__device__ __forceinline__ cpx<T> ldg_c(const cpx<T>* p) {
    const auto v = __ldg(reinterpret_cast<const typename vec2<T>::type*>(p));
    return mk(v.x, v.y);
}

template <typename T>
struct cpx4 { T a, b, c, d; };
template <typename T>
__device__ __forceinline__ void stcs4(T* p, cpx4<T> v) {
    if constexpr (sizeof(T) == 4) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v.a, v.b, v.c, v.d));
    } else {
        __stcs(reinterpret_cast<double2*>(p), make_double2(v.a, v.b));
        __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(v.c, v.d));
    }
}
template <typename T>
__device__ __forceinline__ void stcs_c(cpx<T>* p, cpx<T> v) {
    using V = typename vec2<T>::type;
    V w; w.x = v.x; w.y = v.y;
    __stcs(reinterpret_cast<V*>(p), w);
}

// Rows [0, ny) of a segment whose row holds a power-of-two number ex4 <= NT
// of 16-byte pieces (guard images 16 cells wide, valid rows of 64), from
// shared memory (row stride rs elements) to global memory (row stride dld):
// each of the NT threads keeps one piece column and steps down the rows by
// pointer increments, with no division.  Returns false, storing nothing,
// for other widths.
template <int NT, typename T>
__device__ __forceinline__ bool store_rows_pow2(T* dst, int64_t dld, const T* sp, int rs, int ex4, int ny) {
    if (ex4 <= 0 || (ex4 & (ex4 - 1)) != 0 || ex4 > NT) return false;
    const int lg = 31 - __clz(ex4), x4 = int(threadIdx.x) & (ex4 - 1);
    const int y0 = int(threadIdx.x) >> lg, dyy = NT >> lg;
    const T* s = sp + y0 * rs + 4 * x4;
    T* o = dst + int64_t(y0) * dld + 4 * x4;
    const int64_t ostep = int64_t(dyy) * dld;
    for (int yy = y0; yy < ny; yy += dyy, s += dyy * rs, o += ostep) {
        const cpx<T> u = *reinterpret_cast<const cpx<T>*>(s);
        const cpx<T> w = *reinterpret_cast<const cpx<T>*>(s + 2);
        stcs4(o, cpx4<T>{u.x, u.y, w.x, w.y});
    }
    return true;
}

// ---- asynchronous global -> shared copies (no register staging) ------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n"
                 :: "r"(smem_u32(dst)), "l"(__cvta_generic_to_global(src)) : "memory");
}
// 16 bytes, of which the first src_bytes are read and the rest zero-filled
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
                 :: "r"(smem_u32(dst)), "l"(__cvta_generic_to_global(src)), "r"(src_bytes) : "memory");
}
// 8 bytes, of which the first src_bytes are read and the rest zero-filled
__device__ __forceinline__ void cp_async8z(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n"
                 :: "r"(smem_u32(dst)), "l"(__cvta_generic_to_global(src)), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// one complex value
template <typename T>
__device__ __forceinline__ void cp_async_c(cpx<T>* dst, const cpx<T>* src) {
    if constexpr (sizeof(T) == 4) cp_async8(dst, src);
    else cp_async16(dst, src, 16);
}

// Batched transforms in shared memory.  Transform b starts at b*s_in
// (single-level) or (b mod inner)*s_in + (b / inner)*s_out (two-level, used
// for several fields of one pencil chunk; lg = log2(inner) when inner is a
// power of two, else -1); its elements are es apart.
struct Batch {
    int count;   // number of transforms
    int s_in;
    int lg;
    int s_out;
    int es;
    int inner;
};

template <bool TWO>
__device__ __forceinline__ int boff(const Batch& b, int i) {
    if constexpr (TWO) {
        if (b.lg >= 0) return (i & ((1 << b.lg) - 1)) * b.s_in + (i >> b.lg) * b.s_out;
        const int o = i / b.inner;
        return (i - o * b.inner) * b.s_in + o * b.s_out;
    } else {
        return i * b.s_in;
    }
}

// Visit every (outer, inner) pair with inner in [0, count), outer in
// [0, nouter), pair index outer*count + inner = threadIdx.x + k*kThreads,
// without a division per pair (the inner step is always < count).
template <class F>
__device__ __forceinline__ void loop2(int count, int nouter, F&& f) {
    int o = int(threadIdx.x) / count;
    int i = int(threadIdx.x) - o * count;
    const int dO = kThreads / count, dI = kThreads - dO * count;
    while (o < nouter) {
        f(o, i);
        i += dI;
        o += dO;
        if (i >= count) { i -= count; ++o; }
    }
}

// ---- shared-memory FFT stages ---------------------------------------------
// Strided stage: item (j, b) loads the R values at positions j + r*stride of
// transform b, does an R-point DFT and (forward only) multiplies output r by
// w^{j r}; stores in place.
template <int R, bool INV, bool TW, bool TWO, typename T>
__device__ __forceinline__ void stage_strided(cpx<T>* sm, const Batch& bt, int stride,
                                              const twd<T>* __restrict__ tw) {
    const int es = bt.es * stride;
    loop2(bt.count, stride, [&](int j, int b) {
        cpx<T>* p = sm + boff<TWO>(bt, b) + j * bt.es;
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * es];
        Dft<R, INV>::run(v);
        if constexpr (TW) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = mul_tw(v[r], ld_tw(tw + j * r));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * es] = v[r];
    });
}

// Block stage: item (k, b) loads the R contiguous values k*R + r of transform
// b, does an R-point DFT and (inverse only) multiplies output r by conj(w^{r k}).
template <int R, bool INV, bool TW, bool TWO, typename T>
__device__ __forceinline__ void stage_block(cpx<T>* sm, const Batch& bt, int nblk,
                                            const twd<T>* __restrict__ tw) {
    loop2(bt.count, nblk, [&](int k, int b) {
        cpx<T>* p = sm + boff<TWO>(bt, b) + k * R * bt.es;
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * bt.es];
        Dft<R, INV>::run(v);
        if constexpr (TW) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = mul_tw_conj(v[r], ld_tw(tw + r * k));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * bt.es] = v[r];
    });
}

// Three-factor axes (n = f1 f2 f3, m = f2 f3).  Their first and last
// stages are the two-factor ones (f1-point DFTs at stride m with w_n^{j r};
// f3-point DFTs on contiguous blocks); the middle stage and the first inverse
// stage below use a DFT of run-time size R <= 16 (an R^2 sum with the
// twiddles w_R^e = w_n^{e n/R} read from the axis table), which keeps the
// code of this rarely used path small.
template <bool INV, typename T>
__device__ __forceinline__ void dft_runtime(cpx<T>* v, int R, const twd<T>* __restrict__ tw_n, int nR) {
    cpx<T> out[kMaxDft];
    for (int k = 0; k < R; ++k) {
        cpx<T> acc = v[0];
        int e = 0;
        for (int r = 1; r < R; ++r) {
            e += k;
            if (e >= R) e -= R;                   // e = r k mod R
            const twd<T> w = ld_tw(tw_n + e * nR);
            acc = acc + (INV ? mul_tw_conj(v[r], w) : mul_tw(v[r], w));
        }
        out[k] = acc;
    }
    for (int k = 0; k < R; ++k) v[k] = out[k];
}

// middle stage, inside each block k1 of length m: f2-point DFTs at stride f3
// (item j2 in [0, f3)); forward, output r is then multiplied by
// w_m^{j2 r} = w_n^{j2 r f1}; inverse, the output at position k1 m + j2 + f3 r
// by conj(w_n^{(j2 + f3 r) k1}).
template <bool INV, bool TWO, typename T>
__device__ __forceinline__ void stage_mid(cpx<T>* sm, const Batch& bt, const AxisPlan& ax,
                                          const twd<T>* __restrict__ tw_n) {
    const int f1 = ax.f1, f2 = ax.f2, f3 = ax.f3, m = f2 * f3;
    const int es = bt.es * f3;
    loop2(bt.count, f1 * f3, [&](int i, int b) {
        const int k1 = i / f3, j2 = i - k1 * f3;
        cpx<T>* p = sm + boff<TWO>(bt, b) + (k1 * m + j2) * bt.es;
        cpx<T> v[kMaxDft];
        for (int r = 0; r < f2; ++r) v[r] = p[r * es];
        dft_runtime<INV>(v, f2, tw_n, ax.n / f2);
        for (int r = 0; r < f2; ++r) {
            const twd<T> w = ld_tw(tw_n + (INV ? (j2 + f3 * r) * k1 : j2 * r * f1));
            p[r * es] = INV ? mul_tw_conj(v[r], w) : mul_tw(v[r], w);
        }
    });
}

// first inverse stage: f3-point DFTs on contiguous blocks (block index
// k = k1 f2 + k2), then output r times conj(w_m^{r k2}) = conj(w_n^{r k2 f1}).
template <bool TWO, typename T>
__device__ __forceinline__ void stage_block_m(cpx<T>* sm, const Batch& bt, const AxisPlan& ax,
                                              const twd<T>* __restrict__ tw_n) {
    const int f1 = ax.f1, f2 = ax.f2, f3 = ax.f3;
    loop2(bt.count, f1 * f2, [&](int k, int b) {
        cpx<T>* p = sm + boff<TWO>(bt, b) + k * f3 * bt.es;
        cpx<T> v[kMaxDft];
        for (int r = 0; r < f3; ++r) v[r] = p[r * bt.es];
        dft_runtime<true>(v, f3, tw_n, ax.n / f3);
        const int k2 = k - (k / f2) * f2;
        for (int r = 0; r < f3; ++r) p[r * bt.es] = mul_tw_conj(v[r], ld_tw(tw_n + r * k2 * f1));
    });
}

// natural order in -> position order out (THREE: three-factor axes possible).
// The compiled first and last stages are shared by both splits (one inlined
// copy each): their stride and block count are run-time values.
template <bool TWO, typename T, bool THREE = true>
__device__ __forceinline__ void fft_fwd(cpx<T>* sm, const AxisPlan& ax, const Batch& bt, const twd<T>* tw) {
    const twd<T>* w = tw + ax.tw;
    const bool three = THREE && ax.f3 > 1;
    const int m = three ? ax.f2 * ax.f3 : ax.f2;           // stride of the first stage
    with_size(ax.f1, [&](auto N1) { stage_strided<decltype(N1)::value, false, true, TWO>(sm, bt, m, w); });
    __syncthreads();
    if (three) {
        stage_mid<false, TWO>(sm, bt, ax, w);
        __syncthreads();
    }
    const int last = three ? ax.f3 : ax.f2, nblk = three ? ax.f1 * ax.f2 : ax.f1;
    with_size(last, [&](auto NL) { stage_block<decltype(NL)::value, false, false, TWO>(sm, bt, nblk, w); });
    __syncthreads();
}

// position order in -> natural order out (unnormalised)
template <bool TWO, typename T, bool THREE = true>
__device__ __forceinline__ void fft_inv(cpx<T>* sm, const AxisPlan& ax, const Batch& bt, const twd<T>* tw) {
    const twd<T>* w = tw + ax.tw;
    const bool three = THREE && ax.f3 > 1;
    if (three) {
        stage_block_m<TWO>(sm, bt, ax, w);
        __syncthreads();
        stage_mid<true, TWO>(sm, bt, ax, w);
        __syncthreads();
    } else {
        with_size(ax.f2, [&](auto N2) { stage_block<decltype(N2)::value, true, true, TWO>(sm, bt, ax.f1, w); });
        __syncthreads();
    }
    const int m = three ? ax.f2 * ax.f3 : ax.f2;
    with_size(ax.f1, [&](auto N1) { stage_strided<decltype(N1)::value, true, false, TWO>(sm, bt, m, w); });
    __syncthreads();
}

// Pairs (k, h-k) of the real split in the position order of an h = f1*f2
// transform (frequency k1 + f1 k2 at position k1 f2 + k2).  Pair 0 is k = 0;
// pairs 1..f2/2 pair position P with f2 - P (k1 = 0); the remaining pairs
// pair P >= f2 with h + f2 - 1 - P.  Every unordered pair appears once.
__device__ __forceinline__ int split_pairs(int h, int f2) { return 1 + f2 / 2 + (h - f2 + 1) / 2; }
__device__ __forceinline__ void split_pair(int i, int h, int f2, int& pa, int& pb) {
    const int lower = f2 / 2;
    if (i <= lower) { pa = i; pb = f2 - i; }
    else { pa = f2 + (i - lower - 1); pb = h + f2 - 1 - pa; }
}

// Stages: 0 = pass A, 1 = pass B, 2 = pass C, 3 = standalone exchange; the
// split-plane schedule replaces A by 4 (x rows) + 5 (y columns) and C by
// 6 (y columns) + 7 (x rows and the exchange scatter); 8 is pass B of the
// heat equation (its items are those of pass B).
template <int STAGE>
__device__ __forceinline__ int64_t stage_item(const SubDesc& d) {
    return STAGE == 0 || STAGE == 4 ? d.itemA : STAGE == 1 ? d.itemB : STAGE == 5 ? d.itemA2
         : STAGE == 6 ? d.itemC1 : d.itemC;
}

// Slot of LaunchCommon::per_sub that counts a stage's items per subdomain.
template <int STAGE>
constexpr int per_sub_slot() {
    return STAGE == 0 || STAGE == 4 ? 0 : STAGE == 1 ? 1 : STAGE == 5 ? 3 : STAGE == 6 ? 4 : 2;
}

// Position of frequency k on an axis with a three-factor split.
__device__ __forceinline__ int pos_of3(int k, const AxisPlan& ax) {
    const int k1 = k % ax.f1, kk = k / ax.f1;
    const int k2 = kk % ax.f2, k3 = kk / ax.f2;
    return (k1 * ax.f2 + k2) * ax.f3 + k3;
}
// Unordered pair i of positions (k, h-k) of the packed x transform: the
// two-factor walk of split_pair, or, with three factors, frequency k = i.
__device__ __forceinline__ int split_pairs_ax(int h, const AxisPlan& ax) {
    return ax.f3 > 1 ? h / 2 + 1 : split_pairs(h, ax.f2);
}
__device__ __forceinline__ void split_pair_ax(int i, int h, const AxisPlan& ax, int& pa, int& pb) {
    if (ax.f3 > 1) {
        pa = pos_of3(i, ax);
        pb = pos_of3(h - i, ax);
    } else {
        split_pair(i, h, ax.f2, pa, pb);
    }
}

// Real split after the packed forward x transform: rows r < nrows at
// p0 + r*pitch hold the h-point transform of z[m] = x[2m] + i x[2m+1] in
// position order; each becomes the half spectrum X[0..h] of its real row,
// walking the pairs (k, h-k) directly in position order (see split_pair).
template <typename T>
__device__ __forceinline__ void real_split_rows(cpx<T>* p0, int nrows, int pitch, int h, const AxisPlan& ax,
                                                const twd<T>* __restrict__ wp) {
    loop2(nrows, split_pairs_ax(h, ax), [&](int i, int y) {
        cpx<T>* p = p0 + y * pitch;
        if (i == 0) {
            const cpx<T> z0 = p[0];
            p[0] = mk(z0.x + z0.y, T(0));
            p[h] = mk(z0.x - z0.y, T(0));
        } else {
            int pa, pb;
            split_pair_ax(i, h, ax, pa, pb);
            const cpx<T> A = p[pa], Bc = conj(p[pb]);
            const cpx<T> e = scale(A + Bc, T(0.5));
            const cpx<T> dd = A - Bc;
            const cpx<T> o = mk(T(0.5) * dd.y, T(-0.5) * dd.x);   // (A - conj B)/(2i)
            const cpx<T> wo = mul_tw(o, ld_tw(wp + pa));
            p[pa] = e + wo;
            if (pb != pa) p[pb] = conj(e - wo);
        }
    });
}

// Inverse of real_split_rows before the inverse x transform: merge each row's
// half spectrum into the packed h-point form (C2R: only the real parts of
// X[0] and X[h] are used).
template <typename T>
__device__ __forceinline__ void real_merge_rows(cpx<T>* p0, int nrows, int pitch, int h, const AxisPlan& ax,
                                                const twd<T>* __restrict__ wp) {
    loop2(nrows, split_pairs_ax(h, ax), [&](int i, int y) {
        cpx<T>* p = p0 + y * pitch;
        if (i == 0) {
            const T x0 = p[0].x, xh = p[h].x;
            p[0] = mk(x0 + xh, x0 - xh);
        } else {
            int pa, pb;
            split_pair_ax(i, h, ax, pa, pb);
            const cpx<T> A = p[pa], Bc = conj(p[pb]);
            const cpx<T> e = A + Bc;
            const cpx<T> o = mul_tw_conj(A - Bc, ld_tw(wp + pa));
            p[pa] = e + mul_i(o);
            if (pb != pa) p[pb] = conj(e) + mul_i(conj(o));
        }
    });
}

template <int STAGE>
__device__ __forceinline__ int find_sub(const SubDesc* __restrict__ subs, int nsub, int64_t item) {
    int lo = 0, hi = nsub - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (stage_item<STAGE>(subs[mid]) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}


// Decode work item `it` of a stage: warp 0 finds the subdomain (arithmetic for
// uniform decompositions, else a binary search over the stage's first items)
// and copies its descriptor to shared memory for the whole CTA.
template <int STAGE, typename T>
__device__ __forceinline__ int decode_item(const Args<T>& a, int64_t it, SubDesc* sd) {
    __shared__ int s_sub;
    if (threadIdx.x < 32) {
        int s = 0;
        if (a.per_sub[per_sub_slot<STAGE>()] > 0) {
            s = int(it / a.per_sub[per_sub_slot<STAGE>()]);
        } else if (threadIdx.x == 0) {
            s = find_sub<STAGE>(a.subs, a.nsub, it);
        }
        s = __shfl_sync(0xffffffffu, s, 0);
        const int* src = reinterpret_cast<const int*>(a.subs + s);
        int* dst = reinterpret_cast<int*>(sd);
        for (int i = threadIdx.x; i < int(sizeof(SubDesc) / 4); i += 32) dst[i] = __ldg(src + i);
        if (threadIdx.x == 0) s_sub = s;
    }
    __syncthreads();
    // the item must lie in the subdomain's own range of this stage (checked on
    // the shared copy: the start, and the count when every subdomain has the
    // same number of items)
    if (threadIdx.x == 0) {
        const int64_t rel = it - stage_item<STAGE>(*sd);
        const int64_t per = a.per_sub[per_sub_slot<STAGE>()];
        if (rel < 0 || (per > 0 && rel >= per)) atomicOr(a.err, 1u);
    }
    return s_sub;
}

template <typename T>
__device__ __forceinline__ const T* field_in(const Args<T>& a, int f) {
    return f < 6 ? a.eb[f] : a.jr[f - 6];
}

// Work loop of the stage kernels.  Persistent launches: each CTA draws the
// next unprocessed item of the launch from a global ticket counter until
// every item is taken; the ticket for the following item is drawn at the
// start of the current one, into the other of two shared slots, so no CTA
// waits on the atomic between items.  Every CTA stops after drawing exactly
// one ticket past the last item, so a launch draws nitems + gridDim.x tickets
// in all; the CTA that draws the last of them returns the counter to zero for
// the next launch on the stream (the counter starts at zero when the
// workspace is attached).  Otherwise CTA b processes item item0 + b only.
// Every loop body ends with __syncthreads(), which orders the slot writes and
// reads.
template <typename T>
struct Tickets {
    const Args<T>& a;
    int64_t* slot;
    int par = 0;
    __device__ int64_t draw() const {
        const int64_t k = int64_t(atomicAdd(a.work, 1ull));
        if (k == a.nitems + int64_t(gridDim.x) - 1) *a.work = 0ull;   // the last ticket of the launch
        // more tickets than one launch draws: another launch shares the
        // counter (overlapping pushes of one plan); the ticket is treated as
        // past the end
        if (k >= a.nitems + int64_t(gridDim.x)) atomicOr(a.err, 2u);
        return k;
    }
    __device__ Tickets(const Args<T>& args, int64_t* s) : a(args), slot(s) {
        if (threadIdx.x == 0) slot[0] = a.persistent ? draw() : int64_t(blockIdx.x);
        __syncthreads();
    }
    __device__ int64_t current() const { const int64_t k = slot[par]; return k < a.nitems ? a.item0 + k : -1; }
    __device__ void prefetch() {
        if (threadIdx.x == 0) slot[par ^ 1] = a.persistent ? draw() : a.nitems;
    }
    __device__ void advance() { par ^= 1; }
};

// ---- transform geometry ------------------------------------------------------
// Everything a stage needs to know about one subdomain's local box: read from
// its descriptor (GeoDyn) or fixed at compile time for a cubic box of side L
// with NG guards (GeoFix), in which case every stride, loop bound and DFT size
// below is a constant.
struct GeoDyn {
    static constexpr bool kFixed = false;
    static constexpr bool kThree = true;     // axes may have three-factor splits
    int Lx, Ly, Lz, h, lxh, pitch, q, ng, ngz, nvy, nvz, M, lgM, fs;
    AxisPlan ax, ay, az;
    __device__ explicit GeoDyn(const SubDesc& d)
        : Lx(d.L[0]), Ly(d.L[1]), Lz(d.L[2]), h(d.L[0] >> 1), lxh(d.lxh), pitch(d.pitch), q(d.q), ng(d.ng), ngz(d.ngz),
          nvy(d.nv[1]), nvz(d.nv[2]), M(d.chunkB), lgM(d.lgB), fs(d.fsB), ax(d.ax), ay(d.ay), az(d.az) {}
};

// Descriptor-driven geometry with the pass-B chunk width fixed at compile time
// (the library default), for decompositions of mixed box shapes.
template <int MB>
struct GeoDynM {
    static constexpr bool kFixed = false;
    static constexpr bool kThree = false;
    static constexpr int M = MB, lgM = (MB & (MB - 1)) ? -1 : ilog2(MB);
    int Lx, Ly, Lz, h, lxh, pitch, q, ng, ngz, nvy, nvz, fs;
    AxisPlan ax, ay, az;
    __device__ explicit GeoDynM(const SubDesc& d)
        : Lx(d.L[0]), Ly(d.L[1]), Lz(d.L[2]), h(d.L[0] >> 1), lxh(d.lxh), pitch(d.pitch), q(d.q), ng(d.ng), ngz(d.ngz),
          nvy(d.nv[1]), nvz(d.nv[2]), fs(d.fsB), ax(d.ax), ay(d.ay), az(d.az) {}
};

template <int L, int NG, int MB, int CSZ>
struct GeoFix {
    static constexpr bool kFixed = true;
    static constexpr bool kThree = false;
    static constexpr int Lx = L, Ly = L, Lz = L, h = L / 2, lxh = L / 2 + 1, pitch = (L / 2 + 1) | 1;
    static constexpr int q = L * (L / 2 + 1), ng = NG, ngz = NG, nvy = L - 2 * NG, nvz = L - 2 * NG;
    static constexpr int M = MB, lgM = (MB & (MB - 1)) ? -1 : ilog2(MB), fs = pad_field_stride(L, MB, CSZ);
    AxisPlan ax, ay, az;
    __device__ explicit GeoFix(const SubDesc& d)
        : ax{h, split_first(h), h / split_first(h), d.ax.tw, 0, 0},
          ay{L, split_first(L), L / split_first(L), d.ay.tw, 0, 0},
          az{L, split_first(L), L / split_first(L), d.az.tw, 0, 0} {}
};

// ---- pass A: x (real) and y forward transforms of one plane ---------------
template <typename T, class G>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? (G::kFixed ? PSATD_MINB_A_FIXED : PSATD_MINB_A) : 2)
k_pass_a(Args<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ SubDesc d;
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<0>(a, it, &d);
        const G g(d);
        const int Lx = g.Lx, Ly = g.Ly, Lz = g.Lz;
        const int loc = int(it - d.itemA);
        const int f = loc / Lz, z = loc - (loc / Lz) * Lz;
        const int h = g.h, pitch = g.pitch, lxh = g.lxh;
        const T* src = field_in(a, f) + d.field_off + int64_t(z) * Ly * Lx;
        // packed complex z[m] = x[2m] + i x[2m+1], row y at y*pitch
        loop2(h, Ly, [&](int y, int m) {
            cp_async_c(sm + y * pitch + m, reinterpret_cast<const cpx<T>*>(src) + y * h + m);
        });
        cp_async_wait_all();
        __syncthreads();
        // x: complex FFT of length h over the Ly rows
        fft_fwd<false, T, G::kThree>(sm, g.ax, Batch{Ly, pitch, 0, 0, 1, 1}, a.tw);
        // split the packed transform into the half spectrum X[0..h]
        real_split_rows(sm, Ly, pitch, h, g.ax, a.tw + d.tw_post);
        __syncthreads();
        // y: complex FFT of length Ly over the lxh columns
        fft_fwd<false, T, G::kThree>(sm, g.ay, Batch{lxh, 1, 0, 0, pitch, 1}, a.tw);
        cpx<T>* dst = a.spec + d.spec_off + int64_t(f * Lz + z) * g.q;
        loop2(lxh, Ly, [&](int y, int c) { stcs_c(dst + y * lxh + c, sm[y * pitch + c]); });
        __syncthreads();
    }
}

// ---- pass B: z transforms and the Eq. 1 update -----------------------------
// Sum of v over the CTA (a pairwise tree, in T), returned to thread 0.
// Block sums of two values at once (warp shuffle trees, then thread 0 adds
// the warps' partials in order); the results are valid in thread 0 only.
// The caller synchronises the block before red is written again.
template <typename T>
__device__ __forceinline__ void block_sum2(T& v0, T& v1, T* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[w] = v0;
        red[kThreads / 32 + w] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T s0 = 0, s1 = 0;
        for (int i = 0; i < kThreads / 32; ++i) s0 += red[i];
        for (int i = 0; i < kThreads / 32; ++i) s1 += red[kThreads / 32 + i];
        v0 = s0;
        v1 = s1;
    }
}

// Eq. 1a/1b on one mode (ky, kx at position q of the plane, z position zp):
// p points at its E_x spectrum in a pass-B chunk, the other fields at
// multiples of fs; E and B are replaced by E' and B'; with rho (nf > 9) the
// Gauss partial sums of the mode are added to g_res and g_rho.
template <typename T>
__device__ __forceinline__ void eq1_mode(const Args<T>& a, const SubDesc& d, cpx<T>* p, int fs, int q, int yp, int xp,
                                         int zp, int lxh, int Ly, int64_t NM, int64_t Q, T Nfull, T& g_res,
                                         T& g_rho) {
    const int nf = a.nf;
    const T* __restrict__ tk = a.tab + d.tab_k;
    const T* __restrict__ tb = a.tab + d.tab_coef + int64_t(zp) * Q + q;
    const T C = __ldg(tb), S = __ldg(tb + NM), Sk = __ldg(tb + 2 * NM), omC = __ldg(tb + 3 * NM);
    const T omCk = __ldg(tb + 4 * NM), Dk = __ldg(tb + 5 * NM), inv = __ldg(tb + 6 * NM);
    const T kx = __ldg(tk + xp), ky = __ldg(tk + lxh + yp), kz = __ldg(tk + lxh + Ly + zp);
    const T hx = kx * inv, hy = ky * inv, hz = kz * inv;
    cpx<T> E0 = p[0], E1 = p[fs], E2 = p[2 * fs];
    cpx<T> B0 = p[3 * fs], B1 = p[4 * fs], B2 = p[5 * fs];
    cpx<T> J0 = p[6 * fs], J1 = p[7 * fs], J2 = p[8 * fs];
    cpx<T> px, py, pz;
    if (a.staggered) {
        const cpx<T>* ph = a.tabc + d.tab_ph;
        px = ldg_c(ph + xp); py = ldg_c(ph + lxh + yp); pz = ldg_c(ph + lxh + Ly + zp);
        const cpx<T> pyz = cmul(py, pz), pxz = cmul(px, pz), pxy = cmul(px, py);
        E0 = cmul(E0, px); E1 = cmul(E1, py); E2 = cmul(E2, pz);
        J0 = cmul(J0, px); J1 = cmul(J1, py); J2 = cmul(J2, pz);
        B0 = cmul(B0, pyz); B1 = cmul(B1, pxz); B2 = cmul(B2, pxy);
    }
    // khat x B, khat x E, khat x J, khat.E, khat.J
    const cpx<T> hB0 = scale(B2, hy) - scale(B1, hz), hB1 = scale(B0, hz) - scale(B2, hx), hB2 = scale(B1, hx) - scale(B0, hy);
    const cpx<T> hE0 = scale(E2, hy) - scale(E1, hz), hE1 = scale(E0, hz) - scale(E2, hx), hE2 = scale(E1, hx) - scale(E0, hy);
    const cpx<T> hJ0 = scale(J2, hy) - scale(J1, hz), hJ1 = scale(J0, hz) - scale(J2, hx), hJ2 = scale(J1, hx) - scale(J0, hy);
    const cpx<T> dE = scale(E0, hx) + scale(E1, hy) + scale(E2, hz);
    const cpx<T> dJ = scale(J0, hx) + scale(J1, hy) + scale(J2, hz);
    // Eq. 1a: E' = C E + i S khat x B - S/k J + (1-C) khat (khat.E) + khat (khat.J)(S/k - dt)
    const cpx<T> lo = scale(dE, omC) + scale(dJ, Dk);
    cpx<T> F0 = scale(E0, C) + scale(mul_i(hB0), S) - scale(J0, Sk) + scale(lo, hx);
    cpx<T> F1 = scale(E1, C) + scale(mul_i(hB1), S) - scale(J1, Sk) + scale(lo, hy);
    cpx<T> F2 = scale(E2, C) + scale(mul_i(hB2), S) - scale(J2, Sk) + scale(lo, hz);
    // Eq. 1b: B' = C B - i S khat x E + i (1-C)/k khat x J
    cpx<T> G0 = scale(B0, C) - scale(mul_i(hE0), S) + scale(mul_i(hJ0), omCk);
    cpx<T> G1 = scale(B1, C) - scale(mul_i(hE1), S) + scale(mul_i(hJ1), omCk);
    cpx<T> G2 = scale(B2, C) - scale(mul_i(hE2), S) + scale(mul_i(hJ2), omCk);
    if (nf > 9) {
        // Gauss residual i[k].E' - rho on the unnormalised spectrum
        const cpx<T> rho = p[9 * fs];
        const cpx<T> div = mul_i(scale(F0, kx) + scale(F1, ky) + scale(F2, kz));
        const T rx = fma_t(div.x, Nfull, -rho.x);
        const T ry = fma_t(div.y, Nfull, -rho.y);
        const T wgt = (xp == 0 || xp == lxh - 1) ? T(1) : T(2);
        g_res += wgt * (rx * rx + ry * ry);
        g_rho += wgt * (rho.x * rho.x + rho.y * rho.y);
    }
    if (a.staggered) {
        const cpx<T> pyz = cmul(py, pz), pxz = cmul(px, pz), pxy = cmul(px, py);
        F0 = cmulc(F0, px); F1 = cmulc(F1, py); F2 = cmulc(F2, pz);
        G0 = cmulc(G0, pyz); G1 = cmulc(G1, pxz); G2 = cmulc(G2, pxy);
    }
    p[0] = F0; p[fs] = F1; p[2 * fs] = F2;
    p[3 * fs] = G0; p[4 * fs] = G1; p[5 * fs] = G2;
}

template <typename T, class G>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? PSATD_MINB_B : 2) k_pass_b(Args<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ SubDesc d;
    __shared__ T red[2 * (kThreads / 32)];
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<1>(a, it, &d);
        const G g(d);
        const int Lx = g.Lx, Ly = g.Ly, Lz = g.Lz;
        const int M = g.M, lgM = g.lgM, Q = g.q, lxh = g.lxh;
        const int q0 = int(it - d.itemB) * M;
        const int mc = min(M, Q - q0);
        const int nf = a.nf;
        const int fs = g.fs;                           // padded field stride in shared memory
        cpx<T>* spec = a.spec + d.spec_off;
        const bool pairs = sizeof(T) == 4 && (Q & 1) == 0 && M >= 2 && (M & 1) == 0 && nf * (M >> 1) <= kThreads;
        const int MP = M >> 1;
        if (pairs) {
            // pairs of modes (16-byte aligned: Q, q0 and M are even),
            // zero-filled past the ragged end of the plane; thread (field f,
            // phase r, pair m2) copies rows r, r + R, ... of its mode pair, so
            // that consecutive lanes read consecutive pairs of one row
            const int ncol = nf * MP, R = kThreads / ncol;
            const int m2 = int(threadIdx.x) % MP, fr = int(threadIdx.x) / MP;
            const int f = fr / R, r = fr - f * R, c = f * MP + m2;
            if (c < ncol) {
                const int nb = min(max(mc - 2 * m2, 0), 2) * int(sizeof(cpx<T>));
                const cpx<T>* src = spec + int64_t(f) * Lz * Q + q0 + (nb ? 2 * m2 : 0) + int64_t(r) * Q;
                cpx<T>* dst = sm + f * fs + 2 * m2 + r * M;
                const int64_t step = int64_t(R) * Q;
                for (int z = r; z < Lz; z += R, src += step, dst += R * M) cp_async16(dst, src, nb);
            }
        }
        for (int f = 0; f < nf && !pairs; ++f) {
            const cpx<T>* src = spec + int64_t(f) * Lz * Q + q0;
            cpx<T>* s = sm + f * fs;
            {
                loop2(M, Lz, [&](int z, int m) {
                    const cpx<T>* g = src + int64_t(z) * Q + (m < mc ? m : 0);
                    if constexpr (sizeof(T) == 4) cp_async8z(s + z * M + m, g, m < mc ? 8 : 0);
                    else cp_async16(s + z * M + m, g, m < mc ? 16 : 0);
                });
            }
        }
        cp_async_commit();
        // all fields in one batch: the stages' items spread over the block
        // with fewer partly idle rounds than two batches of 6 and nf - 6
        // (transforming E and B while J and rho were still arriving was
        // 1-5% slower)
        cp_async_wait_all();
        __syncthreads();
        fft_fwd<true, T, G::kThree>(sm, g.az, Batch{nf * M, 1, lgM, fs, M, M}, a.tw);

        const int64_t NM = int64_t(Lz) * Q;
        const T Nfull = T(double(Lx) * double(Ly) * double(Lz));
        // Gauss partial sums in the stage's precision (FP64 throughput is a
        // small fraction of FP32 on this part); one FMA forms the residual
        // with a single rounding; the per-item sums are accumulated in FP64
        // by the reduction kernel
        T g_res = T(0), g_rho = T(0);
        if (lgM >= 0 && M <= kThreads) {
            // a power-of-two chunk divides the block: each thread keeps one
            // mode (its plane position is fixed over the z loop)
            const int m = int(threadIdx.x) & (M - 1);
            if (m < mc) {
                const int q = q0 + m, yp = q / lxh, xp = q - yp * lxh;
                for (int zp = int(threadIdx.x) >> lgM; zp < Lz; zp += kThreads >> lgM)
                    eq1_mode(a, d, sm + zp * M + m, fs, q, yp, xp, zp, lxh, Ly, NM, int64_t(Q), Nfull, g_res, g_rho);
            }
        } else {
            loop2(M, Lz, [&](int zp, int m) {
                if (m >= mc) return;
                const int q = q0 + m, yp = q / lxh;
                eq1_mode(a, d, sm + zp * M + m, fs, q, yp, q - yp * lxh, zp, lxh, Ly, NM, int64_t(Q), Nfull, g_res,
                         g_rho);
            });
        }
        __syncthreads();
        fft_inv<true, T, G::kThree>(sm, g.az, Batch{6 * M, 1, lgM, fs, M, M}, a.tw);
        const int ng = g.ngz, nz = g.nvz;
        if (pairs) {
            // valid z planes of E and B as 16-byte mode pairs: thread (field
            // f, phase r, pair m2) stores rows ng + r, ng + r + R, ...
            const int ncol = 6 * MP, R = kThreads / ncol;
            const int m2 = int(threadIdx.x) % MP, fr = int(threadIdx.x) / MP;
            const int f = fr / R, r = fr - f * R, c = f * MP + m2;
            if (c < ncol && 2 * m2 + 1 < mc) {
                cpx<T>* dst = spec + int64_t(f) * Lz * Q + int64_t(ng + r) * Q + q0 + 2 * m2;
                const cpx<T>* src = sm + f * fs + (ng + r) * M + 2 * m2;
                const int64_t step = int64_t(R) * Q;
                for (int z = r; z < nz; z += R, dst += step, src += R * M)
                    __stcs(reinterpret_cast<float4*>(dst), *reinterpret_cast<const float4*>(src));
            } else if (c < ncol && 2 * m2 < mc) {     // a ragged plane end inside the pair
                cpx<T>* dst = spec + int64_t(f) * Lz * Q + int64_t(ng + r) * Q + q0 + 2 * m2;
                const cpx<T>* src = sm + f * fs + (ng + r) * M + 2 * m2;
                for (int z = r; z < nz; z += R, dst += int64_t(R) * Q, src += R * M) stcs_c(dst, *src);
            }
        }
        for (int f = 0; f < 6 && !pairs; ++f) {
            cpx<T>* dst = spec + int64_t(f) * Lz * Q + int64_t(ng) * Q + q0;
            const cpx<T>* s = sm + f * fs + ng * M;
            loop2(M, nz, [&](int zv, int m) {
                if (m < mc) stcs_c(dst + int64_t(zv) * Q + m, s[zv * M + m]);
            });
        }
        if (nf > 9) {
            block_sum2(g_res, g_rho, red);
            if (threadIdx.x == 0) {
                a.gauss_part[2 * it] = double(g_res);
                a.gauss_part[2 * it + 1] = double(g_rho);
            }
        }
        __syncthreads();
    }
}


// ---- pass B of the heat equation: z transforms and the exact decay ----------
// Same chunking as pass B.  Per mode T~' = A T~ + B S~ with A = exp(-x) and
// B = (1 - exp(-x))/x, x = D dt |[k]|^2 (both scaled by 1/(Lx Ly Lz)), read
// from the first two coefficient arrays; S is the optional source (field 1).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pass_b_heat(Args<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ SubDesc d;
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<1>(a, it, &d);
        const GeoDyn g(d);
        const int Lz = g.Lz, M = g.M, lgM = g.lgM, Q = g.q;
        const int q0 = int(it - d.itemB) * M;
        const int mc = min(M, Q - q0);
        const int nf = a.nf, fs = g.fs;
        cpx<T>* spec = a.spec + d.spec_off;
        for (int f = 0; f < nf; ++f) {
            const cpx<T>* src = spec + int64_t(f) * Lz * Q + q0;
            cpx<T>* s = sm + f * fs;
            if (sizeof(T) == 4 && (Q & 1) == 0 && M >= 2 && (M & 1) == 0) {
                // pairs of modes, 16-byte copies (Q, q0 and M even), zero-filled
                // past the ragged end of the plane
                loop2(M >> 1, Lz, [&](int z, int m2) {
                    const int nb = min(max(mc - 2 * m2, 0), 2) * int(sizeof(cpx<T>));
                    const cpx<T>* gp = src + int64_t(z) * Q + (nb ? 2 * m2 : 0);
                    cp_async16(s + z * M + 2 * m2, gp, nb);
                });
            } else {
                loop2(M, Lz, [&](int z, int m) {
                    const cpx<T>* gp = src + int64_t(z) * Q + (m < mc ? m : 0);
                    if constexpr (sizeof(T) == 4) cp_async8z(s + z * M + m, gp, m < mc ? 8 : 0);
                    else cp_async16(s + z * M + m, gp, m < mc ? 16 : 0);
                });
            }
        }
        cp_async_wait_all();
        __syncthreads();
        fft_fwd<true>(sm, g.az, Batch{nf * M, 1, lgM, fs, M, M}, a.tw);
        const int64_t NM = int64_t(Lz) * Q;
        loop2(M, Lz, [&](int zp, int m) {
            if (m >= mc) return;
            const T* __restrict__ tb = a.tab + d.tab_coef + int64_t(zp) * Q + q0 + m;
            cpx<T>* p = sm + zp * M + m;
            cpx<T> v = scale(p[0], __ldg(tb));
            if (nf > 1) v = v + scale(p[fs], __ldg(tb + NM));
            p[0] = v;
        });
        __syncthreads();
        fft_inv<true>(sm, g.az, Batch{M, 1, lgM, fs, M, M}, a.tw);
        {
            const int ngz = g.ngz, nz = g.nvz;
            cpx<T>* dst = spec + int64_t(ngz) * Q + q0;
            const cpx<T>* s = sm + ngz * M;
            loop2(M, nz, [&](int zv, int m) {
                if (m < mc) stcs_c(dst + int64_t(zv) * Q + m, s[zv * M + m]);
            });
        }
        __syncthreads();
    }
}

// ---- pass C: inverse y and x transforms, fused guard replacement ------------
template <typename T, class G>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? PSATD_MINB_C : 2) k_pass_c(Args<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ SubDesc d;
    __shared__ Segment segs[kSegSmem];
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<2>(a, it, &d);
        const G g(d);
        const int Lx = g.Lx, Ly = g.Ly, Lz = g.Lz;
        const int nz = g.nvz, ny = g.nvy, ng = g.ng;
        const int ngz = g.ngz;
        const int loc = int(it - d.itemC);
        const int f = loc / nz, z = ngz + (loc - (loc / nz) * nz);
        const int h = g.h, pitch = g.pitch, lxh = g.lxh;
        const cpx<T>* src = a.spec + d.spec_off + int64_t(f * Lz + z) * g.q;
        loop2(lxh, Ly, [&](int y, int c) { cp_async_c(sm + y * pitch + c, src + y * lxh + c); });
        // this subdomain's exchange segments (the first kSegSmem of them)
        const int nsg = min(d.seg_end - d.seg_begin, kSegSmem);
        {
            const int* gs = reinterpret_cast<const int*>(a.segs + d.seg_begin);
            int* ss = reinterpret_cast<int*>(segs);
            for (int i = threadIdx.x; i < nsg * int(sizeof(Segment) / 4); i += kThreads) ss[i] = __ldg(gs + i);
        }
        cp_async_wait_all();
        __syncthreads();
        fft_inv<false, T, G::kThree>(sm, g.ay, Batch{lxh, 1, 0, 0, pitch, 1}, a.tw);
        // merge the half spectrum of the valid rows into the packed form
        cpx<T>* rows = sm + ng * pitch;
        real_merge_rows(rows, ny, pitch, h, g.ax, a.tw + d.tw_post);
        __syncthreads();
        fft_inv<false, T, G::kThree>(rows, g.ax, Batch{ny, pitch, 0, 0, 1, 1}, a.tw);
        // store the valid cells of this plane to every box that holds them
        T* out = a.eb[f];
        const T* rp = reinterpret_cast<const T*>(sm);
        const int rs = 2 * pitch;                         // real row stride
        for (int g = 0; g < d.seg_end - d.seg_begin; ++g) {
            const Segment& sg = g < kSegSmem ? segs[g] : a.segs[d.seg_begin + g];
            if (a.own_only && !sg.identity) continue;
            if (z < sg.z0 || z >= sg.z0 + sg.ez) continue;
            T* dst = out + sg.dst_off + (int64_t(z + sg.dz) * sg.dLy + sg.y0 + sg.dy) * sg.dLx + sg.x0 + sg.dx;
            const T* sp = rp + sg.y0 * rs + sg.x0;
            if (!sg.vec4) {
                loop2(sg.ex, sg.ey, [&](int yy, int xx) { __stcs(dst + int64_t(yy) * sg.dLx + xx, sp[yy * rs + xx]); });
            } else if (!store_rows_pow2<kThreads>(dst, sg.dLx, sp, rs, sg.ex >> 2, sg.ey)) {
                loop2(sg.ex >> 2, sg.ey, [&](int yy, int x4) {
                    const cpx<T> u = *reinterpret_cast<const cpx<T>*>(sp + yy * rs + 4 * x4);
                    const cpx<T> w = *reinterpret_cast<const cpx<T>*>(sp + yy * rs + 4 * x4 + 2);
                    stcs4(dst + int64_t(yy) * sg.dLx + 4 * x4, cpx4<T>{u.x, u.y, w.x, w.y});
                });
            }
        }
        __syncthreads();
    }
}


// ---- split-plane schedule: planes larger than shared memory -----------------
// Passes A and C stage a whole (x, y) plane of one field in shared memory.
// When a plane does not fit (a large box, e.g. one box over the whole grid,
// the global solver), each of them is done in two launches instead: row
// items transform a block of `rows` rows of a plane along x, column items
// transform `cols` half-spectrum columns of a plane along y in place in the
// spectra block.  Pass B is unchanged.  Forward: stage 4 (x rows, real split)
// then stage 5 (y columns); inverse: stage 6 (y columns, valid rows stored)
// then stage 7 (real merge, x rows, the exchange scatter of pass C).

// stage 4: x (real) transforms of a block of rows of one input plane
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rows_fwd(Args<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ SubDesc d;
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<4>(a, it, &d);
        const GeoDyn g(d);
        const int R = d.rows, nb = (g.Ly + R - 1) / R;
        const int loc = int(it - d.itemA);
        const int pl = loc / nb, rb = loc - pl * nb;
        const int f = pl / g.Lz, z = pl - f * g.Lz;
        const int y0 = rb * R, nr = min(R, g.Ly - y0);
        const int h = g.h, pitch = g.pitch, lxh = g.lxh;
        const cpx<T>* src = reinterpret_cast<const cpx<T>*>(field_in(a, f) + d.field_off +
                                                            (int64_t(z) * g.Ly + y0) * g.Lx);
        loop2(h, nr, [&](int y, int m) { cp_async_c(sm + y * pitch + m, src + y * h + m); });
        cp_async_wait_all();
        __syncthreads();
        fft_fwd<false>(sm, g.ax, Batch{nr, pitch, 0, 0, 1, 1}, a.tw);
        real_split_rows(sm, nr, pitch, h, g.ax, a.tw + d.tw_post);
        __syncthreads();
        cpx<T>* dst = a.spec + d.spec_off + int64_t(f * g.Lz + z) * g.q + int64_t(y0) * lxh;
        loop2(lxh, nr, [&](int y, int c) { stcs_c(dst + y * lxh + c, sm[y * pitch + c]); });
        __syncthreads();
    }
}

// stages 5 (forward, every plane of the nf input fields) and 6 (inverse, the
// valid z planes of the six outputs): y transforms of `cols` columns of one
// plane; the inverse stores only the valid rows, the only ones stage 7 reads
template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) k_cols(Args<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ SubDesc d;
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<INV ? 6 : 5>(a, it, &d);
        const GeoDyn g(d);
        const int W = d.cols, lxh = g.lxh, Ly = g.Ly, nb = (lxh + W - 1) / W;
        const int loc = int(it - (INV ? d.itemC1 : d.itemA2));
        const int pl = loc / nb, cb = loc - pl * nb;
        int f, z;
        if (INV) { f = pl / g.nvz; z = g.ngz + (pl - f * g.nvz); }
        else { f = pl / g.Lz; z = pl - f * g.Lz; }
        const int c0 = cb * W, wc = min(W, lxh - c0);
        cpx<T>* base = a.spec + d.spec_off + int64_t(f * g.Lz + z) * g.q + c0;
        loop2(W, Ly, [&](int y, int m) {
            const cpx<T>* src = base + int64_t(y) * lxh + (m < wc ? m : 0);
            if constexpr (sizeof(T) == 4) cp_async8z(sm + y * W + m, src, m < wc ? 8 : 0);
            else cp_async16(sm + y * W + m, src, m < wc ? 16 : 0);
        });
        cp_async_wait_all();
        __syncthreads();
        if constexpr (INV) fft_inv<false>(sm, g.ay, Batch{W, 1, 0, 0, W, 1}, a.tw);
        else fft_fwd<false>(sm, g.ay, Batch{W, 1, 0, 0, W, 1}, a.tw);
        const int ya = INV ? g.ng : 0, ny = INV ? g.nvy : Ly;
        loop2(W, ny, [&](int y, int m) {
            if (m < wc) stcs_c(base + int64_t(ya + y) * lxh + m, sm[(ya + y) * W + m]);
        });
        __syncthreads();
    }
}

// stage 7: real merge and inverse x transforms of a block of valid rows of one
// output plane, then the store of pass C (own box and every guard image)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rows_inv(Args<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ SubDesc d;
    __shared__ Segment segs[kSegSmem];
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<7>(a, it, &d);
        const GeoDyn g(d);
        const int R = d.rows, nb = (g.nvy + R - 1) / R;
        const int loc = int(it - d.itemC);
        const int pl = loc / nb, rb = loc - pl * nb;
        const int f = pl / g.nvz, z = g.ngz + (pl - f * g.nvz);
        const int ya = g.ng + rb * R, nr = min(R, g.ng + g.nvy - ya);
        const int h = g.h, pitch = g.pitch, lxh = g.lxh;
        const cpx<T>* src = a.spec + d.spec_off + int64_t(f * g.Lz + z) * g.q + int64_t(ya) * lxh;
        loop2(lxh, nr, [&](int y, int c) { cp_async_c(sm + y * pitch + c, src + y * lxh + c); });
        const int nsg = min(d.seg_end - d.seg_begin, kSegSmem);
        {
            const int* gs = reinterpret_cast<const int*>(a.segs + d.seg_begin);
            int* ss = reinterpret_cast<int*>(segs);
            for (int i = threadIdx.x; i < nsg * int(sizeof(Segment) / 4); i += kThreads) ss[i] = __ldg(gs + i);
        }
        cp_async_wait_all();
        __syncthreads();
        real_merge_rows(sm, nr, pitch, h, g.ax, a.tw + d.tw_post);
        __syncthreads();
        fft_inv<false>(sm, g.ax, Batch{nr, pitch, 0, 0, 1, 1}, a.tw);
        T* out = a.eb[f];
        const T* rp = reinterpret_cast<const T*>(sm);
        const int rs = 2 * pitch;                         // real row stride
        for (int k = 0; k < d.seg_end - d.seg_begin; ++k) {
            const Segment& sg = k < kSegSmem ? segs[k] : a.segs[d.seg_begin + k];
            if (a.own_only && !sg.identity) continue;
            if (z < sg.z0 || z >= sg.z0 + sg.ez) continue;
            const int y_lo = max(sg.y0, ya), y_hi = min(sg.y0 + sg.ey, ya + nr);
            if (y_lo >= y_hi) continue;
            T* dst = out + sg.dst_off + (int64_t(z + sg.dz) * sg.dLy + y_lo + sg.dy) * sg.dLx + sg.x0 + sg.dx;
            const T* sp = rp + (y_lo - ya) * rs + sg.x0;
            if (!sg.vec4) {
                loop2(sg.ex, y_hi - y_lo, [&](int yy, int xx) { __stcs(dst + int64_t(yy) * sg.dLx + xx, sp[yy * rs + xx]); });
            } else if (!store_rows_pow2<kThreads>(dst, sg.dLx, sp, rs, sg.ex >> 2, y_hi - y_lo)) {
                loop2(sg.ex >> 2, y_hi - y_lo, [&](int yy, int x4) {
                    const cpx<T> u = *reinterpret_cast<const cpx<T>*>(sp + yy * rs + 4 * x4);
                    const cpx<T> w = *reinterpret_cast<const cpx<T>*>(sp + yy * rs + 4 * x4 + 2);
                    stcs4(dst + int64_t(yy) * sg.dLx + 4 * x4, cpx4<T>{u.x, u.y, w.x, w.y});
                });
            }
        }
        __syncthreads();
    }
}

// ---- standalone guard exchange ---------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_exchange(Args<T> a) {
    __shared__ int64_t s_ticket[2];
    Tickets<T> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        int lo = 0, hi = a.nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.segs[mid].item <= it) lo = mid; else hi = mid - 1;
        }
        const Segment& sg = a.segs[lo];
        const SubDesc& sd = a.subs[sg.src];
        const int z = sg.z0 + int(it - sg.item);
        for (int f = 0; f < a.nout; ++f) {
            T* fld = a.eb[f];
            const T* src = fld + sd.field_off + (int64_t(z) * sd.L[1] + sg.y0) * sd.L[0] + sg.x0;
            T* dst = fld + sg.dst_off + (int64_t(z + sg.dz) * sg.dLy + sg.y0 + sg.dy) * sg.dLx + sg.x0 + sg.dx;
            loop2(sg.ex, sg.ey, [&](int yy, int xx) { dst[int64_t(yy) * sg.dLx + xx] = src[int64_t(yy) * sd.L[0] + xx]; });
        }
        __syncthreads();
    }
}

// ---- per-subdomain reduction of the Gauss partial sums ----------------------
static __global__ void k_gauss_reduce(const SubDesc* __restrict__ subs, int nsub, const double* __restrict__ part,
                               double* __restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int l = threadIdx.x & 31;
    if (w >= nsub) return;
    const int64_t b = subs[w].itemB;
    const int64_t end = b + (int64_t(subs[w].q) + subs[w].chunkB - 1) / subs[w].chunkB;
    double s1 = 0, s2 = 0;
    for (int64_t i = b + l; i < end; i += 32) { s1 += part[2 * i]; s2 += part[2 * i + 1]; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (l == 0) { out[2 * w] = s1; out[2 * w + 1] = s2; }
}


// ---- launch helpers shared by the per-precision instantiation files ----------
template <typename T>
static Args<T> make_args(const LaunchCommon& c, int64_t item0, int64_t nitems) {
    Args<T> a;
    a.subs = static_cast<const SubDesc*>(c.subs);
    a.segs = static_cast<const Segment*>(c.segs);
    a.tw = static_cast<const twd<T>*>(c.tw);
    a.tab = static_cast<const T*>(c.tab);
    a.tabc = static_cast<const cpx<T>*>(c.tabc);
    a.spec = static_cast<cpx<T>*>(c.spec);
    for (int i = 0; i < 6; ++i) a.eb[i] = static_cast<T*>(c.eb[i]);
    for (int i = 0; i < 4; ++i) a.jr[i] = static_cast<const T*>(c.jr[i]);
    a.gauss_part = c.gauss_part;
    a.work = c.work;
    a.err = c.err;
    a.persistent = c.persistent;
    a.item0 = item0;
    for (int i = 0; i < 5; ++i) a.per_sub[i] = c.per_sub[i];
    a.nitems = nitems;
    a.nsub = c.nsub;
    a.nseg = c.nseg;
    a.nf = c.nf;
    a.nout = c.nout;
    a.staggered = c.staggered;
    a.own_only = c.own_only;
    return a;
}

static inline unsigned grid_for(int64_t n) { return unsigned(n < 2147483647 ? n : 2147483647); }

static inline cudaError_t set_smem_attr(const void* fn, int bytes) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

// Per device and kernel: the dynamic shared memory granted so far and the
// occupancy found for it, so that repeated launches make no attribute calls.
struct LaunchCache {
    const void* fn;
    int dev, smem_set, smem_occ, per_sm, nsm;
};

static cudaError_t launch_shape(const void* fn, int smem, bool persistent, int* resident, int threads = kThreads) {
    static std::mutex mu;
    static LaunchCache cache[128];
    static int ncache = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    LaunchCache* c = nullptr;
    for (int i = 0; i < ncache; ++i)
        if (cache[i].fn == fn && cache[i].dev == dev) c = &cache[i];
    LaunchCache fresh{fn, dev, -1, -1, 0, 0};
    if (!c) c = ncache < 128 ? &cache[ncache++] : &fresh;
    if (c->fn != fn || c->dev != dev) *c = fresh;
    if (smem > c->smem_set) {
        if ((e = set_smem_attr(fn, smem)) != cudaSuccess) return e;
        c->smem_set = smem;
    }
    if (persistent && smem != c->smem_occ) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->per_sm, fn, threads, smem)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        c->smem_occ = smem;
    }
    *resident = (c->per_sm > 0 ? c->per_sm : 1) * c->nsm;
    return cudaSuccess;
}

// One launch of kernel k: persistent (as many CTAs as can be resident, each
// drawing work items from the ticket counter) or one CTA per item.
template <typename T>
static cudaError_t launch_kernel(void (*k)(Args<T>), const Args<T>& a, int smem, cudaStream_t st, int threads = kThreads) {
    int resident = 0;
    cudaError_t e = launch_shape((const void*)k, smem, a.persistent != 0, &resident, threads);
    if (e != cudaSuccess) return e;
    unsigned grid = grid_for(a.nitems);
    if (a.persistent) grid = grid_for(a.nitems < resident ? a.nitems : resident);
    k<<<grid, threads, smem, st>>>(a);
    return cudaPeekAtLastError();
}

// Launch stage `stage` (see stage_item) with geometry G; the exchange and the
// split-plane stages always read the geometry from the descriptors.
template <typename T, class G>
static cudaError_t launch_geo(int stage, const Args<T>& a, int smem, cudaStream_t st) {
    switch (stage) {
        case 0: return launch_kernel<T>(k_pass_a<T, G>, a, smem, st);
        case 1: return launch_kernel<T>(k_pass_b<T, G>, a, smem, st);
        case 2: return launch_kernel<T>(k_pass_c<T, G>, a, smem, st);
        case 4: return launch_kernel<T>(k_rows_fwd<T>, a, smem, st);
        case 5: return launch_kernel<T>(k_cols<T, false>, a, smem, st);
        case 6: return launch_kernel<T>(k_cols<T, true>, a, smem, st);
        case 7: return launch_kernel<T>(k_rows_inv<T>, a, smem, st);
        case 8: return launch_kernel<T>(k_pass_b_heat<T>, a, smem, st);
        default: return launch_kernel<T>(k_exchange<T>, a, 0, st);
    }
}

}  // namespace psatd
