#pragma once
// Plane stages of the FP32 push with thread-private transforms of
// compile-time length (passes A and C, Sec. 3.2 of arXiv:1707.08500).
//
// The generic plane stages (psatd_kernels.cuh) run every 1D transform as
// batched shared-memory stages whose work items are spread over all threads
// of a CTA; the index arithmetic of that mapping and the twiddle loads cost
// as many instructions as the butterflies.  Here one thread owns one whole
// transform instead:
//
//   x (rows):     thread y does the packed half-length complex FFT of row y
//                 and the real split (forward), or the real merge and the
//                 inverse (pass C), entirely on its own row, so the x phase
//                 needs no barrier;
//   y (columns):  a thread works on a pair of adjacent half-spectrum
//                 columns; the four warps take every fourth f1-point and
//                 every fourth f2-point DFT of the 32 column pairs.
//
// The DFT bodies are unrolled for the axis lengths listed in kRegX2 / kRegY
// (compiled per length, dispatched per work item); the loops over them run
// at run time, so the code that one length executes stays small, and the
// twiddles come from the plan's pool.  The position order of the spectra
// (frequency k1 + f1 k2 at position k1 f2 + k2, f1 = split_first(n)) is the
// one of the generic kernels, so pass B and the coefficient tables are
// unchanged.  Planes move between global and shared memory with bulk
// asynchronous copies (cp.async.bulk) completing on an mbarrier; the wait is
// bounded and a timeout sets PSATD_CHECK_WAIT in the device error word.
#include "psatd_kernels.cuh"

#ifndef PSATD_MINB_REG
#define PSATD_MINB_REG 5
#endif

namespace psatd {

// ---- bulk copies completing on an mbarrier ------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// generic-proxy accesses of shared memory before this point are ordered
// before later async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// global -> shared, `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(smem_u32(dst)), "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

constexpr int kWaitSpins = 1 << 22;   // bounded wait on a bulk copy (each try also suspends briefly)
constexpr unsigned kErrWait = 4u;     // PSATD_CHECK_WAIT

// Thread 0 waits for phase `parity` of *bar, at most kWaitSpins tries; on a
// timeout it sets the error bit, waits once more (bounded) for the copies in
// flight, and every thread of the CTA gets false.  Ends with __syncthreads.
__device__ __forceinline__ bool wait_bulk(uint64_t* bar, unsigned parity, unsigned* err, int* s_ok) {
    if (threadIdx.x == 0) {
        int ok = 0;
        for (int i = 0; i < kWaitSpins && !ok; ++i) ok = mbar_try(bar, parity);
        if (!ok) {
            atomicOr(err, kErrWait);
            bool done = false;
            for (int i = 0; i < kWaitSpins && !done; ++i) done = mbar_try(bar, parity);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// ---- compile-time dispatch over the compiled axis lengths ---------------------
// f(integral_constant<int, n>) for n in kRegX2 (local x lengths) or kRegY
// (local y lengths); false if n is not compiled.
template <int I, class F>
__device__ __forceinline__ bool dispatch_x(int n, F&& f) {
    if constexpr (I < int(sizeof(kRegX2) / sizeof(int))) {
        constexpr int v = kRegX2[I];
        if (n == v) { f(std::integral_constant<int, v>{}); return true; }
        return dispatch_x<I + 1>(n, f);
    } else {
        return false;
    }
}
template <int I, class F>
__device__ __forceinline__ bool dispatch_y(int n, F&& f) {
    if constexpr (I < int(sizeof(kRegY) / sizeof(int))) {
        constexpr int v = kRegY[I];
        if (n == v) { f(std::integral_constant<int, v>{}); return true; }
        return dispatch_y<I + 1>(n, f);
    } else {
        return false;
    }
}

__device__ __forceinline__ float4 lds4(const cpx<float>* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(cpx<float>* p, cpx<float> a, cpx<float> b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}

// ---- x: one row per thread -----------------------------------------------------
// The twiddles come from the plan's pool: tw = exp(-2 pi i m/H), m = 0..H-1
// (the axis table), wp = exp(-2 pi i k/Lx) for the frequency k at every
// position of the packed transform (the real-split table); both as FP32
// hi + lo pairs.  Outer loops run at run time so that the code of one length
// stays small; the DFT bodies are unrolled.

// Real split of one pair of positions of the packed transform: A = Z[pa],
// B = Z[pb] (pb the partner of pa); X[pa] = e + w o, X[pb] = conj(e - w o)
// with e = (A + conj B)/2, o = (A - conj B)/(2i), w the real-split twiddle of pa.
__device__ __forceinline__ void split_pair_c(cpx<float> A, cpx<float> B, const twd<float>& w, cpx<float>& outA,
                                             cpx<float>& outB) {
    const cpx<float> Bc = conj(B);
    const cpx<float> e = scale(A + Bc, 0.5f);
    const cpx<float> dd = A - Bc;
    const cpx<float> wo = mul_tw(mk(0.5f * dd.y, -0.5f * dd.x), w);
    outA = e + wo;
    outB = conj(e - wo);
}
// Inverse of split_pair_c: X[pa] = A, X[pb] = B -> Z[pa] = e + i o,
// Z[pb] = conj(e) + i conj(o), e = A + conj B, o = (A - conj B) conj(w).
__device__ __forceinline__ void merge_pair_c(cpx<float> A, cpx<float> B, const twd<float>& w, cpx<float>& outA,
                                             cpx<float>& outB) {
    const cpx<float> Bc = conj(B);
    const cpx<float> e = A + Bc;
    const cpx<float> o = mul_tw_conj(A - Bc, w);
    outA = e + mul_i(o);
    outB = conj(e) + mul_i(conj(o));
}

// Forward real transform of one row: row[0..H) holds z[m] = x[2m] + i x[2m+1]
// (16-byte aligned); on return row[0..H] holds the half spectrum X[0..H] in
// position order.
template <int H>
__device__ __forceinline__ void row_fwd(cpx<float>* row, const twd<float>* __restrict__ tw,
                                        const twd<float>* __restrict__ wp) {
    constexpr int F1 = split_first(H), F2 = H / F1;
    static_assert(F1 > 1 && F2 % 2 == 0, "compiled x lengths need an even second factor");
    // stage 1: F1-point DFTs at stride F2, two at a time (j, j+1), then w^{j r}
#pragma unroll 1
    for (int j = 0; j < F2; j += 2) {
        cpx<float> a[F1], b[F1];
#pragma unroll
        for (int r = 0; r < F1; ++r) {
            const float4 v = lds4(row + j + F2 * r);
            a[r] = mk(v.x, v.y);
            b[r] = mk(v.z, v.w);
        }
        Dft<F1, false>::run(a);
        Dft<F1, false>::run(b);
        sts4(row + j, a[0], b[0]);
#pragma unroll
        for (int r = 1; r < F1; ++r)
            sts4(row + j + F2 * r, mul_tw(a[r], ld_tw(tw + j * r)), mul_tw(b[r], ld_tw(tw + (j + 1) * r)));
    }
    // stage 2 (F2-point DFTs on contiguous blocks) fused with the real split:
    // block k1 pairs with block F1 - k1, block 0 with itself
    auto load_dft = [&](int k1, cpx<float>* v) {
#pragma unroll
        for (int i = 0; i < F2; i += 2) {
            const float4 q = lds4(row + k1 * F2 + i);
            v[i] = mk(q.x, q.y);
            v[i + 1] = mk(q.z, q.w);
        }
        Dft<F2, false>::run(v);
    };
    {
        cpx<float> v[F2], o[F2];
        load_dft(0, v);
        const cpx<float> z0 = v[0];
        o[0] = mk(z0.x + z0.y, 0.f);
        // positions P and F2 - P hold frequencies F1 P and H - F1 P
#pragma unroll
        for (int P = 1; P <= F2 / 2; ++P) {
            cpx<float> oa, ob;
            split_pair_c(v[P], v[F2 - P], ld_tw(wp + P), oa, ob);
            o[P] = oa;
            if (P != F2 - P) o[F2 - P] = ob;
        }
#pragma unroll
        for (int i = 0; i < F2; i += 2) sts4(row + i, o[i], o[i + 1]);
        row[H] = mk(z0.x - z0.y, 0.f);
    }
    // position k1 F2 + k2 pairs with (F1 - k1) F2 + F2 - 1 - k2
#pragma unroll 1
    for (int k1 = 1; k1 < F1 - k1; ++k1) {
        const int kb = F1 - k1;
        cpx<float> va[F2], vb[F2];
        load_dft(k1, va);
        load_dft(kb, vb);
#pragma unroll
        for (int k2 = 0; k2 < F2; ++k2) {
            cpx<float> oa, ob;
            split_pair_c(va[k2], vb[F2 - 1 - k2], ld_tw(wp + k1 * F2 + k2), oa, ob);
            va[k2] = oa;
            vb[F2 - 1 - k2] = ob;
        }
#pragma unroll
        for (int i = 0; i < F2; i += 2) {
            sts4(row + k1 * F2 + i, va[i], va[i + 1]);
            sts4(row + kb * F2 + i, vb[i], vb[i + 1]);
        }
    }
    if constexpr (F1 % 2 == 0) {            // block F1/2 pairs with itself
        constexpr int k1 = F1 / 2;
        cpx<float> v[F2];
        load_dft(k1, v);
#pragma unroll
        for (int k2 = 0; k2 < F2 / 2; ++k2) {
            cpx<float> oa, ob;
            split_pair_c(v[k2], v[F2 - 1 - k2], ld_tw(wp + k1 * F2 + k2), oa, ob);
            v[k2] = oa;
            v[F2 - 1 - k2] = ob;
        }
#pragma unroll
        for (int i = 0; i < F2; i += 2) sts4(row + k1 * F2 + i, v[i], v[i + 1]);
    }
}

// Inverse of row_fwd (unnormalised): row[0..H] holds a half spectrum in
// position order (only the real parts of X[0] and X[H] are used); on return
// row[0..H) holds the packed real row z[m] = x[2m] + i x[2m+1].  8-byte
// accesses only (any pitch).
template <int H>
__device__ __forceinline__ void row_inv(cpx<float>* row, const twd<float>* __restrict__ tw,
                                        const twd<float>* __restrict__ wp) {
    constexpr int F1 = split_first(H), F2 = H / F1;
    static_assert(F1 > 1 && F2 % 2 == 0, "compiled x lengths need an even second factor");
    // the merge fused with the first inverse stage (F2-point DFTs on
    // contiguous blocks, then the twiddle conj(w^{r k}))
    auto dft_store = [&](int k, cpx<float>* v) {
        Dft<F2, true>::run(v);
        row[k * F2] = v[0];
#pragma unroll
        for (int r = 1; r < F2; ++r) row[k * F2 + r] = mul_tw_conj(v[r], ld_tw(tw + r * k));
    };
    {
        cpx<float> v[F2], o[F2];
#pragma unroll
        for (int i = 0; i < F2; ++i) v[i] = row[i];
        const float x0 = v[0].x, xh = row[H].x;
        o[0] = mk(x0 + xh, x0 - xh);
#pragma unroll
        for (int P = 1; P <= F2 / 2; ++P) {
            cpx<float> oa, ob;
            merge_pair_c(v[P], v[F2 - P], ld_tw(wp + P), oa, ob);
            o[P] = oa;
            if (P != F2 - P) o[F2 - P] = ob;
        }
        dft_store(0, o);
    }
#pragma unroll 1
    for (int k1 = 1; k1 < F1 - k1; ++k1) {
        const int kb = F1 - k1;
        cpx<float> va[F2], vb[F2];
#pragma unroll
        for (int i = 0; i < F2; ++i) {
            va[i] = row[k1 * F2 + i];
            vb[i] = row[kb * F2 + i];
        }
#pragma unroll
        for (int k2 = 0; k2 < F2; ++k2) {
            cpx<float> oa, ob;
            merge_pair_c(va[k2], vb[F2 - 1 - k2], ld_tw(wp + k1 * F2 + k2), oa, ob);
            va[k2] = oa;
            vb[F2 - 1 - k2] = ob;
        }
        dft_store(k1, va);
        dft_store(kb, vb);
    }
    if constexpr (F1 % 2 == 0) {
        constexpr int k1 = F1 / 2;
        cpx<float> v[F2];
#pragma unroll
        for (int i = 0; i < F2; ++i) v[i] = row[k1 * F2 + i];
#pragma unroll
        for (int k2 = 0; k2 < F2 / 2; ++k2) {
            cpx<float> oa, ob;
            merge_pair_c(v[k2], v[F2 - 1 - k2], ld_tw(wp + k1 * F2 + k2), oa, ob);
            v[k2] = oa;
            v[F2 - 1 - k2] = ob;
        }
        dft_store(k1, v);
    }
    // second inverse stage: F1-point DFTs at stride F2 -> natural order
#pragma unroll 1
    for (int j = 0; j < F2; ++j) {
        cpx<float> v[F1];
#pragma unroll
        for (int r = 0; r < F1; ++r) v[r] = row[j + F2 * r];
        Dft<F1, true>::run(v);
#pragma unroll
        for (int r = 0; r < F1; ++r) row[j + F2 * r] = v[r];
    }
}

// ---- y: column pairs, four threads per pair ------------------------------------
// Thread (pair c2, quarter q) works on columns 2 c2 and 2 c2 + 1 (the second
// may be past the half spectrum: it is then padding, computed on and never
// stored, or, with `tail` set, neither read nor written); quarter q takes
// every fourth stage-1 (stride) DFT and every fourth stage-2 (block) DFT.
// tw = exp(-2 pi i m/L), m = 0..L-1.

// element pair (columns c, c+1) of row y: one 16-byte access when the pitch
// is even, two 8-byte accesses otherwise (the second skipped for a tail column)
struct ColPair {
    cpx<float>* base;   // element (0, c)
    int P;              // row pitch (complex)
    bool v16, tail;
    __device__ __forceinline__ void ld(int y, cpx<float>& a, cpx<float>& b) const {
        cpx<float>* q = base + y * P;
        if (v16) {
            const float4 v = lds4(q);
            a = mk(v.x, v.y);
            b = mk(v.z, v.w);
        } else {
            a = q[0];
            b = tail ? mk(0.f, 0.f) : q[1];
        }
    }
    __device__ __forceinline__ void st(int y, cpx<float> a, cpx<float> b) const {
        cpx<float>* q = base + y * P;
        if (v16) {
            sts4(q, a, b);
        } else {
            q[0] = a;
            if (!tail) q[1] = b;
        }
    }
};

// forward, stage 1: F1-point DFTs at stride F2, twiddle w^{j r}, in place
template <int LY>
__device__ __forceinline__ void col_fwd1(const ColPair& cp, int q, const twd<float>* __restrict__ tw) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int j = q; j < F2; j += 4) {
        cpx<float> a[F1], b[F1];
#pragma unroll
        for (int r = 0; r < F1; ++r) cp.ld(j + F2 * r, a[r], b[r]);
        Dft<F1, false>::run(a);
        Dft<F1, false>::run(b);
        cp.st(j, a[0], b[0]);
#pragma unroll
        for (int r = 1; r < F1; ++r) {
            const twd<float> w = ld_tw(tw + j * r);
            cp.st(j + F2 * r, mul_tw(a[r], w), mul_tw(b[r], w));
        }
    }
}
// forward, stage 2: F2-point DFTs on contiguous blocks, written to global
// (row stride `ld` complex, columns c and c+1 at dst[0], dst[1]) in position order
template <int LY>
__device__ __forceinline__ void col_fwd2(const ColPair& cp, int q, cpx<float>* dst, int ld, bool second) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int k = q; k < F1; k += 4) {
        cpx<float> a[F2], b[F2];
#pragma unroll
        for (int r = 0; r < F2; ++r) cp.ld(k * F2 + r, a[r], b[r]);
        Dft<F2, false>::run(a);
        Dft<F2, false>::run(b);
#pragma unroll
        for (int r = 0; r < F2; ++r) {
            cpx<float>* d = dst + (k * F2 + r) * ld;
            stcs_c(d, a[r]);
            if (second) stcs_c(d + 1, b[r]);
        }
    }
}
// inverse, stage 1: F2-point DFTs on contiguous blocks, twiddle conj(w^{r k})
template <int LY>
__device__ __forceinline__ void col_inv1(const ColPair& cp, int q, const twd<float>* __restrict__ tw) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int k = q; k < F1; k += 4) {
        cpx<float> a[F2], b[F2];
#pragma unroll
        for (int r = 0; r < F2; ++r) cp.ld(k * F2 + r, a[r], b[r]);
        Dft<F2, true>::run(a);
        Dft<F2, true>::run(b);
        cp.st(k * F2, a[0], b[0]);
#pragma unroll
        for (int r = 1; r < F2; ++r) {
            const twd<float> w = ld_tw(tw + r * k);
            cp.st(k * F2 + r, mul_tw_conj(a[r], w), mul_tw_conj(b[r], w));
        }
    }
}
// inverse, stage 2: F1-point DFTs at stride F2 -> natural order, in place
template <int LY>
__device__ __forceinline__ void col_inv2(const ColPair& cp, int q) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int j = q; j < F2; j += 4) {
        cpx<float> a[F1], b[F1];
#pragma unroll
        for (int r = 0; r < F1; ++r) cp.ld(j + F2 * r, a[r], b[r]);
        Dft<F1, true>::run(a);
        Dft<F1, true>::run(b);
#pragma unroll
        for (int r = 0; r < F1; ++r) cp.st(j + F2 * r, a[r], b[r]);
    }
}

template <int NT, class F>
__device__ __forceinline__ void loop2n(int count, int nouter, F&& f) {
    int o = int(threadIdx.x) / count;
    int i = int(threadIdx.x) - o * count;
    const int dO = NT / count, dI = NT - dO * count;
    while (o < nouter) {
        f(o, i);
        i += dI;
        o += dO;
        if (i >= count) { i -= count; ++o; }
    }
}

// ---- pass A ------------------------------------------------------------------
// Work item (subdomain, field, z plane): the plane's rows are copied to shared
// memory at pitch reg_pitch(Lx/2+1); thread y transforms row y along x; then
// two threads per column transform along y and store the half spectrum.
__global__ void __launch_bounds__(kRegThreads, PSATD_MINB_REG) k_pass_a_reg(Args<float> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<float>* sm = reinterpret_cast<cpx<float>*>(smraw);
    __shared__ SubDesc d;
    __shared__ int64_t s_ticket[2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    unsigned parity = 0;
    Tickets<float> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<0>(a, it, &d);
        const int Lx = d.L[0], Ly = d.L[1], Lz = d.L[2], lxh = d.lxh;
        const int loc = int(it - d.itemA);
        const int f = loc / Lz, z = loc - (loc / Lz) * Lz;
        const int P = reg_pitch(lxh);
        const float* src = field_in(a, f) + d.field_off + int64_t(z) * Ly * Lx;
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) {
                fence_proxy_async();
                mbar_arrive_expect(&bar, unsigned(Ly * Lx * 4));
            }
            __syncwarp();
            for (int y = threadIdx.x; y < Ly; y += 32) bulk_g2s(sm + y * P, src + int64_t(y) * Lx, unsigned(Lx * 4), &bar);
        }
        if (!wait_bulk(&bar, parity, a.err, &s_ok)) return;
        parity ^= 1u;
        if (int(threadIdx.x) < Ly) {
            cpx<float>* row = sm + threadIdx.x * P;
            dispatch_x<0>(Lx, [&](auto lc) { row_fwd<decltype(lc)::value / 2>(row, a.tw + d.ax.tw, a.tw + d.tw_post); });
        }
        __syncthreads();
        // y: warp q takes quarter q of the DFTs of column pair (2 c2, 2 c2 + 1)
        const int c2 = threadIdx.x & 31, q = threadIdx.x >> 5;
        const ColPair cp{sm + 2 * c2, P, true, false};
        const bool act = 2 * c2 < lxh;
        if (act) dispatch_y<0>(Ly, [&](auto lc) { col_fwd1<decltype(lc)::value>(cp, q, a.tw + d.ay.tw); });
        __syncthreads();
        if (act) {
            cpx<float>* dst = a.spec + d.spec_off + int64_t(f * Lz + z) * d.q + 2 * c2;
            dispatch_y<0>(Ly, [&](auto lc) { col_fwd2<decltype(lc)::value>(cp, q, dst, lxh, 2 * c2 + 1 < lxh); });
        }
        __syncthreads();
    }
}

// ---- pass C ------------------------------------------------------------------
// Work item (subdomain, E/B component, valid z plane): the plane's half
// spectrum (contiguous in the spectra block) is copied to shared memory in
// one bulk copy (pitch Lx/2+1); two threads per column do the inverse y
// transform; thread t does the merge and inverse x transform of valid row
// ng + t; then every thread stores the valid cells to every box that holds
// them (own box and guard images, Fig. 3 step 3).
__global__ void __launch_bounds__(kRegThreads, PSATD_MINB_REG) k_pass_c_reg(Args<float> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<float>* sm = reinterpret_cast<cpx<float>*>(smraw);
    __shared__ SubDesc d;
    __shared__ Segment segs[kSegSmem];
    __shared__ int64_t s_ticket[2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    unsigned parity = 0;
    Tickets<float> tk(a, s_ticket);
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<2>(a, it, &d);
        const int Lx = d.L[0], Ly = d.L[1], Lz = d.L[2], lxh = d.lxh;
        const int nz = d.nv[2], ny = d.nv[1], ng = d.ng, ngz = d.ngz;
        const int loc = int(it - d.itemC);
        const int f = loc / nz, z = ngz + (loc - (loc / nz) * nz);
        const int P = lxh;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            const unsigned bytes = unsigned(d.q) * 8u;
            mbar_arrive_expect(&bar, bytes);
            bulk_g2s(sm, a.spec + d.spec_off + int64_t(f * Lz + z) * d.q, bytes, &bar);
        }
        const int nsg = min(d.seg_end - d.seg_begin, kSegSmem);
        {
            const int* gs = reinterpret_cast<const int*>(a.segs + d.seg_begin);
            int* ss = reinterpret_cast<int*>(segs);
            for (int i = threadIdx.x; i < nsg * int(sizeof(Segment) / 4); i += kRegThreads) ss[i] = __ldg(gs + i);
        }
        if (!wait_bulk(&bar, parity, a.err, &s_ok)) return;
        parity ^= 1u;
        const int c2 = threadIdx.x & 31, q = threadIdx.x >> 5;
        const ColPair cp{sm + 2 * c2, P, false, 2 * c2 + 1 >= lxh};
        const bool act = 2 * c2 < lxh;
        if (act) dispatch_y<0>(Ly, [&](auto lc) { col_inv1<decltype(lc)::value>(cp, q, a.tw + d.ay.tw); });
        __syncthreads();
        if (act) dispatch_y<0>(Ly, [&](auto lc) { col_inv2<decltype(lc)::value>(cp, q); });
        __syncthreads();
        if (int(threadIdx.x) < ny) {
            cpx<float>* row = sm + (ng + threadIdx.x) * P;
            dispatch_x<0>(Lx, [&](auto lc) { row_inv<decltype(lc)::value / 2>(row, a.tw + d.ax.tw, a.tw + d.tw_post); });
        }
        __syncthreads();
        // store the valid cells of this plane to every box that holds them
        float* out = a.eb[f];
        const float* rp = reinterpret_cast<const float*>(sm);
        const int rs = 2 * P;                             // real row stride
        for (int g = 0; g < d.seg_end - d.seg_begin; ++g) {
            const Segment& sg = g < kSegSmem ? segs[g] : a.segs[d.seg_begin + g];
            if (a.own_only && !sg.identity) continue;
            if (z < sg.z0 || z >= sg.z0 + sg.ez) continue;
            float* dst = out + sg.dst_off + (int64_t(z + sg.dz) * sg.dLy + sg.y0 + sg.dy) * sg.dLx + sg.x0 + sg.dx;
            const float* sp = rp + sg.y0 * rs + sg.x0;
            if (sg.vec4) {
                loop2n<kRegThreads>(sg.ex >> 2, sg.ey, [&](int yy, int x4) {
                    const cpx<float> u = *reinterpret_cast<const cpx<float>*>(sp + yy * rs + 4 * x4);
                    const cpx<float> w = *reinterpret_cast<const cpx<float>*>(sp + yy * rs + 4 * x4 + 2);
                    stcs4(dst + int64_t(yy) * sg.dLx + 4 * x4, cpx4<float>{u.x, u.y, w.x, w.y});
                });
            } else {
                loop2n<kRegThreads>(sg.ex, sg.ey, [&](int yy, int xx) { __stcs(dst + int64_t(yy) * sg.dLx + xx, sp[yy * rs + xx]); });
            }
        }
        __syncthreads();
    }
}

}  // namespace psatd
