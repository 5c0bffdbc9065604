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
//   y (columns):  a thread works on a pair of half-spectrum columns; the
//                 four warps (eight half-warps when there are at most 16
//                 pairs) take every fourth (eighth) f1-point and f2-point
//                 DFT of the column pairs.
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
#ifndef PSATD_MINB_REG_B
#define PSATD_MINB_REG_B 4
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

// ---- y: column pairs, four or eight threads per pair ------------------------
// Thread (pair c2, group q of nq) works on two columns: 2 c2 and 2 c2 + 1 in
// passes A and B, c2 and c2 + ceil(lxh/2) in pass C (the second may be past
// the half spectrum: it is then padding, computed on and never stored, or,
// with `tail` set, neither read nor written); group q takes every nq-th
// stage-1 (stride) DFT and every nq-th stage-2 (block) DFT.
// tw = exp(-2 pi i m/L), m = 0..L-1.

// element pair (columns c, c + off2) of row y: one 16-byte access for
// adjacent columns at an even pitch, two 8-byte accesses otherwise (the second
// skipped for a tail column)
// Lanes of the y phase: ceil(lxh/2) column pairs, one per lane, in four
// groups of 32 lanes (the four warps); with at most 16 pairs in eight groups
// of 16 (half-warps), so that fewer lanes idle on narrow planes.  Group q
// takes every nq-th f1- and f2-point DFT.
static_assert(kRegThreads == 128, "the y phase maps four warps or eight half-warps");
__device__ __forceinline__ int lane_groups(int lxh) { return (lxh + 1) >> 1 <= 16 ? 8 : 4; }
__device__ __forceinline__ int lane_col(int lxh) {
    return (lxh + 1) >> 1 <= 16 ? int(threadIdx.x & 15) : int(threadIdx.x & 31);
}
__device__ __forceinline__ int lane_group(int lxh) {
    return (lxh + 1) >> 1 <= 16 ? int(threadIdx.x >> 4) : int(threadIdx.x >> 5);
}

struct ColPair {
    cpx<float>* base;   // element (0, c)
    int P;              // row pitch (complex)
    bool v16, tail;
    int off2;           // the second column: c + off2 (1 with v16)
    __device__ __forceinline__ void ld(int y, cpx<float>& a, cpx<float>& b) const {
        cpx<float>* q = base + y * P;
        if (v16) {
            const float4 v = lds4(q);
            a = mk(v.x, v.y);
            b = mk(v.z, v.w);
        } else {
            a = q[0];
            b = tail ? mk(0.f, 0.f) : q[off2];
        }
    }
    __device__ __forceinline__ void st(int y, cpx<float> a, cpx<float> b) const {
        cpx<float>* q = base + y * P;
        if (v16) {
            sts4(q, a, b);
        } else {
            q[0] = a;
            if (!tail) q[off2] = b;
        }
    }
};

// forward, stage 1: F1-point DFTs at stride F2, twiddle w^{j r}, in place
template <int LY>
__device__ __forceinline__ void col_fwd1(const ColPair& cp, int q, int nq, const twd<float>* __restrict__ tw) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int j = q; j < F2; j += nq) {
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
__device__ __forceinline__ void col_fwd2(const ColPair& cp, int q, int nq, cpx<float>* dst, int ld, bool second) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int k = q; k < F1; k += nq) {
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
__device__ __forceinline__ void col_inv1(const ColPair& cp, int q, int nq, const twd<float>* __restrict__ tw) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int k = q; k < F1; k += nq) {
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
__device__ __forceinline__ void col_inv2(const ColPair& cp, int q, int nq) {
    constexpr int F1 = split_first(LY), F2 = LY / F1;
#pragma unroll 1
    for (int j = q; j < F2; j += nq) {
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
        // y: lane group q takes every nq-th DFT of column pair (2 c2, 2 c2 + 1)
        const int c2 = lane_col(lxh), q = lane_group(lxh), nq = lane_groups(lxh);
        const ColPair cp{sm + 2 * c2, P, true, false, 1};
        const bool act = 2 * c2 < lxh;
        if (act) dispatch_y<0>(Ly, [&](auto lc) { col_fwd1<decltype(lc)::value>(cp, q, nq, a.tw + d.ay.tw); });
        __syncthreads();
        if (act) {
            cpx<float>* dst = a.spec + d.spec_off + int64_t(f * Lz + z) * d.q + 2 * c2;
            dispatch_y<0>(Ly, [&](auto lc) { col_fwd2<decltype(lc)::value>(cp, q, nq, dst, lxh, 2 * c2 + 1 < lxh); });
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
        // columns c2 and c2 + np (np = ceil(lxh/2)): consecutive lanes touch
        // consecutive 8-byte elements, free of bank conflicts at the odd pitch
        const int c2 = lane_col(lxh), q = lane_group(lxh), nq = lane_groups(lxh), np = (lxh + 1) >> 1;
        const ColPair cp{sm + c2, P, false, c2 + np >= lxh, np};
        const bool act = c2 < np;
        if (act) dispatch_y<0>(Ly, [&](auto lc) { col_inv1<decltype(lc)::value>(cp, q, nq, a.tw + d.ay.tw); });
        __syncthreads();
        if (act) dispatch_y<0>(Ly, [&](auto lc) { col_inv2<decltype(lc)::value>(cp, q, nq); });
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
            if (!sg.vec4) {
                loop2n<kRegThreads>(sg.ex, sg.ey, [&](int yy, int xx) { __stcs(dst + int64_t(yy) * sg.dLx + xx, sp[yy * rs + xx]); });
            } else if (!store_rows_pow2<kRegThreads>(dst, sg.dLx, sp, rs, sg.ex >> 2, sg.ey)) {
                loop2n<kRegThreads>(sg.ex >> 2, sg.ey, [&](int yy, int x4) {
                    const cpx<float> u = *reinterpret_cast<const cpx<float>*>(sp + yy * rs + 4 * x4);
                    const cpx<float> w = *reinterpret_cast<const cpx<float>*>(sp + yy * rs + 4 * x4 + 2);
                    stcs4(dst + int64_t(yy) * sg.dLx + 4 * x4, cpx4<float>{u.x, u.y, w.x, w.y});
                });
            }
        }
        __syncthreads();
    }
}

// ---- packed column pairs (P2 lanes: the two columns) ---------------------------
// A pair of complex numbers (a, b) as C2: x = (re a, re b), y = (im a, im b).
// In shared memory a pair is 16 bytes, either interleaved per number
// ("aos": re a, im a, re b, im b, the layout of the spectra) or by part
// ("planar": re a, re b, im a, im b, the layout between the packed stages).
using C2 = cpx<P2>;
__device__ __forceinline__ C2 ld_aos(const cpx<float>* q) {
    const float4 v = lds4(q);
    return mk(P2(v.x, v.z), P2(v.y, v.w));
}
__device__ __forceinline__ C2 ld_pl(const cpx<float>* q) {
    const float4 v = lds4(q);
    return mk(P2(v.x, v.y), P2(v.z, v.w));
}
__device__ __forceinline__ void st_pl(cpx<float>* q, C2 c) {
    *reinterpret_cast<float4*>(q) = make_float4(c.x.x, c.x.y, c.y.x, c.y.y);
}
__device__ __forceinline__ void st_aos(cpx<float>* q, C2 c) {
    *reinterpret_cast<float4*>(q) = make_float4(c.x.x, c.y.x, c.x.y, c.y.y);
}
// v * w and v * conj(w) for one twiddle w shared by both lanes
__device__ __forceinline__ C2 mul_tw2(C2 v, const twd<float>& w) {
    const P2 c(w.hi.x), s(w.hi.y), ms(-w.hi.y);
    return mk(fma_t(v.x, c, v.y * ms), fma_t(v.x, s, v.y * c));
}
__device__ __forceinline__ C2 mul_tw2_conj(C2 v, const twd<float>& w) {
    const P2 c(w.hi.x), s(w.hi.y), ms(-w.hi.y);
    return mk(fma_t(v.x, c, v.y * s), fma_t(v.y, c, v.x * ms));
}

// z transforms of a column pair of the pass-B chunk (pair base `col`, row
// pitch P complex), quarter q of the DFTs as in col_fwd1 / col_fwd2 /
// col_inv1 / col_inv2.  Forward stage 1 reads the interleaved spectra and
// writes planar pairs; inverse stage 2 reads planar pairs and writes the
// interleaved spectra back.
template <int LZ>
__device__ __forceinline__ void zp_fwd1(cpx<float>* col, int P, int q, const twd<float>* __restrict__ tw) {
    constexpr int F1 = split_first(LZ), F2 = LZ / F1;
#pragma unroll 1
    for (int j = q; j < F2; j += 4) {
        C2 v[F1];
#pragma unroll
        for (int r = 0; r < F1; ++r) v[r] = ld_aos(col + (j + F2 * r) * P);
        Dft<F1, false>::run(v);
        st_pl(col + j * P, v[0]);
#pragma unroll
        for (int r = 1; r < F1; ++r) st_pl(col + (j + F2 * r) * P, mul_tw2(v[r], ld_tw(tw + j * r)));
    }
}
template <int LZ>
__device__ __forceinline__ void zp_fwd2(cpx<float>* col, int P, int q) {
    constexpr int F1 = split_first(LZ), F2 = LZ / F1;
#pragma unroll 1
    for (int k = q; k < F1; k += 4) {
        C2 v[F2];
#pragma unroll
        for (int r = 0; r < F2; ++r) v[r] = ld_pl(col + (k * F2 + r) * P);
        Dft<F2, false>::run(v);
#pragma unroll
        for (int r = 0; r < F2; ++r) st_pl(col + (k * F2 + r) * P, v[r]);
    }
}
template <int LZ>
__device__ __forceinline__ void zp_inv1(cpx<float>* col, int P, int q, const twd<float>* __restrict__ tw) {
    constexpr int F1 = split_first(LZ), F2 = LZ / F1;
#pragma unroll 1
    for (int k = q; k < F1; k += 4) {
        C2 v[F2];
#pragma unroll
        for (int r = 0; r < F2; ++r) v[r] = ld_pl(col + (k * F2 + r) * P);
        Dft<F2, true>::run(v);
        st_pl(col + k * F2 * P, v[0]);
#pragma unroll
        for (int r = 1; r < F2; ++r) st_pl(col + (k * F2 + r) * P, mul_tw2_conj(v[r], ld_tw(tw + r * k)));
    }
}
template <int LZ>
__device__ __forceinline__ void zp_inv2(cpx<float>* col, int P, int q) {
    constexpr int F1 = split_first(LZ), F2 = LZ / F1;
#pragma unroll 1
    for (int j = q; j < F2; j += 4) {
        C2 v[F1];
#pragma unroll
        for (int r = 0; r < F1; ++r) v[r] = ld_pl(col + (j + F2 * r) * P);
        Dft<F1, true>::run(v);
#pragma unroll
        for (int r = 0; r < F1; ++r) st_aos(col + (j + F2 * r) * P, v[r]);
    }
}

// Eq. 1a/1b on a pair of modes (positions q, q + 1 of a plane, both at z
// position zp), packed: p points at the E_x pair in planar layout, the other
// fields at multiples of fs.  Same arithmetic as eq1_mode, lane by lane.
__device__ __forceinline__ void eq1_pair(const Args<float>& a, const SubDesc& d, cpx<float>* p, int fs, int q, int yp0,
                                         int xp0, int yp1, int xp1, int zp, int lxh, int Ly, int64_t NM, int64_t Q,
                                         P2 Nfull, P2& g_res, P2& g_rho) {
    const int nf = a.nf;
    const float* __restrict__ tk = a.tab + d.tab_k;
    const float* __restrict__ tb = a.tab + d.tab_coef + int64_t(zp) * Q + q;
    auto ld2 = [&](const float* t) { const float2 v = __ldg(reinterpret_cast<const float2*>(t)); return P2(v.x, v.y); };
    const P2 C = ld2(tb), S = ld2(tb + NM), Sk = ld2(tb + 2 * NM), omC = ld2(tb + 3 * NM);
    const P2 omCk = ld2(tb + 4 * NM), Dk = ld2(tb + 5 * NM), inv = ld2(tb + 6 * NM);
    const P2 kx(__ldg(tk + xp0), __ldg(tk + xp1)), ky(__ldg(tk + lxh + yp0), __ldg(tk + lxh + yp1));
    const P2 kz(__ldg(tk + lxh + Ly + zp));
    const P2 hx = kx * inv, hy = ky * inv, hz = kz * inv;
    const P2 mhx = -hx, mhy = -hy, mhz = -hz, mS = -S, mSk = -Sk, momCk = -omCk;
    C2 E0 = ld_pl(p), E1 = ld_pl(p + fs), E2 = ld_pl(p + 2 * fs);
    C2 B0 = ld_pl(p + 3 * fs), B1 = ld_pl(p + 4 * fs), B2 = ld_pl(p + 5 * fs);
    C2 J0 = ld_pl(p + 6 * fs), J1 = ld_pl(p + 7 * fs), J2 = ld_pl(p + 8 * fs);
    // complex pair times complex pair, and times its conjugate
    auto cm = [](C2 u, C2 w) { return mk(fma_t(u.x, w.x, u.y * -w.y), fma_t(u.x, w.y, u.y * w.x)); };
    auto cmc = [](C2 u, C2 w) { return mk(fma_t(u.x, w.x, u.y * w.y), fma_t(u.y, w.x, u.x * -w.y)); };
    C2 px, py, pz;
    if (a.staggered) {
        const cpx<float>* ph = a.tabc + d.tab_ph;
        const cpx<float> x0 = ldg_c(ph + xp0), x1 = ldg_c(ph + xp1), y0 = ldg_c(ph + lxh + yp0), y1 = ldg_c(ph + lxh + yp1);
        const cpx<float> z0 = ldg_c(ph + lxh + Ly + zp);
        px = mk(P2(x0.x, x1.x), P2(x0.y, x1.y));
        py = mk(P2(y0.x, y1.x), P2(y0.y, y1.y));
        pz = mk(P2(z0.x), P2(z0.y));
        const C2 pyz = cm(py, pz), pxz = cm(px, pz), pxy = cm(px, py);
        E0 = cm(E0, px); E1 = cm(E1, py); E2 = cm(E2, pz);
        J0 = cm(J0, px); J1 = cm(J1, py); J2 = cm(J2, pz);
        B0 = cm(B0, pyz); B1 = cm(B1, pxz); B2 = cm(B2, pxy);
    }
    // khat x F (component by component: u * h - w * h')
    auto cr = [](C2 u, P2 hu, C2 w, P2 mhw) { return mk(fma_t(u.x, hu, w.x * mhw), fma_t(u.y, hu, w.y * mhw)); };
    const C2 hB0 = cr(B2, hy, B1, mhz), hB1 = cr(B0, hz, B2, mhx), hB2 = cr(B1, hx, B0, mhy);
    const C2 hE0 = cr(E2, hy, E1, mhz), hE1 = cr(E0, hz, E2, mhx), hE2 = cr(E1, hx, E0, mhy);
    const C2 hJ0 = cr(J2, hy, J1, mhz), hJ1 = cr(J0, hz, J2, mhx), hJ2 = cr(J1, hx, J0, mhy);
    auto dot = [&](C2 u0, C2 u1, C2 u2) {
        return mk(fma_t(u0.x, hx, fma_t(u1.x, hy, u2.x * hz)), fma_t(u0.y, hx, fma_t(u1.y, hy, u2.y * hz)));
    };
    const C2 dE = dot(E0, E1, E2), dJ = dot(J0, J1, J2);
    // (1-C) khat.E + (S/k - dt) khat.J
    const C2 lo = mk(fma_t(dE.x, omC, dJ.x * Dk), fma_t(dE.y, omC, dJ.y * Dk));
    // Eq. 1a: E' = C E + i S khat x B - S/k J + khat lo
    auto eq_e = [&](C2 e, C2 hb, C2 j, P2 h) {
        return mk(fma_t(C, e.x, fma_t(mS, hb.y, fma_t(mSk, j.x, h * lo.x))),
                  fma_t(C, e.y, fma_t(S, hb.x, fma_t(mSk, j.y, h * lo.y))));
    };
    // Eq. 1b: B' = C B - i S khat x E + i (1-C)/k khat x J
    auto eq_b = [&](C2 b, C2 he, C2 hj) {
        return mk(fma_t(C, b.x, fma_t(S, he.y, momCk * hj.y)), fma_t(C, b.y, fma_t(mS, he.x, omCk * hj.x)));
    };
    C2 F0 = eq_e(E0, hB0, J0, hx), F1 = eq_e(E1, hB1, J1, hy), F2 = eq_e(E2, hB2, J2, hz);
    C2 G0 = eq_b(B0, hE0, hJ0), G1 = eq_b(B1, hE1, hJ1), G2 = eq_b(B2, hE2, hJ2);
    if (nf > 9) {
        // |i[k].E' N - rho|^2 = (N sy + rho_x)^2 + (rho_y - N sx)^2 with
        // s = [k].E'; weighted by the half-spectrum multiplicity
        const C2 rho = ld_pl(p + 9 * fs);
        const P2 sx = fma_t(kx, F0.x, fma_t(ky, F1.x, kz * F2.x)), sy = fma_t(kx, F0.y, fma_t(ky, F1.y, kz * F2.y));
        const P2 rx = fma_t(sy, Nfull, rho.x), ry = fma_t(sx, -Nfull, rho.y);
        const P2 wgt(xp0 == 0 || xp0 == lxh - 1 ? 1.f : 2.f, xp1 == 0 || xp1 == lxh - 1 ? 1.f : 2.f);
        g_res = fma_t(wgt, fma_t(rx, rx, ry * ry), g_res);
        g_rho = fma_t(wgt, fma_t(rho.x, rho.x, rho.y * rho.y), g_rho);
    }
    if (a.staggered) {
        const C2 pyz = cm(py, pz), pxz = cm(px, pz), pxy = cm(px, py);
        F0 = cmc(F0, px); F1 = cmc(F1, py); F2 = cmc(F2, pz);
        G0 = cmc(G0, pyz); G1 = cmc(G1, pxz); G2 = cmc(G2, pxy);
    }
    st_pl(p, F0); st_pl(p + fs, F1); st_pl(p + 2 * fs, F2);
    st_pl(p + 3 * fs, G0); st_pl(p + 4 * fs, G1); st_pl(p + 5 * fs, G2);
}

// ---- pass B -------------------------------------------------------------------
// Work item (subdomain, kRegM consecutive (ky, kx) modes, all z): the z
// pencils of every field are copied to shared memory ([field][z][mode]);
// warp q takes every fourth DFT of each z transform of one mode pair (lane:
// field and mode pair); Eq. 1 per (z, mode pair); the inverse z transforms
// of E and B the same way; the valid z planes are stored.  The two modes of
// a pair share every twiddle and every step, so all arithmetic runs on
// packed FP32 lanes (one instruction for both modes).
template <int NT>
__device__ __forceinline__ float block_sum_n(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) s += red[i];
    }
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kRegThreads, PSATD_MINB_REG_B) k_pass_b_reg(Args<float> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<float>* sm = reinterpret_cast<cpx<float>*>(smraw);
    __shared__ SubDesc d;
    __shared__ float red[2][kRegThreads / 32];
    __shared__ int64_t s_ticket[2];
    Tickets<float> tk(a, s_ticket);
    constexpr int M = kRegM, MP = kRegM / 2;
    for (int64_t it = tk.current(); it >= 0; tk.advance(), it = tk.current()) {
        tk.prefetch();
        decode_item<1>(a, it, &d);
        const int Lx = d.L[0], Ly = d.L[1], Lz = d.L[2], Q = d.q, lxh = d.lxh;
        const int q0 = int(it - d.itemB) * M;
        const int mc = min(M, Q - q0);
        const int nf = a.nf, fs = d.fsB;
        cpx<float>* spec = a.spec + d.spec_off;
        // pairs of modes (16-byte copies: Q, q0 and M are even), zero-filled
        // past the ragged end of the plane: thread (column c, phase r) copies
        // rows z = r, r + 4, ... of mode-pair column c = (field, pair)
        {
            const int c = threadIdx.x >> 2, r = threadIdx.x & 3;
            if (c < nf * MP) {
                const int f = c / MP, m2 = c - f * MP;
                const int nb = min(max(mc - 2 * m2, 0), 2) * int(sizeof(cpx<float>));
                const cpx<float>* src = spec + int64_t(f) * Lz * Q + q0 + (nb ? 2 * m2 : 0) + int64_t(r) * Q;
                cpx<float>* dst = sm + f * fs + 2 * m2 + r * M;
                const int64_t step = 4 * int64_t(Q);
#pragma unroll 4
                for (int z = r; z < Lz; z += 4, src += step, dst += 4 * M) cp_async16(dst, src, nb);
            }
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int lf = lane / MP, lp = lane - lf * MP;
        cpx<float>* col = sm + lf * fs + 2 * lp;          // this lane's mode pair of field lf
        const twd<float>* twz = a.tw + d.az.tw;
        if (lf < nf) dispatch_y<0>(Lz, [&](auto lc) { zp_fwd1<decltype(lc)::value>(col, M, q, twz); });
        __syncthreads();
        if (lf < nf) dispatch_y<0>(Lz, [&](auto lc) { zp_fwd2<decltype(lc)::value>(col, M, q); });
        __syncthreads();
        const int64_t NM = int64_t(Lz) * Q;
        const P2 Nfull(float(double(Lx) * double(Ly) * double(Lz)));
        P2 g_res(0.f), g_rho(0.f);
        // (ky, kx) positions of the chunk's modes: one division per item
        const int yp0 = q0 / lxh, xp0 = q0 - yp0 * lxh;
        loop2n<kRegThreads>(MP, Lz, [&](int zp, int m2) {
            const int m = 2 * m2;
            if (m >= mc) return;           // mc is even: both modes of the pair are present
            int xa = xp0 + m, ya = yp0;
            if (xa >= lxh) { xa -= lxh; ++ya; }          // M <= lxh: at most one wrap
            int xb = xa + 1, yb = ya;
            if (xb >= lxh) { xb -= lxh; ++yb; }
            eq1_pair(a, d, sm + zp * M + m, fs, q0 + m, ya, xa, yb, xb, zp, lxh, Ly, NM, int64_t(Q), Nfull, g_res,
                     g_rho);
        });
        __syncthreads();
        if (lf < 6) dispatch_y<0>(Lz, [&](auto lc) { zp_inv1<decltype(lc)::value>(col, M, q, twz); });
        __syncthreads();
        if (lf < 6) dispatch_y<0>(Lz, [&](auto lc) { zp_inv2<decltype(lc)::value>(col, M, q); });
        __syncthreads();
        // valid z planes of E and B, mode pairs as 16-byte stores: thread
        // (column c, phase r) stores rows ngz + r, ngz + r + 4, ...
        {
            const int ng = d.ngz, nz = d.nv[2];
            const int c = threadIdx.x >> 2, r = threadIdx.x & 3;
            if (c < 6 * MP) {
                const int f = c / MP, m2 = c - f * MP;
                if (2 * m2 < mc) {
                    cpx<float>* dst = spec + int64_t(f) * Lz * Q + int64_t(ng + r) * Q + q0 + 2 * m2;
                    const cpx<float>* src = sm + f * fs + (ng + r) * M + 2 * m2;
                    const int64_t step = 4 * int64_t(Q);
#pragma unroll 4
                    for (int z = r; z < nz; z += 4, dst += step, src += 4 * M)
                        __stcs(reinterpret_cast<float4*>(dst), lds4(src));
                }
            }
        }
        if (nf > 9) {
            const double s1 = double(block_sum_n<kRegThreads>(g_res.x + g_res.y, red[0]));
            const double s2 = double(block_sum_n<kRegThreads>(g_rho.x + g_rho.y, red[1]));
            if (threadIdx.x == 0) {
                a.gauss_part[2 * it] = s1;
                a.gauss_part[2 * it + 1] = s2;
            }
        }
        __syncthreads();
    }
}

}  // namespace psatd
