// Register-resident DFTs of sizes 1..16 with compile-time twiddle constants.
//
// Dft<N, INV>::run(v) transforms N complex values in place, natural order in
// and out: forward X[k] = sum_n v[n] exp(-2 pi i n k / N) (INV = false) or
// the unnormalised inverse with exp(+2 pi i n k / N) (INV = true).
//
// Primes use the symmetric form X[k] = v0 + sum_j a_j cos(2 pi jk/P)
// +/- i sum_j b_j sin(2 pi jk/P) with a_j = v_j + v_{P-j}, b_j = v_j - v_{P-j};
// composite sizes use one Cooley-Tukey split N = A*B done entirely in
// registers.  The cos/sin constants are evaluated at compile time from their
// Taylor series after an exact quadrant reduction of the rational angle.
#pragma once
#include <stdint.h>
#include <type_traits>
#include <utility>

namespace psatd {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
    T x, y;
};

// Two FP32 lanes advanced by one packed instruction (FFMA2 / FMUL2 of the
// sm_100 family): the same operation on two independent data sets, e.g. two
// columns that share every constant and twiddle.  Additions are issued as
// fused multiply-adds with a unit factor, which round exactly like an
// addition.
struct __align__(8) P2 {
    float x, y;   // lane 0, lane 1
    P2() = default;
    __host__ __device__ constexpr P2(float a) : x(a), y(a) {}
    __host__ __device__ constexpr P2(float a, float b) : x(a), y(b) {}
};
__device__ __forceinline__ float2 f2of(P2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ P2 p2of(float2 a) { return P2(a.x, a.y); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ P2 fma_t(P2 a, P2 b, P2 c) { return p2of(__ffma2_rn(f2of(a), f2of(b), f2of(c))); }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return p2of(__fmul2_rn(f2of(a), f2of(b))); }
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return fma_t(a, P2(1.f), b); }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return fma_t(b, P2(-1.f), a); }
__device__ __forceinline__ P2 operator-(P2 a) { return a * P2(-1.f); }
__device__ __forceinline__ P2& operator+=(P2& a, P2 b) { a = a + b; return a; }

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T x, T y) { cpx<T> r; r.x = x; r.y = y; return r; }
template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>   // a * conj(b)
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T>
__device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T>   // i * a
__device__ __forceinline__ cpx<T> mul_i(cpx<T> a) { return mk(-a.y, a.x); }
template <typename T>
__device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }

// ---- compile-time trigonometry of rational angles ------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int n = 1; n < 22; ++n) { term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0)); sum += term; }
    return sum;
}
constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int n = 1; n < 22; ++n) { term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n)); sum += term; }
    return sum;
}
// 2 pi m / N = q pi/2 + phi with phi in [0, pi/2)
constexpr long quad_of(long m, long N) { return (4 * (((m % N) + N) % N)) / N; }
constexpr double phi_of(long m, long N) {
    return (kPi / 2) * double(4 * (((m % N) + N) % N) - quad_of(m, N) * N) / double(N);
}
constexpr double cos2pi(long m, long N) {
    return quad_of(m, N) == 0 ? taylor_cos(phi_of(m, N))
         : quad_of(m, N) == 1 ? -taylor_sin(phi_of(m, N))
         : quad_of(m, N) == 2 ? -taylor_cos(phi_of(m, N))
                              : taylor_sin(phi_of(m, N));
}
constexpr double sin2pi(long m, long N) {
    return quad_of(m, N) == 0 ? taylor_sin(phi_of(m, N))
         : quad_of(m, N) == 1 ? taylor_cos(phi_of(m, N))
         : quad_of(m, N) == 2 ? -taylor_sin(phi_of(m, N))
                              : -taylor_cos(phi_of(m, N));
}

// ---- compile-time loop ----------------------------------------------------
template <int I, int N, class F>
__device__ __forceinline__ void static_for_impl(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for_impl<I + 1, N>(f);
    }
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) { static_for_impl<0, N>(f); }

// FP32 constants are split into hi + lo (lo = the FP32 rounding of the
// remainder), so that a product with a constant carries no systematic
// quantisation error; in FP64 the lo part is dropped.  PSATD_DFT_HILO 0
// keeps only the FP32 rounding.
#ifndef PSATD_DFT_HILO
#define PSATD_DFT_HILO 1
#endif
template <typename T>
struct Split32 {
    static constexpr bool kOn = sizeof(T) == 4 && PSATD_DFT_HILO;
};
template <>
struct Split32<P2> {
    static constexpr bool kOn = PSATD_DFT_HILO;
};
template <typename T>
constexpr T hi_of(double v) { return T(v); }
template <typename T>
constexpr T lo_of(double v) { return T(v - double(T(v))); }
template <>
constexpr P2 hi_of<P2>(double v) { return P2(float(v)); }
template <>
constexpr P2 lo_of<P2>(double v) { return P2(float(v - double(float(v)))); }

template <typename T>
constexpr bool kPacked = std::is_same<T, P2>::value;

// v * (c + i s) with c, s given as (hi, lo) pairs; msh, msl = -sh, -sl are
// passed separately so that packed lanes need no negation instruction (the
// scalar forms leave the multiply-adds to the compiler)
template <typename T>
__device__ __forceinline__ cpx<T> cmul_const4(cpx<T> v, T ch, T cl, T sh, T sl, T msh, T msl) {
    if constexpr (kPacked<T>) {
        if constexpr (Split32<T>::kOn) {
            const T tr = fma_t(v.x, cl, v.y * msl);
            const T ti = fma_t(v.x, sl, v.y * cl);
            return mk(fma_t(v.x, ch, fma_t(v.y, msh, tr)), fma_t(v.x, sh, fma_t(v.y, ch, ti)));
        } else {
            return mk(fma_t(v.x, ch, v.y * msh), fma_t(v.x, sh, v.y * ch));
        }
    } else if constexpr (Split32<T>::kOn) {
        const T tr = fmaf(v.x, cl, -v.y * sl);
        const T ti = fmaf(v.x, sl, v.y * cl);
        return mk(fmaf(v.x, ch, fmaf(-v.y, sh, tr)), fmaf(v.x, sh, fmaf(v.y, ch, ti)));
    } else {
        return mk(v.x * ch - v.y * sh, v.x * sh + v.y * ch);
    }
}
template <typename T>
__device__ __forceinline__ cpx<T> cmul_const(cpx<T> v, T ch, T cl, T sh, T sl) {
    return cmul_const4(v, ch, cl, sh, sl, T(-sh), T(-sl));
}

// multiply by exp(sgn 2 pi i M / N), sgn = -1 forward, +1 inverse
template <int M, int N, bool INV, typename T>
__device__ __forceinline__ cpx<T> twiddle(cpx<T> v) {
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) {
        return v;
    } else if constexpr (2 * m == N) {
        return mk(-v.x, -v.y);
    } else if constexpr (4 * m == N) {          // exp(sgn i pi/2) = sgn i
        return INV ? mk(-v.y, v.x) : mk(v.y, -v.x);
    } else if constexpr (4 * m == 3 * N) {      // exp(sgn i 3pi/2) = -sgn i
        return INV ? mk(v.y, -v.x) : mk(-v.y, v.x);
    } else {
        constexpr double c = cos2pi(m, N);
        constexpr double s = INV ? sin2pi(m, N) : -sin2pi(m, N);
        return cmul_const4(v, hi_of<T>(c), lo_of<T>(c), hi_of<T>(s), lo_of<T>(s), hi_of<T>(-s), lo_of<T>(-s));
    }
}

template <int N, bool INV>
struct Dft;

template <bool INV>
struct Dft<1, INV> {
    template <typename T>
    __device__ __forceinline__ static void run(cpx<T>*) {}
};

template <bool INV>
struct Dft<2, INV> {
    template <typename T>
    __device__ __forceinline__ static void run(cpx<T>* v) {
        cpx<T> a = v[0];
        v[0] = a + v[1];
        v[1] = a - v[1];
    }
};

template <bool INV>
struct Dft<4, INV> {
    template <typename T>
    __device__ __forceinline__ static void run(cpx<T>* v) {
        cpx<T> a = v[0] + v[2], b = v[0] - v[2], c = v[1] + v[3], d = v[1] - v[3];
        v[0] = a + c;
        v[2] = a - c;
        if constexpr (kPacked<T>) {
            // b -/+ i d, written out so that no component is negated on its own
            const cpx<T> bm = mk(b.x + d.y, b.y - d.x), bp = mk(b.x - d.y, b.y + d.x);
            if (INV) { v[1] = bp; v[3] = bm; }
            else     { v[1] = bm; v[3] = bp; }
        } else {
            cpx<T> id = mul_i(d);
            if (INV) { v[1] = b + id; v[3] = b - id; }
            else     { v[1] = b - id; v[3] = b + id; }
        }
    }
};

template <int P, bool INV>
struct DftPrime {
    template <typename T>
    __device__ __forceinline__ static void run(cpx<T>* v) {
        constexpr int H = (P - 1) / 2;
        cpx<T> a[H], b[H];
        static_for<H>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            a[j] = v[j + 1] + v[P - 1 - j];
            b[j] = v[j + 1] - v[P - 1 - j];
        });
        const cpx<T> x0 = v[0];
        cpx<T> s0 = x0 + a[0];
        static_for<H - 1>([&](auto jc) { s0 = s0 + a[decltype(jc)::value + 1]; });
        v[0] = s0;
        static_for<H>([&](auto kc) {
            constexpr int k = decltype(kc)::value + 1;
            cpx<T> R = x0, Q = mk(T(0), T(0));
            cpx<T> Rl = mk(T(0), T(0)), Ql = mk(T(0), T(0));
            static_for<H>([&](auto jc) {
                constexpr int j = decltype(jc)::value + 1;
                constexpr double c = cos2pi((long)j * k, P);
                constexpr double s = sin2pi((long)j * k, P);
                constexpr T ch = hi_of<T>(c), sh = hi_of<T>(s);
                if constexpr (kPacked<T>) {     // packed lanes: explicit multiply-adds
                    R.x = fma_t(a[j - 1].x, ch, R.x); R.y = fma_t(a[j - 1].y, ch, R.y);
                    Q.x = fma_t(b[j - 1].x, sh, Q.x); Q.y = fma_t(b[j - 1].y, sh, Q.y);
                } else {
                    R.x += a[j - 1].x * ch; R.y += a[j - 1].y * ch;
                    Q.x += b[j - 1].x * sh; Q.y += b[j - 1].y * sh;
                }
                if constexpr (Split32<T>::kOn) {
                    constexpr T cl = lo_of<T>(c), sl = lo_of<T>(s);
                    if constexpr (kPacked<T>) {
                        Rl.x = fma_t(a[j - 1].x, cl, Rl.x); Rl.y = fma_t(a[j - 1].y, cl, Rl.y);
                        Ql.x = fma_t(b[j - 1].x, sl, Ql.x); Ql.y = fma_t(b[j - 1].y, sl, Ql.y);
                    } else {
                        Rl.x += a[j - 1].x * cl; Rl.y += a[j - 1].y * cl;
                        Ql.x += b[j - 1].x * sl; Ql.y += b[j - 1].y * sl;
                    }
                }
            });
            if constexpr (Split32<T>::kOn) { R = R + Rl; Q = Q + Ql; }
            // X_k = R + sgn i Q, X_{P-k} = R - sgn i Q
            if (INV) { v[k] = mk(R.x - Q.y, R.y + Q.x); v[P - k] = mk(R.x + Q.y, R.y - Q.x); }
            else     { v[k] = mk(R.x + Q.y, R.y - Q.x); v[P - k] = mk(R.x - Q.y, R.y + Q.x); }
        });
    }
};

template <int N, int A, bool INV>
struct DftSplit {
    template <typename T>
    __device__ __forceinline__ static void run(cpx<T>* v) {
        constexpr int B = N / A;
        cpx<T> y[N];
        // A-point DFTs over n1 of v[B n1 + n2], then twiddle w_N^{n2 k1}
        static_for<B>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            cpx<T> t[A];
            static_for<A>([&](auto n1c) { t[decltype(n1c)::value] = v[B * decltype(n1c)::value + n2]; });
            Dft<A, INV>::run(t);
            static_for<A>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                y[n2 * A + k1] = twiddle<n2 * k1, N, INV>(t[k1]);
            });
        });
        // B-point DFTs over n2, output X[k1 + A k2]
        static_for<A>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            cpx<T> t[B];
            static_for<B>([&](auto n2c) { t[decltype(n2c)::value] = y[decltype(n2c)::value * A + k1]; });
            Dft<B, INV>::run(t);
            static_for<B>([&](auto k2c) { v[k1 + A * decltype(k2c)::value] = t[decltype(k2c)::value]; });
        });
    }
};

template <bool INV> struct Dft<3, INV> : DftPrime<3, INV> {};
template <bool INV> struct Dft<5, INV> : DftPrime<5, INV> {};
template <bool INV> struct Dft<7, INV> : DftPrime<7, INV> {};
template <bool INV> struct Dft<11, INV> : DftPrime<11, INV> {};
template <bool INV> struct Dft<13, INV> : DftPrime<13, INV> {};
template <bool INV> struct Dft<6, INV> : DftSplit<6, 2, INV> {};
template <bool INV> struct Dft<8, INV> : DftSplit<8, 2, INV> {};
template <bool INV> struct Dft<9, INV> : DftSplit<9, 3, INV> {};
template <bool INV> struct Dft<10, INV> : DftSplit<10, 2, INV> {};
template <bool INV> struct Dft<12, INV> : DftSplit<12, 4, INV> {};
template <bool INV> struct Dft<14, INV> : DftSplit<14, 2, INV> {};
template <bool INV> struct Dft<15, INV> : DftSplit<15, 3, INV> {};
template <bool INV> struct Dft<16, INV> : DftSplit<16, 4, INV> {};

// Call f(integral_constant<int, n>) for a runtime n in 1..16.
template <class F>
__device__ __forceinline__ void with_size(int n, F&& f) {
    switch (n) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 5: f(std::integral_constant<int, 5>{}); break;
        case 6: f(std::integral_constant<int, 6>{}); break;
        case 7: f(std::integral_constant<int, 7>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 9: f(std::integral_constant<int, 9>{}); break;
        case 10: f(std::integral_constant<int, 10>{}); break;
        case 11: f(std::integral_constant<int, 11>{}); break;
        case 12: f(std::integral_constant<int, 12>{}); break;
        case 13: f(std::integral_constant<int, 13>{}); break;
        case 14: f(std::integral_constant<int, 14>{}); break;
        case 15: f(std::integral_constant<int, 15>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        default: break;
    }
}

}  // namespace psatd
