// Host side of libpsatd.so: plan validation, decomposition bookkeeping, the
// FP64 construction of the Eq. 1 tables (Sec. 3.1 of arXiv:1707.08500) and
// the C ABI declared in include/psatd.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "psatd.h"
#include "psatd_internal.h"
#include "psatd_io.h"

namespace psatd {
cudaError_t launch_stage_f32(int stage, const LaunchCommon& c, int64_t i0, int64_t n, int smem, cudaStream_t s);
cudaError_t launch_stage_f64(int stage, const LaunchCommon& c, int64_t i0, int64_t n, int smem, cudaStream_t s);
cudaError_t launch_gauss_reduce(const void* subs, int nsub, const double* part, double* out, cudaStream_t st);
cudaError_t launch_stage_reg(int stage, const LaunchCommon& c, int64_t i0, int64_t n, int smem, cudaStream_t s);
}  // namespace psatd

using namespace psatd;
using cd = std::complex<double>;

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// exp(-2 pi i m / n) with an exact octant reduction of the rational angle
cd unit_root(long m, long n) {
    long r = ((m % n) + n) % n;
    // angle = 2 pi r / n in [0, 2 pi); reduce to [0, pi/4] by symmetry
    long num = 8 * r;            // angle = (pi/4) * num / n
    long oct = num / n;
    long rem = num - oct * n;    // angle = (pi/4)(oct + rem/n)
    double phi = (kPi / 4) * double(rem) / double(n);
    double c, s;
    // angle = oct*pi/4 + phi; evaluate with the reflection that keeps the
    // argument of sin/cos in [0, pi/4]
    switch (oct) {
        case 0: c = std::cos(phi); s = std::sin(phi); break;
        case 1: { double t = kPi / 4 - phi; c = std::sin(t); s = std::cos(t); break; }
        case 2: c = -std::sin(phi); s = std::cos(phi); break;
        case 3: { double t = kPi / 4 - phi; c = -std::cos(t); s = std::sin(t); break; }
        case 4: c = -std::cos(phi); s = -std::sin(phi); break;
        case 5: { double t = kPi / 4 - phi; c = -std::sin(t); s = -std::cos(t); break; }
        case 6: c = std::sin(phi); s = -std::cos(phi); break;
        default: { double t = kPi / 4 - phi; c = std::cos(t); s = -std::sin(t); break; }
    }
    return cd(c, -s);
}

// centred nodal weights w_j of f' ~ sum_j w_j (f_{+j} - f_{-j})/du (order p)
std::vector<double> weights_nodal(int p) {
    int m = p / 2;
    std::vector<double> w(m);
    w[0] = double(m) / (m + 1.0);
    for (int j = 1; j < m; ++j) w[j] = -w[j - 1] * j * (m - j) / ((j + 1.0) * (m + j + 1.0));
    return w;
}

// staggered weights c_j of f' ~ sum_j c_j (f_{+(j-1/2)} - f_{-(j-1/2)})/du
std::vector<double> weights_staggered(int p) {
    int m = p / 2;
    double lg = 0;
    for (int i = 1; i <= m; ++i) lg += std::log(2.0 * i - 1.0);
    double lc1 = 2 * lg - std::lgamma(double(m)) - std::lgamma(double(m) + 1) - (m - 1) * std::log(4.0);
    std::vector<double> c(m);
    c[0] = std::exp(lc1);
    for (int j = 1; j < m; ++j) c[j] = -c[j - 1] * double(2 * j - 1) * (2 * j - 1) * (m - j) / (double(2 * j + 1) * (2 * j + 1) * (m + j));
    return c;
}

// exact wavenumber of DFT index i of an L-point axis; L/2 carries -pi/du
double kexact(int i, int L, double du) {
    int nn = (i < (L + 1) / 2) ? i : i - L;
    return 2.0 * kPi * nn / (L * du);
}

// order-p modified wavenumber (Sec. 3.1); zero at the Nyquist index
double kmod(int i, int L, double du, int p, bool stag) {
    if (L % 2 == 0 && i == L / 2) return 0.0;
    double k = kexact(i, L, du);
    if (p == 0) return k;
    double s = 0;
    if (!stag) {
        std::vector<double> w = weights_nodal(p);
        for (size_t j = 0; j < w.size(); ++j) s += w[j] * std::sin((j + 1) * k * du) / (du / 2);
    } else {
        std::vector<double> c = weights_staggered(p);
        for (size_t j = 0; j < c.size(); ++j) s += c[j] * 2.0 * std::sin((2.0 * j + 1.0) * k * du / 2) / du;
    }
    return s;
}

// [k] of the heat-equation Laplacian symbol: the order-p staggered first
// difference (p = 0: exact k), the Nyquist index keeping k = -pi/du
double kheat(int i, int L, double du, int p) {
    const double k = kexact(i, L, du);
    if (p == 0) return k;
    const std::vector<double> c = weights_staggered(p);
    double s = 0;
    for (size_t j = 0; j < c.size(); ++j) s += c[j] * 2.0 * std::sin((2.0 * j + 1.0) * k * du / 2) / du;
    return s;
}

// Split of an axis length: two factors in 1..16 (the most balanced pair),
// else three in 2..16 (f3 > 1); false if neither exists.
bool factor(int n, AxisPlan& ax) {
    ax.f3 = 0;
    ax.pad = 0;
    ax.f1 = split_first(n);
    if (ax.f1) {
        ax.f2 = n / ax.f1;
        return true;
    }
    ax.f1 = split3_first(n);
    if (!ax.f1) return false;
    ax.f2 = split_first(n / ax.f1);
    ax.f3 = n / ax.f1 / ax.f2;
    return true;
}

// Natural (frequency) index held at position P of an n-point axis split
// with first factor f1 (the position order of the forward transforms:
// frequency k1 + f1 k2 at position k1 f2 + k2, or with three factors
// k1 + f1 k2 + f1 f2 k3 at position (k1 f2 + k2) f3 + k3).
int axis_nat(int n, int f1, int P) {
    const int m = n / f1;
    if (m <= kMaxDft) return P / m + f1 * (P % m);
    const int f2 = split_first(m), f3 = m / f2;
    const int k1 = P / m, rem = P % m, k2 = rem / f3, k3 = rem % f3;
    return k1 + f1 * (k2 + f2 * k3);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// FP32 pair (x, y) near (a, b) whose squared norm is closest to r2: among
// the roundings of a and b and their neighbours two units in the last place
// away, the pair with the smallest |x^2 + y^2 - r2| (ties: the nearer pair).
// A unit twiddle (r2 = 1) rounded this way keeps each stage of the FP32
// transform closer to unitary than independent rounding does.  The phase
// error it trades in cancels between a forward transform and the inverse
// that conjugates the same twiddle, while a magnitude error would not; the
// rotation (C, S) of Eq. 1 is rounded to nearest instead, because its phase
// error accumulates from step to step.
void unit_round(double a, double b, double r2, float& x, float& y) {
    float ca[5], cb[5];
    ca[2] = float(a);
    cb[2] = float(b);
    ca[1] = std::nextafter(ca[2], -INFINITY); ca[0] = std::nextafter(ca[1], -INFINITY);
    ca[3] = std::nextafter(ca[2], INFINITY); ca[4] = std::nextafter(ca[3], INFINITY);
    cb[1] = std::nextafter(cb[2], -INFINITY); cb[0] = std::nextafter(cb[1], -INFINITY);
    cb[3] = std::nextafter(cb[2], INFINITY); cb[4] = std::nextafter(cb[3], INFINITY);
    double best = INFINITY, bestd = INFINITY;
    x = ca[2];
    y = cb[2];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            const double u = ca[i], v = cb[j];
            const double e = std::fabs((u * u + v * v) - r2);
            const double dd = (u - a) * (u - a) + (v - b) * (v - b);
            if (e < best || (e == best && dd < bestd)) { best = e; bestd = dd; x = ca[i]; y = cb[j]; }
        }
}

}  // namespace

struct psatd_plan_s {
    int flags = 0;
    int gn[3] = {0, 0, 0};
    std::vector<psatd_sub> subs;
    std::vector<SubDesc> desc;
    std::vector<Segment> segs;
    std::vector<IoDesc> io;            // global-array <-> arena copy descriptors
    std::vector<int> io_plane_sub;     // subdomain of every local plane, then of every valid plane
    int64_t io_planes_local = 0, io_planes_valid = 0;
    int64_t arena_elems = 0;
    int nf = 9;
    bool f64 = false, stag = false, plain = false, diag = false;
    bool heat = false, heat_src = false;   // the heat equation (Sec. 5) instead of Maxwell
    int nout = 6;                          // fields written back: E, B (heat: T)
    // twiddle pool: (n) -> offset; post twiddles: (Lx) -> offset
    std::map<int, int> tw_off, post_off;
    int64_t n_tw = 0;
    // table sets keyed by (Lx, Ly, Lz, p, fx1, fy1, fz1)
    struct TabKey { int Lx, Ly, Lz, p, f1x, f1y, f1z; bool operator<(const TabKey& o) const {
        return std::tie(Lx, Ly, Lz, p, f1x, f1y, f1z) < std::tie(o.Lx, o.Ly, o.Lz, o.p, o.f1x, o.f1y, o.f1z); } };
    std::map<TabKey, int> tab_index;
    std::vector<TabKey> tab_keys;
    std::vector<int64_t> tab_coef_off, tab_k_off, tab_ph_off;
    int64_t n_tab = 0, n_tabc = 0;
    int64_t items[5] = {0, 0, 0, 0, 0};   // stages A (or x rows), B, C (or x rows), y columns fwd, inv
    int64_t exch_items = 0;
    int64_t per_sub[5] = {0, 0, 0, 0, 0};   // items per subdomain when uniform
    int variant = -1;                  // compile-time geometry variant, or -1
    int smemA = 0, smemB = 0, smemC = 0, smemR = 0, smemK = 0;
    bool split = false;                // split-plane schedule (row and column launches)
    bool reg = false;                  // FP32 plane stages with compile-time-length transforms
    bool regB = false;                 // FP32 z/Eq. 1 stage with compile-time-length transforms
    int smemAreg = 0, smemCreg = 0;
    // workspace layout (bytes)
    size_t off_desc = 0, off_seg = 0, off_tw = 0, off_tab = 0, off_tabc = 0, off_gauss = 0, off_work = 0, off_spec = 0, ws_need = 0;
    size_t off_io = 0, off_io_map = 0;
    int64_t spec_elems = 0;
    char* ws = nullptr;
    size_t ws_size = 0;
    cudaStream_t setup_stream = nullptr;   // stream of the set-up copies (psatd_plan), or the legacy stream
    bool bound_stream = false;
    bool coeffs = false;
    std::string err;
    // host images for pushes into library-owned device memory (push_into)
    bool img_valid = false;
    char* static_base = nullptr;       // static workspace of the last psatd_push_static on this plan
    double img_c_dt = 0, img_dx[3] = {0, 0, 0};
    std::vector<char> img_tw, img_tab, img_tabc;
};

static int fail(psatd_plan_s* p, int code, const std::string& msg) {
    if (p) p->err = msg;
    return code;
}

static int cuda_fail(psatd_plan_s* p, cudaError_t e, const char* where) {
    return fail(p, PSATD_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device image of the twiddle pool: exp(-2 pi i m/n) per transform length and
// the real-split twiddles exp(-2 pi i k/Lx) in position order.
static std::vector<char> twiddle_image(const psatd_plan_s* p) {
    std::vector<cd> tw(size_t(p->n_tw));
    for (auto& kv : p->tw_off)
        for (int m = 0; m < kv.first; ++m) tw[kv.second + m] = unit_root(m, kv.first);
    for (auto& kv : p->post_off) {
        const int Lx = kv.first / 32, f1 = kv.first % 32, h = Lx / 2;
        for (int P = 0; P < h; ++P) tw[kv.second + P] = unit_root(axis_nat(h, f1, P), Lx);
    }
    // each twiddle is stored as (hi, lo): in FP32 lo is the rounding of the
    // remainder so that hi + lo carries the FP64 value; in FP64 lo = 0
    std::vector<char> out;
    if (p->f64) {
        std::vector<double> t64(tw.size() * 4, 0.0);
        for (size_t i = 0; i < tw.size(); ++i) { t64[4 * i] = tw[i].real(); t64[4 * i + 1] = tw[i].imag(); }
        out.assign(reinterpret_cast<const char*>(t64.data()), reinterpret_cast<const char*>(t64.data() + t64.size()));
    } else {
        std::vector<float> t32(tw.size() * 4);
        for (size_t i = 0; i < tw.size(); ++i) {
            float hr, hi;
            unit_round(tw[i].real(), tw[i].imag(), 1.0, hr, hi);
            t32[4 * i] = hr;
            t32[4 * i + 1] = hi;
            t32[4 * i + 2] = float(tw[i].real() - double(hr));
            t32[4 * i + 3] = float(tw[i].imag() - double(hi));
        }
        out.assign(reinterpret_cast<const char*>(t32.data()), reinterpret_cast<const char*>(t32.data() + t32.size()));
    }
    return out;
}

// Device images of the Eq. 1 coefficient tables (real part) and of the
// stagger phases (complex part) for c_dt and dx, built in FP64 and stored in
// the plan's precision.
static void table_images(const psatd_plan_s* p, double c_dt, const double dx[3], std::vector<char>& out_tab,
                         std::vector<char>& out_tabc) {
    std::vector<double> tab(size_t(p->n_tab), 0.0);
    std::vector<cd> tabc(size_t(std::max<int64_t>(p->n_tabc, 1)));
    for (size_t ti = 0; ti < p->tab_keys.size(); ++ti) {
        const auto& key = p->tab_keys[ti];
        const int L[3] = {key.Lx, key.Ly, key.Lz};
        const int h = L[0] / 2, lxh = h + 1, q = L[1] * lxh;
        const int f1[3] = {key.f1x, key.f1y, key.f1z};
        const int n[3] = {h, L[1], L[2]};
        // natural index held at each position of an axis (position order of the
        // forward transforms: frequency k1 + f1 k2 at position k1 f2 + k2)
        std::vector<int> nat[3];
        for (int a = 0; a < 3; ++a) {
            int len = a == 0 ? lxh : n[a];
            nat[a].resize(len);
            for (int P = 0; P < n[a]; ++P) nat[a][P] = axis_nat(n[a], f1[a], P);
            if (a == 0) nat[0][h] = h;
        }
        std::vector<double> km[3];
        for (int a = 0; a < 3; ++a) {
            km[a].resize(nat[a].size());
            for (size_t P = 0; P < nat[a].size(); ++P) km[a][P] = kmod(nat[a][P], L[a], dx[a], key.p, p->stag);
        }
        double* tk = tab.data() + p->tab_k_off[ti];
        for (int P = 0; P < lxh; ++P) tk[P] = km[0][P];
        for (int P = 0; P < L[1]; ++P) tk[lxh + P] = km[1][P];
        for (int P = 0; P < L[2]; ++P) tk[lxh + L[1] + P] = km[2][P];
        if (p->stag) {
            cd* ph = tabc.data() + p->tab_ph_off[ti];
            for (int P = 0; P < lxh; ++P) ph[P] = std::exp(cd(0, -kexact(nat[0][P], L[0], dx[0]) * dx[0] / 2));
            for (int P = 0; P < L[1]; ++P) ph[lxh + P] = std::exp(cd(0, -kexact(nat[1][P], L[1], dx[1]) * dx[1] / 2));
            for (int P = 0; P < L[2]; ++P) ph[lxh + L[1] + P] = std::exp(cd(0, -kexact(nat[2][P], L[2], dx[2]) * dx[2] / 2));
        }
        // Eq. 1 coefficients per mode, scaled by 1/(Lx Ly Lz) (the inverse
        // transforms are unnormalised); 1/|k| is not scaled
        const double invN = 1.0 / (double(L[0]) * L[1] * L[2]);
        const int64_t NM = int64_t(L[2]) * q;
        double* tc = tab.data() + p->tab_coef_off[ti];
        if (p->heat) {
            // heat equation: exp(-x) and (1 - exp(-x))/x, x = D dt |[k]|^2
            // (c_dt holds D dt), scaled by 1/(Lx Ly Lz)
            std::vector<double> k2[3];
            for (int a = 0; a < 3; ++a) {
                k2[a].resize(nat[a].size());
                for (size_t P = 0; P < nat[a].size(); ++P) {
                    const double v = kheat(nat[a][P], L[a], dx[a], key.p);
                    k2[a][P] = v * v;
                }
            }
            for (int zp = 0; zp < L[2]; ++zp)
                for (int yp = 0; yp < L[1]; ++yp)
                    for (int xp = 0; xp < lxh; ++xp) {
                        const double x = c_dt * (k2[0][xp] + k2[1][yp] + k2[2][zp]);
                        const int64_t i = int64_t(zp) * q + int64_t(yp) * lxh + xp;
                        tc[TAB_C * NM + i] = std::exp(-x) * invN;
                        tc[TAB_S * NM + i] = (x > 0 ? -std::expm1(-x) / x : 1.0) * invN;
                    }
            continue;
        }
        for (int zp = 0; zp < L[2]; ++zp)
            for (int yp = 0; yp < L[1]; ++yp)
                for (int xp = 0; xp < lxh; ++xp) {
                    const double kx = km[0][xp], ky = km[1][yp], kz = km[2][zp];
                    const double k = std::sqrt(kx * kx + ky * ky + kz * kz);
                    const double x = k * c_dt;
                    const double C = std::cos(x), S = std::sin(x);
                    const double omc = 2.0 * std::sin(x / 2) * std::sin(x / 2);
                    double Sk, omck, dk, inv;
                    if (k > 0) {
                        Sk = S / k; omck = omc / k; inv = 1.0 / k;
                        dk = (std::fabs(x) < 1e-3) ? c_dt * (-x * x / 6.0 + x * x * x * x / 120.0) : Sk - c_dt;
                    } else {
                        Sk = c_dt; omck = 0.0; inv = 0.0; dk = 0.0;
                    }
                    const int64_t i = int64_t(zp) * q + int64_t(yp) * lxh + xp;
                    tc[TAB_C * NM + i] = C * invN;
                    tc[TAB_S * NM + i] = S * invN;
                    tc[TAB_SK * NM + i] = Sk * invN;
                    tc[TAB_OMC * NM + i] = omc * invN;
                    tc[TAB_OMCK * NM + i] = omck * invN;
                    tc[TAB_DK * NM + i] = dk * invN;
                    tc[TAB_INVK * NM + i] = inv;
                }
    }
    if (p->f64) {
        out_tab.assign(reinterpret_cast<const char*>(tab.data()), reinterpret_cast<const char*>(tab.data() + tab.size()));
        out_tabc.assign(reinterpret_cast<const char*>(tabc.data()), reinterpret_cast<const char*>(tabc.data() + size_t(p->n_tabc)));
    } else {
        std::vector<float> t32(tab.begin(), tab.end());
        out_tab.assign(reinterpret_cast<const char*>(t32.data()), reinterpret_cast<const char*>(t32.data() + t32.size()));
        std::vector<float> c32(size_t(p->n_tabc) * 2);
        for (int64_t i = 0; i < p->n_tabc; ++i) { c32[2 * i] = float(tabc[i].real()); c32[2 * i + 1] = float(tabc[i].imag()); }
        out_tabc.assign(reinterpret_cast<const char*>(c32.data()), reinterpret_cast<const char*>(c32.data() + c32.size()));
    }
}

extern "C" {

const char* psatd_status_string(int s) {
    switch (s) {
        case PSATD_OK: return "ok";
        case PSATD_E_ARG: return "invalid argument";
        case PSATD_E_SHAPE: return "invalid decomposition or shape";
        case PSATD_E_NOMEM: return "workspace too small";
        case PSATD_E_CUDA: return "CUDA error";
        case PSATD_E_UNSUPPORTED: return "unsupported local length";
        case PSATD_E_STATE: return "workspace or coefficients not set";
        case PSATD_E_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char* psatd_last_error(psatd_plan_t p) { return p ? p->err.c_str() : "null plan"; }

int psatd_plan_create(psatd_plan_t* out, const int32_t global_n[3], const psatd_sub* subs, int32_t nsub, int32_t flags) {
    return psatd_plan_create_tuned(out, global_n, subs, nsub, flags, nullptr);
}

int psatd_plan(psatd_plan_t* out, const int32_t global_n[3], const psatd_sub* subs, int32_t nsub, int32_t flags,
               void* cuda_stream) {
    const int r = psatd_plan_create_tuned(out, global_n, subs, nsub, flags, nullptr);
    if (r == PSATD_OK) {
        (*out)->setup_stream = static_cast<cudaStream_t>(cuda_stream);
        (*out)->bound_stream = true;
    }
    return r;
}

int psatd_plan_create_tuned(psatd_plan_t* out, const int32_t global_n[3], const psatd_sub* subs, int32_t nsub,
                            int32_t flags, const psatd_tuning* tuning) {
    if (!out || !global_n || !subs || nsub <= 0) return PSATD_E_ARG;
    if (tuning) {
        const int cb = tuning->chunk_b;
        if (cb < 0 || cb > 1024) return PSATD_E_ARG;
        for (int a = 0; a < 3; ++a) if (tuning->f1[a] < 0 || tuning->f1[a] > kMaxDft) return PSATD_E_ARG;
    }
    *out = nullptr;
    psatd_plan_s* p = new (std::nothrow) psatd_plan_s();
    if (!p) return PSATD_E_ARG;
    auto bad = [&](int code, const std::string& m) { int c = fail(p, code, m); delete p; return c; };
    int prec = flags & (PSATD_F32 | PSATD_F64);
    if (prec != PSATD_F32 && prec != PSATD_F64) return bad(PSATD_E_ARG, "flags must hold exactly one of PSATD_F32, PSATD_F64");
    if (flags & ~(PSATD_F32 | PSATD_F64 | PSATD_STAGGERED | PSATD_GAUSS_DIAG | PSATD_PLAIN | PSATD_GRID_PER_ITEM | PSATD_2D |
                  PSATD_SPLIT_PLANES | PSATD_HEAT | PSATD_HEAT_SOURCE | PSATD_GENERIC_PLANES | PSATD_PACKED_Z))
        return bad(PSATD_E_ARG, "unknown flag bits");
    p->flags = flags;
    p->f64 = prec == PSATD_F64;
    p->stag = flags & PSATD_STAGGERED;
    p->plain = flags & PSATD_PLAIN;
    p->diag = flags & PSATD_GAUSS_DIAG;
    p->nf = p->diag ? 10 : 9;
    p->heat = flags & PSATD_HEAT;
    p->heat_src = flags & PSATD_HEAT_SOURCE;
    if (p->heat_src && !p->heat) return bad(PSATD_E_ARG, "PSATD_HEAT_SOURCE needs PSATD_HEAT");
    if (p->heat && (p->stag || p->diag)) return bad(PSATD_E_ARG, "PSATD_HEAT excludes PSATD_STAGGERED and PSATD_GAUSS_DIAG");
    if (p->heat) {
        p->nf = p->heat_src ? 2 : 1;
        p->nout = 1;
    }
    for (int a = 0; a < 3; ++a) {
        if (global_n[a] <= 0) return bad(PSATD_E_SHAPE, "global extents must be positive");
        p->gn[a] = global_n[a];
    }
    const bool two_d = flags & PSATD_2D;
    if (two_d && global_n[2] != 1) return bad(PSATD_E_SHAPE, "PSATD_2D needs global_n[2] == 1");
    p->subs.assign(subs, subs + nsub);
    // --- tiling: inside the grid, disjoint, volumes add up -------------------
    int64_t vol = 0;
    for (int s = 0; s < nsub; ++s) {
        const psatd_sub& d = subs[s];
        for (int a = 0; a < 3; ++a) {
            if (d.n[a] <= 0 || d.lo[a] < 0 || d.lo[a] + d.n[a] > global_n[a])
                return bad(PSATD_E_SHAPE, "subdomain " + std::to_string(s) + " leaves the global grid");
        }
        if (d.ng < 0) return bad(PSATD_E_SHAPE, "negative guard width");
        if (d.order < 0 || d.order % 2) return bad(PSATD_E_SHAPE, "order must be 0 or even");
        vol += int64_t(d.n[0]) * d.n[1] * d.n[2];
    }
    if (vol != int64_t(global_n[0]) * global_n[1] * global_n[2])
        return bad(PSATD_E_SHAPE, "subdomain volumes do not add up to the global grid");
    {
        // sweep: sort by x-low and test overlaps of boxes (O(n^2) worst case, plan time only)
        std::vector<int> ord(nsub);
        for (int i = 0; i < nsub; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return subs[a].lo[0] < subs[b].lo[0]; });
        for (int ii = 0; ii < nsub; ++ii) {
            const psatd_sub& A = subs[ord[ii]];
            for (int jj = ii + 1; jj < nsub; ++jj) {
                const psatd_sub& B = subs[ord[jj]];
                if (B.lo[0] >= A.lo[0] + A.n[0]) break;
                bool ov = true;
                for (int a = 0; a < 3; ++a)
                    ov = ov && (A.lo[a] < B.lo[a] + B.n[a]) && (B.lo[a] < A.lo[a] + A.n[a]);
                if (ov) return bad(PSATD_E_SHAPE, "subdomains " + std::to_string(ord[ii]) + " and " + std::to_string(ord[jj]) + " overlap");
            }
        }
    }
    // --- per-subdomain descriptors -------------------------------------------
    const int64_t esz = p->f64 ? 8 : 4;
    p->desc.resize(nsub);
    int64_t aoff = 0;
    for (int s = 0; s < nsub; ++s) {
        const psatd_sub& u = subs[s];
        SubDesc& d = p->desc[s];
        std::memset(&d, 0, sizeof(d));
        const int ngz = two_d ? 0 : u.ng;
        for (int a = 0; a < 3; ++a) { d.nv[a] = u.n[a]; d.L[a] = u.n[a] + 2 * (a == 2 ? ngz : u.ng); }
        d.ng = u.ng;
        d.ngz = ngz;
        if (d.L[0] % 2 || d.L[0] < 2) return bad(PSATD_E_UNSUPPORTED, "local x length must be even");
        int h = d.L[0] / 2;
        if (!factor(h, d.ax) || !factor(d.L[1], d.ay) || !factor(d.L[2], d.az))
            return bad(PSATD_E_UNSUPPORTED, "subdomain " + std::to_string(s) +
                                                ": local length is not a product of two or three factors <= 16");
        if (tuning) {
            AxisPlan* ap[3] = {&d.ax, &d.ay, &d.az};
            const int len[3] = {h, d.L[1], d.L[2]};
            for (int a = 0; a < 3; ++a) {
                const int f = tuning->f1[a];
                if (f > 0 && ap[a]->f3 <= 1 && len[a] % f == 0 && len[a] / f <= kMaxDft) {
                    ap[a]->f1 = f;
                    ap[a]->f2 = len[a] / f;
                }
            }
        }
        d.ax.n = h; d.ay.n = d.L[1]; d.az.n = d.L[2];
        d.lxh = h + 1;
        d.pitch = d.lxh | 1;
        d.q = d.L[1] * d.lxh;
        d.field_off = aoff;
        int64_t cells = int64_t(d.L[0]) * d.L[1] * d.L[2];
        aoff += align_up(cells, 64);            // 256-byte aligned boxes (FP32), 512 (FP64)
    }
    p->arena_elems = aoff;
    // --- twiddles -------------------------------------------------------------
    auto add_tw = [&](int n) {
        auto it = p->tw_off.find(n);
        if (it != p->tw_off.end()) return it->second;
        int off = int(p->n_tw);
        p->tw_off[n] = off;
        p->n_tw += n;
        return off;
    };
    for (auto& d : p->desc) {
        for (AxisPlan* ap : {&d.ax, &d.ay, &d.az}) ap->tw = add_tw(ap->n);
    }
    // real-split twiddles exp(-2 pi i k/Lx) stored in the position order of the
    // x transform (entry P holds k = P/f2 + f1*(P%f2)), one table per (Lx, f1)
    for (auto& d : p->desc) {
        const int key = d.L[0] * 32 + d.ax.f1;   // (Lx, f1) fixes the split (axis_nat)
        auto it = p->post_off.find(key);
        if (it == p->post_off.end()) {
            p->post_off[key] = int(p->n_tw);
            p->n_tw += d.ax.n;
        }
        d.tw_post = p->post_off[key];
    }
    // --- coefficient tables, one set per (shape, order, factorisation) ----------
    for (int s = 0; s < nsub; ++s) {
        SubDesc& d = p->desc[s];
        psatd_plan_s::TabKey k{d.L[0], d.L[1], d.L[2], subs[s].order, d.ax.f1, d.ay.f1, d.az.f1};
        auto it = p->tab_index.find(k);
        int ti;
        if (it == p->tab_index.end()) {
            ti = int(p->tab_keys.size());
            p->tab_index[k] = ti;
            p->tab_keys.push_back(k);
            int64_t nm = int64_t(d.L[2]) * d.q;
            p->tab_coef_off.push_back(p->n_tab);
            p->n_tab += align_up(TAB_N * nm, 64);
            p->tab_k_off.push_back(p->n_tab);
            p->n_tab += align_up(d.lxh + d.L[1] + d.L[2], 64);
            p->tab_ph_off.push_back(p->stag ? p->n_tabc : -1);
            if (p->stag) p->n_tabc += align_up(d.lxh + d.L[1] + d.L[2], 32);
        } else {
            ti = it->second;
        }
        d.tab_coef = p->tab_coef_off[ti];
        d.tab_k = p->tab_k_off[ti];
        d.tab_ph = p->tab_ph_off[ti];
    }
    // --- pass-B chunk, shared memory, work items --------------------------------
    const int csz = p->f64 ? 16 : 8;
    // FP32 z/Eq. 1 stage with compile-time-length z transforms: every local z
    // length compiled in, the default z factorisation, an even number of
    // modes per plane, kRegM modes per item
    if ((flags & PSATD_PACKED_Z) && !p->f64 && !p->heat && !(flags & PSATD_GENERIC_PLANES) &&
        (!tuning || !tuning->chunk_b || tuning->chunk_b == kRegM)) {
        bool ok = true;
        for (const SubDesc& d : p->desc) {
            bool in = false;
            for (int v : kRegY) in = in || v == d.L[2];
            ok = ok && in && d.az.f1 == split_first(d.L[2]) && d.q % 2 == 0;   // 16-byte mode pairs
        }
        p->regB = ok;
    }
    int64_t iA = 0, iB = 0, iC = 0, iA2 = 0, iC1 = 0, spec = 0, maxspec = 0;
    for (int s = 0; s < nsub; ++s) {
        SubDesc& d = p->desc[s];
        int M = p->regB ? kRegM : (tuning && tuning->chunk_b) ? tuning->chunk_b : (p->f64 ? 4 : 8);
        if (!p->regB && !(tuning && tuning->chunk_b) && d.L[2] < 16)   // short z pencils (2D): widen up to 512 modes
            while (M < 512 && int64_t(p->nf) * d.L[2] * (2 * M) * csz <= 48 * 1024) M *= 2;
        if (!p->regB && !(tuning && tuning->chunk_b) && p->heat)       // one or two fields: wider chunks
            while (M < 64 && int64_t(p->nf) * d.L[2] * (2 * M) * csz <= 32 * 1024) M *= 2;
        while (!p->regB && M > 1 && int64_t(p->nf) * (d.L[2] * M + 16) * csz > 200 * 1024) M /= 2;
        d.chunkB = M;
        d.lgB = 0;
        while ((1 << d.lgB) < M) ++d.lgB;
        if ((1 << d.lgB) != M) d.lgB = -1;
        // field stride padded so that consecutive fields of a chunk fall on
        // different shared-memory banks
        int fs = d.L[2] * M;
        while ((fs * csz) % 128 != (M * csz) % 128) ++fs;
        d.fsB = fs;
        p->smemA = std::max(p->smemA, d.L[1] * d.pitch * csz);
        p->smemC = p->smemA;
        p->smemB = std::max(p->smemB, p->nf * d.fsB * csz);
        int64_t sp = int64_t(p->nf) * d.L[2] * d.q;
        d.spec_off = p->plain ? 0 : spec;
        spec += int64_t(align_up(sp, 32));
        maxspec = std::max<int64_t>(maxspec, int64_t(align_up(sp, 32)));
    }
    // planes that do not fit in shared memory take the split-plane schedule:
    // x rows and y columns in separate launches (stages 4-7 of the kernels)
    p->split = (flags & PSATD_SPLIT_PLANES) || p->smemA > kPlaneSmemMax;
    for (int s = 0; s < nsub; ++s) {
        SubDesc& d = p->desc[s];
        d.itemA = iA; d.itemB = iB; d.itemC = iC;
        d.rows = d.L[1];
        d.cols = d.lxh;
        if (p->split) {
            d.rows = std::max(1, std::min(d.L[1], kSplitRowBytes / (d.pitch * csz)));
            d.cols = std::min(d.lxh, p->f64 ? 8 : 16);
            d.itemA2 = iA2; d.itemC1 = iC1;
            const int64_t rb_in = (d.L[1] + d.rows - 1) / d.rows, rb_out = (d.nv[1] + d.rows - 1) / d.rows;
            const int64_t cb = (d.lxh + d.cols - 1) / d.cols;
            iA += int64_t(p->nf) * d.L[2] * rb_in;
            iA2 += int64_t(p->nf) * d.L[2] * cb;
            iC1 += int64_t(p->nout) * d.nv[2] * cb;
            iC += int64_t(p->nout) * d.nv[2] * rb_out;
            p->smemR = std::max(p->smemR, d.rows * d.pitch * csz);
            p->smemK = std::max(p->smemK, d.L[1] * d.cols * csz);
        } else {
            iA += int64_t(p->nf) * d.L[2];
            iC += int64_t(p->nout) * d.nv[2];
        }
        iB += (d.q + d.chunkB - 1) / d.chunkB;
    }
    p->items[0] = iA; p->items[1] = iB; p->items[2] = iC; p->items[3] = iA2; p->items[4] = iC1;
    {
        bool uni = true;
        const SubDesc& d0 = p->desc[0];
        for (const SubDesc& d : p->desc)
            uni = uni && d.L[0] == d0.L[0] && d.L[1] == d0.L[1] && d.L[2] == d0.L[2] && d.nv[1] == d0.nv[1] &&
                  d.nv[2] == d0.nv[2] && d.chunkB == d0.chunkB && d.rows == d0.rows && d.cols == d0.cols;
        if (uni)
            for (int k = 0; k < 5; ++k) p->per_sub[k] = p->items[k] / nsub;
    }
    p->spec_elems = p->plain ? maxspec : spec;
    // kernels with compile-time geometry apply when every subdomain is the
    // same cubic box with the default splits and chunk width
    {
        const FixedGeo* list = p->f64 ? kFixedF64 : kFixedF32;
        const int nl = p->f64 ? int(sizeof(kFixedF64) / sizeof(FixedGeo)) : int(sizeof(kFixedF32) / sizeof(FixedGeo));
        for (int v = 0; v < nl && p->variant < 0 && !p->split; ++v) {
            const int L = list[v].L, g = list[v].ng, M = list[v].M;
            bool ok = true;
            for (const SubDesc& d : p->desc) {
                ok = ok && d.L[0] == L && d.L[1] == L && d.L[2] == L && d.ng == g && d.ngz == g && d.nv[0] == L - 2 * g &&
                     d.nv[1] == L - 2 * g && d.nv[2] == L - 2 * g && d.chunkB == M && d.ax.f1 == split_first(L / 2) &&
                     d.ay.f1 == split_first(L) && d.az.f1 == split_first(L) && d.fsB == pad_field_stride(L, M, csz) &&
                     d.pitch == ((L / 2 + 1) | 1);
            }
            if (ok) p->variant = v;
        }
    }
    // mixed box shapes with the default chunk width: descriptor-driven
    // geometry with that width compiled in
    if (p->variant < 0 && !p->split) {
        bool dflt = true;
        for (const SubDesc& d : p->desc)
            dflt = dflt && d.chunkB == (p->f64 ? 4 : 8) && d.ax.f3 <= 1 && d.ay.f3 <= 1 && d.az.f3 <= 1;
        if (dflt) p->variant = -2;
    }
    if (p->smemB > kPlaneSmemMax || (p->split && std::max(p->smemR, p->smemK) > kPlaneSmemMax))
        return bad(PSATD_E_UNSUPPORTED, "a stage's tile does not fit in shared memory");
    // FP32 plane stages with compile-time-length transforms: every local x
    // and y length compiled in, default factorisations, at most 128 rows and
    // 64 half-spectrum columns (one thread per row, two per column)
    if (!p->f64 && !p->split && !(flags & PSATD_GENERIC_PLANES)) {
        auto listed = [](const int* l, int n, int v) { for (int i = 0; i < n; ++i) if (l[i] == v) return true; return false; };
        bool ok = true;
        for (const SubDesc& d : p->desc) {
            ok = ok && listed(kRegX2, int(sizeof(kRegX2) / sizeof(int)), d.L[0]) &&
                 listed(kRegY, int(sizeof(kRegY) / sizeof(int)), d.L[1]) && d.ax.f1 == split_first(d.L[0] / 2) &&
                 d.ay.f1 == split_first(d.L[1]) && d.lxh <= kRegThreads / 2 && d.L[1] <= kRegThreads;
            p->smemAreg = std::max(p->smemAreg, d.L[1] * reg_pitch(d.lxh) * 8);
            p->smemCreg = std::max(p->smemCreg, d.q * 8);
        }
        p->reg = ok && p->smemAreg <= kPlaneSmemMax && p->smemCreg <= kPlaneSmemMax;
    }
    // --- exchange segments (source valid box -> destination local box) ----------
    for (int s = 0; s < nsub; ++s) {
        p->desc[s].seg_begin = int(p->segs.size());
        const psatd_sub& S = subs[s];
        for (int dd = 0; dd < nsub; ++dd) {
            const psatd_sub& D = subs[dd];
            const SubDesc& Dd = p->desc[dd];
            // per axis: list of (shift, lo, hi) intersections in global unwrapped coords
            std::vector<std::tuple<long, long, long>> ax[3];
            for (int a = 0; a < 3; ++a) {
                long N = global_n[a];
                const long gD = (a == 2 && two_d) ? 0 : D.ng;
                long b0 = long(D.lo[a]) - gD, b1 = long(D.lo[a]) + D.n[a] + gD;
                long tmin = (long)std::floor(double(b0 - (S.lo[a] + S.n[a])) / N) - 1;
                long tmax = (long)std::ceil(double(b1 - S.lo[a]) / N) + 1;
                for (long t = tmin; t <= tmax; ++t) {
                    long a0 = S.lo[a] + t * N, a1 = S.lo[a] + S.n[a] + t * N;
                    long lo = std::max(a0, b0), hi = std::min(a1, b1);
                    if (lo < hi) ax[a].emplace_back(t, lo, hi);
                }
            }
            for (auto& X : ax[0]) for (auto& Y : ax[1]) for (auto& Z : ax[2]) {
                Segment g;
                std::memset(&g, 0, sizeof(g));
                g.src = s; g.dst = dd;
                g.dst_off = Dd.field_off;
                g.dLx = Dd.L[0]; g.dLy = Dd.L[1];
                long t[3] = {std::get<0>(X), std::get<0>(Y), std::get<0>(Z)};
                long lo[3] = {std::get<1>(X), std::get<1>(Y), std::get<1>(Z)};
                long hi[3] = {std::get<2>(X), std::get<2>(Y), std::get<2>(Z)};
                int x0[3], ext[3], off[3];
                for (int a = 0; a < 3; ++a) {
                    const long gS = (a == 2 && two_d) ? 0 : S.ng, gD = (a == 2 && two_d) ? 0 : D.ng;
                    long src_origin = S.lo[a] + t[a] * global_n[a] - gS;   // global coord of source local 0
                    long dst_origin = long(D.lo[a]) - gD;
                    x0[a] = int(lo[a] - src_origin);
                    ext[a] = int(hi[a] - lo[a]);
                    off[a] = int(src_origin - dst_origin);
                }
                g.x0 = x0[0]; g.y0 = x0[1]; g.z0 = x0[2];
                g.ex = ext[0]; g.ey = ext[1]; g.ez = ext[2];
                g.dx = off[0]; g.dy = off[1]; g.dz = off[2];
                g.identity = (dd == s && t[0] == 0 && t[1] == 0 && t[2] == 0) ? 1 : 0;
                g.vec4 = (g.x0 % 4 == 0 && (g.x0 + g.dx) % 4 == 0 && g.ex % 4 == 0 && g.dLx % 4 == 0) ? 1 : 0;
                p->segs.push_back(g);
            }
        }
        p->desc[s].seg_end = int(p->segs.size());
    }
    int64_t ei = 0;
    for (auto& g : p->segs) {
        g.item = ei;
        if (!g.identity) ei += g.ez;
    }
    p->exch_items = ei;
    // --- workspace layout ------------------------------------------------------
    size_t o = 0;
    p->off_desc = o; o = align_up(o + sizeof(SubDesc) * p->desc.size(), 256);
    p->off_seg = o; o = align_up(o + sizeof(Segment) * p->segs.size(), 256);
    p->off_tw = o; o = align_up(o + size_t(p->n_tw) * 4 * esz, 256);   // hi/lo pairs
    p->off_tab = o; o = align_up(o + size_t(p->n_tab) * esz, 256);
    p->off_tabc = o; o = align_up(o + size_t(std::max<int64_t>(p->n_tabc, 1)) * 2 * esz, 256);
    p->off_gauss = o; o = align_up(o + size_t(std::max<int64_t>(p->items[1], 1)) * 2 * sizeof(double), 256);
    p->off_work = o; o = align_up(o + 8 * sizeof(unsigned long long), 256);
    p->off_spec = o; o = align_up(o + size_t(p->spec_elems) * 2 * esz, 256);
    // descriptors of the global-array <-> arena copies
    for (int s = 0; s < nsub; ++s) {
        const SubDesc& d = p->desc[s];
        IoDesc q;
        std::memset(&q, 0, sizeof(q));
        q.field_off = d.field_off;
        q.zstart_local = p->io_planes_local;
        q.zstart_valid = p->io_planes_valid;
        for (int a = 0; a < 3; ++a) {
            q.L[a] = d.L[a];
            q.g[a] = a == 2 ? d.ngz : d.ng;
            q.lo[a] = subs[s].lo[a];
            q.n[a] = subs[s].n[a];
            q.org[a] = q.lo[a] - q.g[a];
        }
        p->io.push_back(q);
        p->io_planes_local += d.L[2];
        p->io_planes_valid += d.nv[2];
    }
    for (int s = 0; s < nsub; ++s) p->io_plane_sub.insert(p->io_plane_sub.end(), size_t(p->desc[s].L[2]), s);
    for (int s = 0; s < nsub; ++s) p->io_plane_sub.insert(p->io_plane_sub.end(), size_t(p->desc[s].nv[2]), s);
    p->off_io = o; o = align_up(o + sizeof(IoDesc) * p->io.size(), 256);
    p->off_io_map = o; o = align_up(o + sizeof(int) * p->io_plane_sub.size(), 256);
    p->ws_need = o;
    *out = p;
    return PSATD_OK;
}

int psatd_layout(psatd_plan_t p, int32_t sub, int64_t* offset_elems, int32_t local_n[3]) {
    if (!p) return PSATD_E_ARG;
    if (sub < 0 || sub >= int(p->desc.size())) return fail(p, PSATD_E_ARG, "subdomain index out of range");
    if (offset_elems) *offset_elems = p->desc[sub].field_off;
    if (local_n) for (int a = 0; a < 3; ++a) local_n[a] = p->desc[sub].L[a];
    return PSATD_OK;
}

int psatd_arena_elems(psatd_plan_t p, int64_t* n) {
    if (!p || !n) return PSATD_E_ARG;
    *n = p->arena_elems;
    return PSATD_OK;
}

int psatd_workspace_bytes(psatd_plan_t p, size_t* b) {
    if (!p || !b) return PSATD_E_ARG;
    *b = p->ws_need;
    return PSATD_OK;
}

int psatd_geometry_variant(psatd_plan_t p, int32_t* v) {
    if (!p || !v) return PSATD_E_ARG;
    *v = p->variant;
    return PSATD_OK;
}

int psatd_plane_engine(psatd_plan_t p, int32_t* engine) {
    if (!p || !engine) return PSATD_E_ARG;
    *engine = (p->reg ? 1 : 0) | (p->regB ? 2 : 0);
    return PSATD_OK;
}

static int io_call(psatd_plan_s* p, bool scatter, const void* const* src, void* const* dst, int32_t nfields,
                   void* stream) {
    if (!p || !src || !dst) return PSATD_E_ARG;
    if (nfields < 1 || nfields > kIoMaxFields) return fail(p, PSATD_E_ARG, "nfields must be in 1..10");
    if (!p->ws) return fail(p, PSATD_E_STATE, "set the workspace first");
    IoArgs a;
    std::memset(&a, 0, sizeof(a));
    a.desc = reinterpret_cast<const IoDesc*>(p->ws + p->off_io);
    a.plane_sub_local = reinterpret_cast<const int*>(p->ws + p->off_io_map);
    a.plane_sub_valid = a.plane_sub_local + p->io_planes_local;
    a.nsub = int(p->desc.size());
    a.nfields = nfields;
    for (int i = 0; i < 3; ++i) a.gn[i] = p->gn[i];
    a.planes_local = p->io_planes_local;
    a.planes_valid = p->io_planes_valid;
    const size_t esz = p->f64 ? 8 : 4;
    for (int f = 0; f < nfields; ++f) {
        if (!src[f] || !dst[f]) return fail(p, PSATD_E_ARG, "null array");
        if (reinterpret_cast<uintptr_t>(src[f]) % esz || reinterpret_cast<uintptr_t>(dst[f]) % esz)
            return fail(p, PSATD_E_ARG, "arrays must be aligned to their element size");
        a.in[f] = src[f];
        a.out[f] = dst[f];
    }
    cudaError_t e = launch_io(scatter, p->f64, a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(p, e, scatter ? "scatter launch" : "gather launch");
    return PSATD_OK;
}

int psatd_scatter_global(psatd_plan_t p, const void* const* global_in, void* const* arenas, int32_t nfields,
                         void* stream) {
    return io_call(p, true, global_in, arenas, nfields, stream);
}

int psatd_gather_global(psatd_plan_t p, const void* const* arenas, void* const* global_out, int32_t nfields,
                        void* stream) {
    return io_call(p, false, arenas, global_out, nfields, stream);
}

int psatd_debug_tables(psatd_plan_t p, double c_dt, const double dx[3], void* out, size_t* bytes) {
    if (!p || !bytes || !dx) return PSATD_E_ARG;
    if (!(c_dt == c_dt) || !(dx[0] > 0 && dx[1] > 0 && dx[2] > 0)) return fail(p, PSATD_E_ARG, "bad c_dt or dx");
    std::vector<char> tab, tabc;
    table_images(p, c_dt, dx, tab, tabc);
    if (out) {
        if (*bytes < tab.size()) return fail(p, PSATD_E_NOMEM, "buffer smaller than the table image");
        std::memcpy(out, tab.data(), tab.size());
    }
    *bytes = tab.size();
    return PSATD_OK;
}

int psatd_exchange_segments(psatd_plan_t p, int32_t* count, int32_t* segs) {
    if (!p || !count) return PSATD_E_ARG;
    *count = int32_t(p->segs.size());
    if (segs) {
        for (size_t i = 0; i < p->segs.size(); ++i) {
            const Segment& g = p->segs[i];
            const int32_t v[12] = {g.src, g.dst, g.x0, g.y0, g.z0, g.ex, g.ey, g.ez, g.dx, g.dy, g.dz, g.identity};
            std::memcpy(segs + 12 * i, v, sizeof(v));
        }
    }
    return PSATD_OK;
}

int psatd_check(psatd_plan_t p, int32_t* error_bits) {
    if (!p || !error_bits) return PSATD_E_ARG;
    // the attached workspace, else the static workspace of psatd_push_static
    char* base = p->ws ? p->ws : p->static_base;
    if (!base) return fail(p, PSATD_E_STATE, "set the workspace first");
    cudaError_t e = cudaDeviceSynchronize();
    unsigned int w = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&w, base + p->off_work + 7 * sizeof(unsigned long long), sizeof(w), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(base + p->off_work + 7 * sizeof(unsigned long long), 0, sizeof(w));
    if (e != cudaSuccess) return cuda_fail(p, e, "read the device error word");
    *error_bits = int32_t(w);
    return PSATD_OK;
}

int psatd_push_launches(psatd_plan_t p, int32_t* n) {
    if (!p || !n) return PSATD_E_ARG;
    int nsub = int(p->desc.size());
    const int per = p->split ? 5 : 3;
    *n = p->plain ? per * nsub + (p->exch_items > 0 ? 1 : 0) : per;
    if (p->diag) *n += 1;
    return PSATD_OK;
}

// Host-to-device copy of a set-up call: blocking on the legacy default
// stream, or enqueued on the plan's bound stream (psatd_plan) and that stream
// synchronised.
static cudaError_t setup_copy(psatd_plan_s* p, void* dst, const void* src, size_t n) {
    if (!p->bound_stream) return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
    cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, p->setup_stream);
    return e == cudaSuccess ? cudaStreamSynchronize(p->setup_stream) : e;
}

static cudaError_t setup_zero(psatd_plan_s* p, void* dst, size_t n) {
    if (!p->bound_stream) return cudaMemset(dst, 0, n);
    cudaError_t e = cudaMemsetAsync(dst, 0, n, p->setup_stream);
    return e == cudaSuccess ? cudaStreamSynchronize(p->setup_stream) : e;
}

int psatd_set_workspace(psatd_plan_t p, void* dev, size_t bytes) {
    if (!p || !dev) return PSATD_E_ARG;
    if (reinterpret_cast<uintptr_t>(dev) % 256) return fail(p, PSATD_E_ARG, "workspace must be 256-byte aligned");
    if (bytes < p->ws_need) return fail(p, PSATD_E_NOMEM, "workspace smaller than psatd_workspace_bytes");
    p->ws = static_cast<char*>(dev);
    p->ws_size = bytes;
    p->coeffs = false;
    cudaError_t e = setup_copy(p, p->ws + p->off_desc, p->desc.data(), sizeof(SubDesc) * p->desc.size());
    if (e != cudaSuccess) { p->ws = nullptr; return cuda_fail(p, e, "copy descriptors"); }
    if (!p->segs.empty()) {
        e = setup_copy(p, p->ws + p->off_seg, p->segs.data(), sizeof(Segment) * p->segs.size());
        if (e != cudaSuccess) { p->ws = nullptr; return cuda_fail(p, e, "copy segments"); }
    }
    e = setup_copy(p, p->ws + p->off_io, p->io.data(), sizeof(IoDesc) * p->io.size());
    if (e == cudaSuccess)
        e = setup_copy(p, p->ws + p->off_io_map, p->io_plane_sub.data(), sizeof(int) * p->io_plane_sub.size());
    if (e != cudaSuccess) { p->ws = nullptr; return cuda_fail(p, e, "copy the copy descriptors"); }
    {
        const std::vector<char> tw = twiddle_image(p);
        e = setup_copy(p, p->ws + p->off_tw, tw.data(), tw.size());
    }
    // the persistent launches' ticket counters and the error word (the last
    // slot) start at zero (each launch returns its counter to zero when it ends)
    if (e == cudaSuccess) e = setup_zero(p, p->ws + p->off_work, 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) { p->ws = nullptr; return cuda_fail(p, e, "copy twiddles"); }
    return PSATD_OK;
}

int psatd_set_coeffs(psatd_plan_t p, double c_dt, const double dx[3]) {
    if (!p || !dx) return PSATD_E_ARG;
    if (!p->ws) return fail(p, PSATD_E_STATE, "set the workspace first");
    if (!(c_dt == c_dt) || !(dx[0] > 0 && dx[1] > 0 && dx[2] > 0)) return fail(p, PSATD_E_ARG, "bad c_dt or dx");
    std::vector<char> tab, tabc;
    table_images(p, c_dt, dx, tab, tabc);
    cudaError_t e = setup_copy(p, p->ws + p->off_tab, tab.data(), tab.size());
    if (e == cudaSuccess && p->n_tabc)
        e = setup_copy(p, p->ws + p->off_tabc, tabc.data(), tabc.size());
    if (e != cudaSuccess) return cuda_fail(p, e, "copy coefficient tables");
    p->coeffs = true;
    return PSATD_OK;
}

static int check_fields(psatd_plan_s* p, const psatd_fields* f, bool need_j) {
    if (!f) return fail(p, PSATD_E_ARG, "null fields");
    if (p->heat) {
        if (!f->E[0] || reinterpret_cast<uintptr_t>(f->E[0]) % 16) return fail(p, PSATD_E_ARG, "T (fields->E[0]) must be a 16-byte aligned arena");
        if (need_j && p->heat_src && (!f->J[0] || reinterpret_cast<uintptr_t>(f->J[0]) % 16))
            return fail(p, PSATD_E_ARG, "PSATD_HEAT_SOURCE needs a 16-byte aligned source arena in fields->J[0]");
        return PSATD_OK;
    }
    for (int a = 0; a < 3; ++a) {
        if (!f->E[a] || !f->B[a]) return fail(p, PSATD_E_ARG, "null E or B arena");
        if (need_j && !f->J[a]) return fail(p, PSATD_E_ARG, "null J arena");
        const void* ptrs[3] = {f->E[a], f->B[a], need_j ? f->J[a] : f->E[a]};
        for (auto q : ptrs) if (reinterpret_cast<uintptr_t>(q) % 16) return fail(p, PSATD_E_ARG, "field arenas must be 16-byte aligned");
    }
    if (need_j && p->diag) {
        if (!f->rho) return fail(p, PSATD_E_ARG, "PSATD_GAUSS_DIAG needs rho");
        if (reinterpret_cast<uintptr_t>(f->rho) % 16) return fail(p, PSATD_E_ARG, "rho must be 16-byte aligned");
    }
    return PSATD_OK;
}

// Launch arguments for a workspace image that starts at `base`.
static LaunchCommon common_at(psatd_plan_s* p, char* base, const psatd_fields* f) {
    LaunchCommon c;
    std::memset(&c, 0, sizeof(c));
    c.subs = base + p->off_desc;
    c.segs = base + p->off_seg;
    c.tw = base + p->off_tw;
    c.tab = base + p->off_tab;
    c.tabc = base + p->off_tabc;
    c.spec = base + p->off_spec;
    for (int a = 0; a < 3; ++a) { c.eb[a] = f->E[a]; c.eb[3 + a] = f->B[a]; c.jr[a] = f->J[a]; }
    c.jr[3] = f->rho;
    if (p->heat) {
        // the heat equation's inputs are field 0 (T, written back) and field 1
        // (the source, read by the forward stages only)
        for (int a = 0; a < 6; ++a) c.eb[a] = nullptr;
        for (int a = 0; a < 4; ++a) c.jr[a] = nullptr;
        c.eb[0] = f->E[0];
        c.eb[1] = p->heat_src ? const_cast<void*>(f->J[0]) : nullptr;   // never written (nout = 1)
    }
    c.gauss_part = reinterpret_cast<double*>(base + p->off_gauss);
    c.work = reinterpret_cast<unsigned long long*>(base + p->off_work);
    c.err = reinterpret_cast<unsigned int*>(base + p->off_work + 7 * sizeof(unsigned long long));
    c.persistent = (p->flags & PSATD_GRID_PER_ITEM) ? 0 : 1;
    c.nsub = int(p->desc.size());
    c.nseg = int(p->segs.size());
    c.nf = p->nf;
    c.nout = p->nout;
    c.staggered = p->stag ? 1 : 0;
    c.own_only = 0;
    for (int i = 0; i < 5; ++i) c.per_sub[i] = p->per_sub[i];
    c.variant = p->variant;
    return c;
}

static LaunchCommon common(psatd_plan_s* p, const psatd_fields* f) { return common_at(p, p->ws, f); }

static cudaError_t stage(psatd_plan_s* p, int st, const LaunchCommon& c, int64_t i0, int64_t n, int smem, cudaStream_t s) {
    return p->f64 ? launch_stage_f64(st, c, i0, n, smem, s) : launch_stage_f32(st, c, i0, n, smem, s);
}

int psatd_exchange_guards(psatd_plan_t p, const psatd_fields* f, void* stream) {
    if (!p) return PSATD_E_ARG;
    if (!p->ws) return fail(p, PSATD_E_STATE, "set the workspace first");
    int r = check_fields(p, f, false);
    if (r) return r;
    LaunchCommon c = common(p, f);
    cudaError_t e = stage(p, 3, c, 0, p->exch_items, 0, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(p, e, "exchange launch");
    return PSATD_OK;
}

static int launch_push(psatd_plan_s* p, LaunchCommon c, double* gauss_dev, cudaStream_t s, void* const* ev);

static int push_impl(psatd_plan_s* p, const psatd_fields* f, double* gauss_dev, void* stream, void* const* ev) {
    if (!p) return PSATD_E_ARG;
    if (!p->ws || !p->coeffs) return fail(p, PSATD_E_STATE, "workspace and coefficients must be set before psatd_push");
    int r = check_fields(p, f, true);
    if (r) return r;
    if (gauss_dev && !p->diag) return fail(p, PSATD_E_ARG, "gauss output needs PSATD_GAUSS_DIAG");
    return launch_push(p, common(p, f), gauss_dev, static_cast<cudaStream_t>(stream), ev);
}

// Enqueue every stage of one push (and the Gauss reduction) on stream s.
static int launch_push(psatd_plan_s* p, LaunchCommon c, double* gauss_dev, cudaStream_t s, void* const* ev) {
    auto mark = [&](int i) -> cudaError_t {
        if (!ev || !ev[i]) return cudaSuccess;
        return cudaEventRecord(static_cast<cudaEvent_t>(ev[i]), s);
    };
    cudaError_t e = cudaSuccess;
    if ((e = mark(0)) != cudaSuccess) return cuda_fail(p, e, "event record");
    // the forward stages, pass B and the inverse stages over items [i0, i0+n)
    // of each (n < 0: every item of the stage)
    struct Range { int64_t a0, an, a20, a2n, b0, bn, c10, c1n, c0, cn; };
    auto run = [&](const Range& r) -> int {
        if (p->reg) {
            if ((e = launch_stage_reg(0, c, r.a0, r.an, p->smemAreg, s)) != cudaSuccess) return cuda_fail(p, e, "pass A launch");
        } else if (!p->split) {
            if ((e = stage(p, 0, c, r.a0, r.an, p->smemA, s)) != cudaSuccess) return cuda_fail(p, e, "pass A launch");
        } else {
            if ((e = stage(p, 4, c, r.a0, r.an, p->smemR, s)) != cudaSuccess) return cuda_fail(p, e, "x rows launch");
            if ((e = stage(p, 5, c, r.a20, r.a2n, p->smemK, s)) != cudaSuccess) return cuda_fail(p, e, "y columns launch");
        }
        if (!p->plain && (e = mark(1)) != cudaSuccess) return cuda_fail(p, e, "event record");
        if (p->regB) {
            if ((e = launch_stage_reg(1, c, r.b0, r.bn, p->smemB, s)) != cudaSuccess) return cuda_fail(p, e, "pass B launch");
        } else if ((e = stage(p, p->heat ? 8 : 1, c, r.b0, r.bn, p->smemB, s)) != cudaSuccess) {
            return cuda_fail(p, e, "pass B launch");
        }
        if (!p->plain && (e = mark(2)) != cudaSuccess) return cuda_fail(p, e, "event record");
        if (p->reg) {
            if ((e = launch_stage_reg(2, c, r.c0, r.cn, p->smemCreg, s)) != cudaSuccess) return cuda_fail(p, e, "pass C launch");
        } else if (!p->split) {
            if ((e = stage(p, 2, c, r.c0, r.cn, p->smemC, s)) != cudaSuccess) return cuda_fail(p, e, "pass C launch");
        } else {
            if ((e = stage(p, 6, c, r.c10, r.c1n, p->smemK, s)) != cudaSuccess) return cuda_fail(p, e, "y columns launch");
            if ((e = stage(p, 7, c, r.c0, r.cn, p->smemR, s)) != cudaSuccess) return cuda_fail(p, e, "x rows launch");
        }
        return PSATD_OK;
    };
    if (!p->plain) {
        int r = run(Range{0, p->items[0], 0, p->items[3], 0, p->items[1], 0, p->items[4], 0, p->items[2]});
        if (r) return r;
    } else {
        c.own_only = 1;
        const int nsub = int(p->desc.size());
        for (int i = 0; i < nsub; ++i) {
            const SubDesc& d = p->desc[i];
            // item ranges of subdomain i: up to the next subdomain's first items
            const bool last = i + 1 == nsub;
            const SubDesc* n = last ? nullptr : &p->desc[i + 1];
            Range g{d.itemA, (last ? p->items[0] : n->itemA) - d.itemA,
                    d.itemA2, (last ? p->items[3] : n->itemA2) - d.itemA2,
                    d.itemB, (last ? p->items[1] : n->itemB) - d.itemB,
                    d.itemC1, (last ? p->items[4] : n->itemC1) - d.itemC1,
                    d.itemC, (last ? p->items[2] : n->itemC) - d.itemC};
            int r = run(g);
            if (r) return r;
        }
        if ((e = stage(p, 3, c, 0, p->exch_items, 0, s)) != cudaSuccess) return cuda_fail(p, e, "exchange launch");
    }
    if ((e = mark(3)) != cudaSuccess) return cuda_fail(p, e, "event record");
    if (p->diag && gauss_dev) {
        e = launch_gauss_reduce(c.subs, c.nsub, c.gauss_part, gauss_dev, s);
        if (e != cudaSuccess) return cuda_fail(p, e, "gauss reduce launch");
    }
    return PSATD_OK;
}

int psatd_push(psatd_plan_t p, const psatd_fields* f, double* gauss_dev, void* stream) {
    return push_impl(p, f, gauss_dev, stream, nullptr);
}

int psatd_push_profiled(psatd_plan_t p, const psatd_fields* f, double* gauss_dev, void* stream, void* const events[4]) {
    return push_impl(p, f, gauss_dev, stream, events);
}

int psatd_destroy(psatd_plan_t p) {
    delete p;
    return PSATD_OK;
}

}  // extern "C"

namespace psatd {

// psatd_push on a workspace image at `base` (cap bytes) that the library owns
// instead of the caller: descriptors, segments, twiddles and tables for
// (c_dt, dx) are copied there on stream s (stream-ordered, from host images
// kept in the plan) before the stages are enqueued on the same stream.
int push_into(psatd_plan_s* p, char* base, size_t cap, double c_dt, const double dx[3], const psatd_fields* f,
              double* gauss_dev, cudaStream_t s) {
    if (!p) return PSATD_E_ARG;
    if (!base) return fail(p, PSATD_E_CUDA, "static workspace address unavailable");
    if (!dx || !(c_dt == c_dt) || !(dx[0] > 0 && dx[1] > 0 && dx[2] > 0)) return fail(p, PSATD_E_ARG, "bad c_dt or dx");
    if (p->ws_need > cap)
        return fail(p, PSATD_E_NOMEM, "plan needs " + std::to_string(p->ws_need) + " bytes of workspace, the static workspace holds " +
                                          std::to_string(cap));
    int r = check_fields(p, f, true);
    if (r) return r;
    if (gauss_dev && !p->diag) return fail(p, PSATD_E_ARG, "gauss output needs PSATD_GAUSS_DIAG");
    if (!p->img_valid || p->img_c_dt != c_dt || p->img_dx[0] != dx[0] || p->img_dx[1] != dx[1] || p->img_dx[2] != dx[2]) {
        p->img_tw = twiddle_image(p);
        table_images(p, c_dt, dx, p->img_tab, p->img_tabc);
        p->img_c_dt = c_dt;
        for (int a = 0; a < 3; ++a) p->img_dx[a] = dx[a];
        p->img_valid = true;
    }
    // the ticket counters start at zero; the error word (slot 7) is kept, so
    // that psatd_check can report what earlier static pushes recorded
    static const unsigned long long zero_work[7] = {0, 0, 0, 0, 0, 0, 0};
    struct Part { size_t off; const void* src; size_t n; } parts[] = {
        {p->off_work, zero_work, sizeof(zero_work)},
        {p->off_desc, p->desc.data(), sizeof(SubDesc) * p->desc.size()},
        {p->off_seg, p->segs.data(), sizeof(Segment) * p->segs.size()},
        {p->off_tw, p->img_tw.data(), p->img_tw.size()},
        {p->off_tab, p->img_tab.data(), p->img_tab.size()},
        {p->off_tabc, p->img_tabc.data(), p->n_tabc ? p->img_tabc.size() : 0},
    };
    for (const Part& q : parts) {
        if (!q.n) continue;
        cudaError_t e = cudaMemcpyAsync(base + q.off, q.src, q.n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(p, e, "copy plan image to the static workspace");
    }
    p->static_base = base;
    return launch_push(p, common_at(p, base, f), gauss_dev, s, nullptr);
}

// Record a message on the plan from outside this file.
int set_error(psatd_plan_s* p, int code, const char* msg) { return fail(p, code, msg); }

}  // namespace psatd
