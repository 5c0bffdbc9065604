// Internal descriptors shared by the host plan builder and the CUDA kernels.
#pragma once
#include <stdint.h>

namespace psatd {

constexpr int kMaxDft = 16;       // largest register DFT
constexpr int kThreads = 256;     // threads per CTA of every stage kernel
constexpr int kSegSmem = 64;      // exchange segments staged in shared memory per CTA
constexpr int kPlaneSmemMax = 216 * 1024;   // dynamic shared memory of one stage tile (the rest: static)
constexpr int kSplitRowBytes = 32 * 1024;   // row block of the split-plane schedule

// Default split n = f1 * f2 of an FFT length (both factors in 1..16): the
// most balanced pair, then the larger f1; 0 if none exists.
constexpr int split_first(int n) {
    int best = -1, f1 = 0;
    for (int a = 1; a <= kMaxDft; ++a) {
        if (n % a) continue;
        const int b = n / a;
        if (b > kMaxDft) continue;
        const int score = (a < b ? a : b) * 64 + a;
        if (score > best) { best = score; f1 = a; }
    }
    return best >= 0 ? f1 : 0;
}

// Field stride of a pass-B chunk in shared memory (complex elements of csz
// bytes): at least lz*m and padded so that consecutive fields fall on
// different banks.
constexpr int pad_field_stride(int lz, int m, int csz) {
    int fs = lz * m;
    while ((fs * csz) % 128 != (m * csz) % 128) ++fs;
    return fs;
}

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// FP32 plane stages with thread-private transforms of compile-time length
// (psatd_regfft.cuh): the local x and y lengths they are compiled for, the
// CTA size, and the shared-memory row pitch of pass A (complex elements: at
// least Lx/2+1 and = 2 mod 4, so rows are 16-byte aligned and eight
// consecutive rows start on distinct 16-byte bank groups).
constexpr int kRegThreads = 128;
constexpr int kRegX2[] = {32, 40, 48, 56, 64, 72, 88, 96, 104};
constexpr int kRegY[] = {32, 48, 64, 80, 96};
constexpr int reg_pitch(int lxh) { return lxh + ((2 - lxh % 4) + 4) % 4; }
// modes per item of the compiled-length z/Eq. 1 stage (pass B): three pairs,
// so that the ten fields' pairs fill 30 lanes of a warp; the z lengths it is
// compiled for are those of kRegY
constexpr int kRegM = 6;

// Cubic local boxes (side L, ng guards, pass-B chunk M, default splits) that
// have kernels compiled with their geometry fixed at compile time.
struct FixedGeo { int L, ng, M; };
constexpr FixedGeo kFixedF32[5] = {{96, 16, 8}, {64, 16, 8}, {48, 8, 8}, {32, 0, 8}, {96, 16, 4}};
constexpr FixedGeo kFixedF64[3] = {{96, 16, 4}, {48, 8, 4}, {32, 0, 4}};

// Three-factor split n = f1 * f2 * f3 (each in 2..16) of a length with no
// two-factor split: f1 the largest factor in 2..16 whose cofactor has one,
// (f2, f3) that cofactor's default split; 0 if none exists.
constexpr int split3_first(int n) {
    for (int a = kMaxDft; a >= 2; --a)
        if (n % a == 0 && split_first(n / a) > 0 && n / a > kMaxDft) return a;
    return 0;
}

// One local FFT axis of length n = f1 * f2 (f3 <= 1), done as two register
// stages, or n = f1 * f2 * f3 (f3 > 1), done as three.  Forward output (and
// inverse input) is in "position" order: frequency k1 + f1*k2 sits at
// position k1*f2 + k2; with three factors, frequency k1 + f1*k2 + f1*f2*k3
// sits at position k1*f2*f3 + k2*f3 + k3.
struct AxisPlan {
    int n, f1, f2;
    int tw;          // offset of the n twiddles exp(-2 pi i m/n) in the pool
    int f3;          // third factor (0 or 1: a two-factor split)
    int pad;
};

// Per subdomain, everything a stage kernel needs (device copy in workspace).
struct SubDesc {
    int L[3];            // local extents x, y, z
    int nv[3];           // valid extents
    int ng;              // guard cells per side along x and y
    int lxh;             // Lx/2 + 1 (half-spectrum columns)
    int pitch;           // complex row pitch of a plane in shared memory (odd)
    int q;               // Ly * lxh: modes per z plane
    AxisPlan ax;         // x: half length h = Lx/2 (complex FFT of packed pairs)
    AxisPlan ay, az;
    int tw_post;         // offset of exp(-2 pi i k/Lx), k = 0..Lx/2, in the pool
    int pad0;
    int64_t field_off;   // element offset of the local box in every field arena
    int64_t spec_off;    // complex offset of this subdomain's spectra block
    int64_t tab_coef;    // element offset of the 7 x (Lz*q) coefficient table
    int64_t tab_k;       // element offset of [k] in position order: x (lxh), y (Ly), z (Lz)
    int64_t tab_ph;      // complex offset of stagger phases (same layout), or -1
    int seg_begin, seg_end;     // exchange segments whose source is this subdomain
    int64_t itemA, itemB, itemC; // first work item of this subdomain in each stage
    int64_t itemA2, itemC1;      // split-plane schedule: first items of the column stages
    int ngz;             // guard cells per side along z (0 for 2D problems)
    int chunkB;          // modes per pass-B chunk (M)
    int lgB;             // log2(M) when M is a power of two, else -1
    int fsB;             // padded stride between fields of a pass-B chunk in shared memory
    int rows;            // split-plane schedule: rows per x-transform item
    int cols;            // split-plane schedule: columns per y-transform item
};

// A box of source valid cells copied into a destination local box.
struct Segment {
    int64_t dst_off;     // field-arena offset of the destination local box
    int dLx, dLy;        // destination local extents x, y
    int src;             // source subdomain
    int dst;             // destination subdomain
    int x0, y0, z0;      // first source local cell
    int ex, ey, ez;      // extents
    int dx, dy, dz;      // destination local = source local + (dx, dy, dz)
    int identity;        // 1 when it is the source's own valid box (dst == src, no shift)
    int vec4;            // 1 when rows can be stored as aligned 4-element vectors
    int64_t item;        // first exchange work item (one per z row of the segment)
};

// Pointers and counts common to every stage launch.
struct LaunchCommon {
    const void* subs; const void* segs; const void* tw; const void* tab; const void* tabc; void* spec;
    void* eb[6]; const void* jr[4]; double* gauss_part;
    unsigned long long* work;   // persistent-launch work counter (in the workspace)
    unsigned int* err;          // device error word (bits PSATD_CHECK_*), in the workspace
    int persistent;             // 1: persistent grids drawing tickets; 0: one CTA per work item
    int nsub, nseg, nf, staggered, own_only;
    int nout;             // output fields written by the inverse stages: 6 (E, B) or 1 (heat: T)
    int64_t per_sub[5];   // items per subdomain of passes A, B, C and of the split schedule's column stages
                          // (forward, inverse) when every subdomain has the same shape, else 0
    int variant;          // index into kFixedF32 / kFixedF64, or -1 for the descriptor-driven kernels
};

// Coefficient table component order (each Lz*q long, position order).
enum { TAB_C = 0, TAB_S, TAB_SK, TAB_OMC, TAB_OMCK, TAB_DK, TAB_INVK, TAB_N };

}  // namespace psatd
