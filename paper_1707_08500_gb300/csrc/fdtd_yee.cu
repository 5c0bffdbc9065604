// Yee FDTD step (Sec. 2, Eqs. 2a/2b of arXiv:1707.08500), the finite-
// difference solver the paper compares PSATD against, as one fused
// HBM-streaming kernel.
//
// Each CTA owns a TX x TY column of cells and marches along z over KZ
// planes.  Shared memory holds a ring of E planes (one-cell halo in x and y),
// the old B of the next plane and J of the next plane (both prefetched), and
// the new B of planes z-1 and z (one-cell halo on the low x and y sides).
// For plane z:
//   1. wait for the copies issued one plane earlier (E(z+1), B(z), J(z));
//   2. issue the copies of E(z+2), B(z+1) and J(z+1) (cp.async: 16-byte
//      pieces along full tile rows, single elements for the halo columns and
//      for tiles that are cut by the grid edge), which land while this plane
//      is computed;
//   3. B^{n+1/2}(z) = B^{n-1/2}(z) - dt curl E(z) on the tile and its low
//      halo (the halo values are recomputed, not written); store the tile;
//   4. E^{n+1}(z) = E^n(z) + dt (curl B^{n+1/2} - J(z)) on the tile; store.
// The first plane of a chunk also needs B at z0-1, recomputed from E at
// z0-1 and z0.  Inputs and outputs are distinct arrays, so CTAs never race.
// Bytes per cell: read E, B, J and write E, B once (15 values); the halo
// re-reads are L2 hits of the neighbouring tiles.
#include <cuda_runtime.h>

#include <cstdint>

#include "psatd.h"
#include "psatd_fdtd.h"

namespace {

constexpr int TX = 32, TY = 8, KZ = 32, NT = TX * TY;
constexpr int EX = TX + 2, EY = TY + 2;      // E tile with a halo on both sides
constexpr int BX = TX + 1, BY = TY + 1;      // B tile with a halo on the low sides
constexpr int NE = EX * EY, NB = BX * BY;
constexpr int PE = (NE + NT - 1) / NT, PB = (NB + NT - 1) / NT;

template <typename T>
struct YeeArgs {
    const T* ein[3];
    const T* bin[3];
    const T* jin[3];
    T* eout[3];
    T* bout[3];
    int nx, ny, nz;
    T dt, rdx, rdy, rdz;   // dt and 1/du
};

// Shared-memory tiles.  Rows are padded so that the first tile column x0
// sits on a 16-byte boundary (column V of a row, V = elements per 16 bytes):
// E-tile column ex (x = x0 - 1 + ex) is stored at ex + V - 1, and the same
// for the B tiles.
template <typename T>
struct Tiles {
    static constexpr int V = 16 / int(sizeof(T));
    static constexpr int EXP = TX + 2 * V, BXP = TX + V, NVR = TX / V;
    T e[3][3][EY][EXP];     // E ring: planes z, z+1 and the prefetched z+2
    T bo[2][3][BY][BXP];    // old B: plane z and the prefetched z+1
    T j[2][3][TY][TX];      // J: plane z and the prefetched z+1
    T b[2][3][BY][BXP];     // new B ring: planes z-1 and z
};

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// global -> shared, asynchronous: one element, or 16 bytes
template <typename T>
__device__ __forceinline__ void cp_elem(unsigned dst, const T* src) {
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" :: "r"(dst), "l"(__cvta_generic_to_global(src)) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" :: "r"(dst), "l"(__cvta_generic_to_global(src)) : "memory");
}
__device__ __forceinline__ void cp_16(unsigned dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" :: "r"(dst), "l"(__cvta_generic_to_global(src)) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ const T* pick(const T* const (&p)[3], int c) {
    return c == 0 ? p[0] : c == 1 ? p[1] : p[2];
}

// One copy of a plane-independent tile piece: shared byte offset within a
// ring slot, global address in plane 0, 16 bytes or one element.
template <typename T>
struct Piece {
    const T* g;
    unsigned s;
    bool vec;
};

// FAST: every tile is full along x and rows are 16-byte aligned
// (Nx % 32 == 0), so tile rows move as 16-byte pieces; otherwise every
// element is copied on its own (any grid).
template <typename T, bool FAST>
__global__ void __launch_bounds__(NT) k_yee(YeeArgs<T> a) {
    using L = Tiles<T>;
    constexpr int V = L::V, NVR = L::NVR;
    // full-tile copies: per component and row, NVR 16-byte pieces plus the
    // single-element halo columns (two for E, one for B)
    constexpr int NIE = 3 * EY * (NVR + 2), NIB = 3 * BY * (NVR + 1), NIJ = 3 * TY * NVR;
    constexpr int KE = (NIE + NT - 1) / NT, KB = (NIB + NT - 1) / NT, KJ = (NIJ + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    L& s = *reinterpret_cast<L*>(smraw);
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * KZ, z1 = min(z0 + KZ, a.nz);
    const int64_t plane = int64_t(a.nx) * a.ny;
    const unsigned base = smem_addr(smraw);
    const unsigned sE = sizeof(s.e[0]), sB = sizeof(s.bo[0]), sJ = sizeof(s.j[0]);
    const unsigned oE = smem_addr(&s.e[0]) - base, oBo = smem_addr(&s.bo[0]) - base, oJ = smem_addr(&s.j[0]) - base;

    // this thread's own cell
    const int tx = t % TX, ty = t / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < a.nx && gy < a.ny;
    const int64_t offO = int64_t(gy) * a.nx + gx;

    Piece<T> pe[FAST ? KE : 1], pb[FAST ? KB : 1], pj[FAST ? KJ : 1];
    int64_t offE[FAST ? 1 : PE], offB[FAST ? 1 : PB];
    int le[FAST ? 1 : PE], lb[FAST ? 1 : PB];
    if constexpr (FAST) {
#pragma unroll
        for (int r = 0; r < KE; ++r) {
            const int i = t + r * NT;
            pe[r].g = nullptr;
            if (i >= NIE) continue;
            const int c = i / (EY * (NVR + 2)), rem = i - c * (EY * (NVR + 2));
            const int ey = rem / (NVR + 2), k = rem - ey * (NVR + 2);
            const int64_t row = int64_t(wrap(y0 - 1 + ey, a.ny)) * a.nx;
            const int col = k < NVR ? V + k * V : k == NVR ? V - 1 : V + TX;
            const int x = k < NVR ? x0 + k * V : k == NVR ? wrap(x0 - 1, a.nx) : wrap(x0 + TX, a.nx);
            pe[r].g = pick(a.ein, c) + row + x;
            pe[r].s = oE + unsigned(((c * EY + ey) * L::EXP + col) * sizeof(T));
            pe[r].vec = k < NVR;
        }
#pragma unroll
        for (int r = 0; r < KB; ++r) {
            const int i = t + r * NT;
            pb[r].g = nullptr;
            if (i >= NIB) continue;
            const int c = i / (BY * (NVR + 1)), rem = i - c * (BY * (NVR + 1));
            const int by = rem / (NVR + 1), k = rem - by * (NVR + 1);
            const int64_t row = int64_t(wrap(y0 - 1 + by, a.ny)) * a.nx;
            const int col = k < NVR ? V + k * V : V - 1;
            const int x = k < NVR ? x0 + k * V : wrap(x0 - 1, a.nx);
            pb[r].g = pick(a.bin, c) + row + x;
            pb[r].s = oBo + unsigned(((c * BY + by) * L::BXP + col) * sizeof(T));
            pb[r].vec = k < NVR;
        }
#pragma unroll
        for (int r = 0; r < KJ; ++r) {
            const int i = t + r * NT;
            pj[r].g = nullptr;
            if (i >= NIJ) continue;
            const int c = i / (TY * NVR), rem = i - c * (TY * NVR);
            const int jy = rem / NVR, k = rem - jy * NVR;
            if (y0 + jy >= a.ny) continue;
            pj[r].g = pick(a.jin, c) + int64_t(y0 + jy) * a.nx + x0 + k * V;
            pj[r].s = oJ + unsigned(((c * TY + jy) * TX + k * V) * sizeof(T));
            pj[r].vec = true;
        }
    } else {
#pragma unroll
        for (int r = 0; r < PE; ++r) {
            const int e = t + r * NT;
            le[r] = e < NE ? e : -1;
            const int ey = e / EX, ex = e - (e / EX) * EX;
            offE[r] = int64_t(wrap(y0 - 1 + ey, a.ny)) * a.nx + wrap(x0 - 1 + ex, a.nx);
        }
#pragma unroll
        for (int r = 0; r < PB; ++r) {
            const int e = t + r * NT;
            lb[r] = e < NB ? e : -1;
            const int by = e / BX, bx = e - (e / BX) * BX;
            offB[r] = int64_t(wrap(y0 - 1 + by, a.ny)) * a.nx + wrap(x0 - 1 + bx, a.nx);
        }
    }

    auto issue = [&](const Piece<T>& q, unsigned slot_base, int64_t zo) {
        if (!q.g) return;
        if (q.vec) cp_16(base + slot_base + q.s, q.g + zo);
        else cp_elem(base + slot_base + q.s, q.g + zo);
    };
    auto issue_e = [&](int z, int slot) {
        const int64_t zo = int64_t(wrap(z, a.nz)) * plane;
        if constexpr (FAST) {
#pragma unroll
            for (int r = 0; r < KE; ++r) issue(pe[r], slot * sE, zo);
        } else {
#pragma unroll
            for (int r = 0; r < PE; ++r) {
                if (le[r] < 0) continue;
                const int ey = le[r] / EX, ex = le[r] - (le[r] / EX) * EX;
#pragma unroll
                for (int c = 0; c < 3; ++c) cp_elem(smem_addr(&s.e[slot][c][ey][ex + V - 1]), a.ein[c] + zo + offE[r]);
            }
        }
    };
    auto issue_b = [&](int z, int slot) {
        const int64_t zo = int64_t(wrap(z, a.nz)) * plane;
        if constexpr (FAST) {
#pragma unroll
            for (int r = 0; r < KB; ++r) issue(pb[r], slot * sB, zo);
        } else {
#pragma unroll
            for (int r = 0; r < PB; ++r) {
                if (lb[r] < 0) continue;
                const int by = lb[r] / BX, bx = lb[r] - (lb[r] / BX) * BX;
#pragma unroll
                for (int c = 0; c < 3; ++c) cp_elem(smem_addr(&s.bo[slot][c][by][bx + V - 1]), a.bin[c] + zo + offB[r]);
            }
        }
    };
    auto issue_j = [&](int z, int slot) {
        const int64_t zo = int64_t(z) * plane;
        if constexpr (FAST) {
#pragma unroll
            for (int r = 0; r < KJ; ++r) issue(pj[r], slot * sJ, zo);
        } else if (own) {
#pragma unroll
            for (int c = 0; c < 3; ++c) cp_elem(smem_addr(&s.j[slot][c][ty][tx]), a.jin[c] + zo + offO);
        }
    };
    // new B at plane z on the tile and its low halo, from E(z) (slot se0),
    // E(z+1) (slot se1) and the old B (slot so) into slot sb; `store`
    // writes the tile cells to the output
    auto push_b = [&](int z, int se0, int se1, int so, int sb, bool store) {
        const int64_t zo = int64_t(wrap(z, a.nz)) * plane;
#pragma unroll
        for (int r = 0; r < PB; ++r) {
            const int e = t + r * NT;
            if (e >= NB) continue;
            const int by = e / BX, bx = e - (e / BX) * BX;
            const int cb = bx + V - 1;               // column of this cell in the E and B tiles
            const T ex0 = s.e[se0][0][by][cb], ey0 = s.e[se0][1][by][cb], ez0 = s.e[se0][2][by][cb];
            const T cx = (s.e[se0][2][by + 1][cb] - ez0) * a.rdy - (s.e[se1][1][by][cb] - ey0) * a.rdz;
            const T cy = (s.e[se1][0][by][cb] - ex0) * a.rdz - (s.e[se0][2][by][cb + 1] - ez0) * a.rdx;
            const T cz = (s.e[se0][1][by][cb + 1] - ey0) * a.rdx - (s.e[se0][0][by + 1][cb] - ex0) * a.rdy;
            const T nbx = s.bo[so][0][by][cb] - a.dt * cx;
            const T nby = s.bo[so][1][by][cb] - a.dt * cy;
            const T nbz = s.bo[so][2][by][cb] - a.dt * cz;
            s.b[sb][0][by][cb] = nbx;
            s.b[sb][1][by][cb] = nby;
            s.b[sb][2][by][cb] = nbz;
            const int x = x0 + bx - 1, y = y0 + by - 1;
            if (store && bx > 0 && by > 0 && x < a.nx && y < a.ny) {
                const int64_t o = zo + int64_t(y) * a.nx + x;
                a.bout[0][o] = nbx;
                a.bout[1][o] = nby;
                a.bout[2][o] = nbz;
            }
        }
    };

    // prologue: E at z0-1 and z0 and old B at z0-1 give the new B at z0-1
    // (not stored: it belongs to the chunk below); then prefetch plane z0
    issue_e(z0 - 1, 0);
    issue_e(z0, 1);
    issue_b(z0 - 1, 0);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    push_b(z0 - 1, 0, 1, 0, 0, false);
    issue_e(z0 + 1, 2);
    issue_b(z0, 1);
    issue_j(z0, 0);
    cp_commit();
    int e0 = 1, e1 = 2, e2 = 0;   // E ring slots of planes z, z+1, z+2
    int sl = 1;                   // slot of old B(z) and new B(z); J(z) is in slot sl ^ 1
    for (int z = z0; z < z1; ++z) {
        cp_wait_all();
        __syncthreads();          // E(z+1), B(z), J(z) landed; plane z-1 fully done
        if (z + 1 < z1) {
            issue_e(z + 2, e2);
            issue_b(z + 1, sl ^ 1);
            issue_j(z + 1, sl);
        }
        cp_commit();
        push_b(z, e0, e1, sl, sl, true);
        __syncthreads();
        if (own) {
            const int64_t o = int64_t(z) * plane + offO;
            const int ly = ty + 1, lc = tx + V;      // B/E-tile row and column of the cell
            const auto& b1 = s.b[sl];                // B(z)
            const auto& b0 = s.b[sl ^ 1];            // B(z-1)
            const auto& jj = s.j[sl ^ 1];            // J(z)
            const T cx = (b1[2][ly][lc] - b1[2][ly - 1][lc]) * a.rdy - (b1[1][ly][lc] - b0[1][ly][lc]) * a.rdz;
            const T cy = (b1[0][ly][lc] - b0[0][ly][lc]) * a.rdz - (b1[2][ly][lc] - b1[2][ly][lc - 1]) * a.rdx;
            const T cz = (b1[1][ly][lc] - b1[1][ly][lc - 1]) * a.rdx - (b1[0][ly][lc] - b1[0][ly - 1][lc]) * a.rdy;
            a.eout[0][o] = s.e[e0][0][ly][lc] + a.dt * (cx - jj[0][ty][tx]);
            a.eout[1][o] = s.e[e0][1][ly][lc] + a.dt * (cy - jj[1][ty][tx]);
            a.eout[2][o] = s.e[e0][2][ly][lc] + a.dt * (cz - jj[2][ty][tx]);
        }
        const int r = e0;
        e0 = e1; e1 = e2; e2 = r;
        sl ^= 1;
    }
    cp_wait_all();
}

bool overlaps(const void* a, const void* b, size_t n) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + n && y < x + n;
}

template <typename T>
int launch(const int32_t n[3], double c_dt, const double dx[3], const psatd_fields* in, const psatd_fields* out,
           cudaStream_t st) {
    YeeArgs<T> a;
    for (int c = 0; c < 3; ++c) {
        a.ein[c] = static_cast<const T*>(in->E[c]);
        a.bin[c] = static_cast<const T*>(in->B[c]);
        a.jin[c] = static_cast<const T*>(in->J[c]);
        a.eout[c] = static_cast<T*>(out->E[c]);
        a.bout[c] = static_cast<T*>(out->B[c]);
    }
    a.nx = n[0]; a.ny = n[1]; a.nz = n[2];
    a.dt = T(c_dt);
    a.rdx = T(1.0 / dx[0]); a.rdy = T(1.0 / dx[1]); a.rdz = T(1.0 / dx[2]);
    const dim3 grid((n[0] + TX - 1) / TX, (n[1] + TY - 1) / TY, (n[2] + KZ - 1) / KZ);
    const int smem = int(sizeof(Tiles<T>));
    const bool fast = n[0] % TX == 0;
    auto k = fast ? k_yee<T, true> : k_yee<T, false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return PSATD_E_CUDA;
    k<<<grid, NT, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? PSATD_OK : PSATD_E_CUDA;
}

}  // namespace

extern "C" {

int psatd_yee_step(const int32_t global_n[3], int32_t flags, double c_dt, const double dx[3],
                   const psatd_fields* in, const psatd_fields* out, void* stream) {
    if (!global_n || !dx || !in || !out) return PSATD_E_ARG;
    const int prec = flags & (PSATD_F32 | PSATD_F64);
    if ((flags & ~(PSATD_F32 | PSATD_F64)) || (prec != PSATD_F32 && prec != PSATD_F64)) return PSATD_E_ARG;
    if (!(c_dt == c_dt) || c_dt > 1e300 || c_dt < -1e300) return PSATD_E_ARG;
    for (int c = 0; c < 3; ++c)
        if (!(dx[c] > 0) || dx[c] > 1e300) return PSATD_E_ARG;
    int64_t cells = 1;
    for (int c = 0; c < 3; ++c) {
        if (global_n[c] < 1) return PSATD_E_SHAPE;
        cells *= global_n[c];
        if (cells > (int64_t(1) << 31)) return PSATD_E_SHAPE;
    }
    if ((global_n[1] + TY - 1) / TY > 65535 || (global_n[2] + KZ - 1) / KZ > 65535) return PSATD_E_SHAPE;
    const size_t bytes = size_t(cells) * (prec == PSATD_F32 ? 4 : 8);
    const void* ins[9];
    const void* outs[6];
    for (int c = 0; c < 3; ++c) {
        ins[c] = in->E[c]; ins[3 + c] = in->B[c]; ins[6 + c] = in->J[c];
        outs[c] = out->E[c]; outs[3 + c] = out->B[c];
    }
    for (const void* p : ins)
        if (!p || reinterpret_cast<uintptr_t>(p) % 16) return PSATD_E_ARG;
    for (int i = 0; i < 6; ++i) {
        if (!outs[i] || reinterpret_cast<uintptr_t>(outs[i]) % 16) return PSATD_E_ARG;
        for (const void* p : ins)
            if (overlaps(outs[i], p, bytes)) return PSATD_E_ARG;
        for (int j = 0; j < i; ++j)
            if (overlaps(outs[i], outs[j], bytes)) return PSATD_E_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return prec == PSATD_F32 ? launch<float>(global_n, c_dt, dx, in, out, st)
                             : launch<double>(global_n, c_dt, dx, in, out, st);
}

int psatd_yee_launches(int32_t* launches) {
    if (!launches) return PSATD_E_ARG;
    *launches = 1;
    return PSATD_OK;
}

}  // extern "C"
