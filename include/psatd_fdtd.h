/* C ABI of the Yee FDTD Maxwell step, the finite-difference solver that
 * arXiv:1707.08500 compares PSATD against (Sec. 2, Eqs. 2a/2b).  Part of
 * libpsatd.so; shares the status codes, precision flags and psatd_fields of
 * psatd.h.
 *
 * Scheme (c = eps0 = 1).  Yee mesh: Ex at (i+1/2, j, k), Ey at (i, j+1/2, k),
 * Ez at (i, j, k+1/2), Bx at (i, j+1/2, k+1/2), By at (i+1/2, j, k+1/2),
 * Bz at (i+1/2, j+1/2, k); J on the E positions.  One step advances the
 * state (E^n, B^{n-1/2}) with J^{n+1/2}:
 *     B^{n+1/2} = B^{n-1/2} - dt curl E^n                     (Eq. 2a)
 *     E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2})       (Eq. 2b)
 * with one-cell centred differences D_x, D_y, D_z on a periodic grid.
 * Stability needs c dt <= 1/sqrt(1/dx^2 + 1/dy^2 + 1/dz^2); not checked.
 */
#ifndef PSATD_FDTD_H
#define PSATD_FDTD_H

#include <stdint.h>

#include "psatd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One Yee step on the periodic global grid global_n = (Nx, Ny, Nz), every
 * extent >= 1 (Nz = 1: a 2D problem).
 *
 * flags: exactly one of PSATD_F32 / PSATD_F64; any other bit is rejected.
 * c_dt: c dt (finite); dx: cell sizes (x, y, z), each > 0.
 * in:  E^n, B^{n-1/2}, J^{n+1/2} (rho is ignored);
 * out: E^{n+1}, B^{n+1/2} (out->J and out->rho are ignored).
 * Every array is a dense device array [Nz][Ny][Nx] of float (PSATD_F32) or
 * double (PSATD_F64), 16-byte aligned, owned by the caller.  No out array may
 * overlap another out array or any in array (checked on the address ranges:
 * PSATD_E_ARG); ping-pong two field sets across steps.
 *
 * Enqueued on `stream` (a cudaStream_t; NULL = legacy default stream);
 * returns before the step runs.  Allocates nothing.  Returns PSATD_OK,
 * PSATD_E_ARG (null or misaligned pointer, bad flags, overlap, bad c_dt/dx),
 * PSATD_E_SHAPE (an extent < 1, a grid above 2^31 cells, Ny > 524280 or
 * Nz > 2097120) or PSATD_E_CUDA
 * (launch failure). */
int psatd_yee_step(const int32_t global_n[3], int32_t flags, double c_dt, const double dx[3],
                   const psatd_fields* in, const psatd_fields* out, void* stream);

/* Kernel launches one psatd_yee_step enqueues (1). */
int psatd_yee_launches(int32_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* PSATD_FDTD_H */
