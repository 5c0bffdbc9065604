"""Plain FP64 CPU oracle of the local-FFT PSATD Maxwell push.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
product path never imports, links or calls it.  It shares no code with the CUDA
path: the only common module is the seeded input generator, which holds none
of the method's arithmetic.

What it computes (Vincenti & Vay, arXiv:1707.08500):

* Sec. 3.1, Eq. 1a/1b -- the PSATD update of E and B per Fourier mode, with
  C = cos(k dt), S = sin(k dt), J taken at n+1/2, in c = eps0 = 1 units;
* Sec. 3.1 (text after Eq. 1) -- the order-p substitution of each wavenumber
  component k_u by sum_{j=1}^{p/2} w_j sin(j k_u du)/(du/2);
* Sec. 3.2, Fig. 2a, Fig. 3 steps 1-3 -- the domain is cut into subdomains
  padded with guard cells; each subdomain is advanced with local FFTs over its
  padded box; the spurious guard values are then replaced by the valid values
  of the subdomain that owns those cells.

Readings where the paper is silent (each is listed with its reason in the
design notes of the repository):

* the FD weights w_j are the centred Fornberg weights of
  f' ~ sum_j w_j (f_{+j} - f_{-j}) / du (nodal), and the staggered variant uses
  f' ~ sum_j c_j (f_{+(j-1/2)} - f_{-(j-1/2)}) / du;
* p = 0 denotes the infinite-order limit (exact k);
* on an even axis the Nyquist index L/2 carries k = -pi/du and its modified
  wavenumber is set to zero for every order, so every self-conjugate mode has
  |[k]| = 0 and the update maps Hermitian spectra to Hermitian spectra;
* at k = 0 the limits are taken: S/k -> dt, (1-C)/k -> 0, S/k - dt -> 0 and the
  khat terms vanish, so E' = E - dt J and B' = B;
* the padded local box is the DFT period; forward transforms are unnormalised,
  inverses carry 1/(Lx Ly Lz); a C2R transform ignores the imaginary part of the
  kx = 0 and kx = Lx/2 columns, as any real inverse FFT does;
* staggered fields (not in the paper) are phase-shifted by exp(-i k.s) with the
  exact k into nodal position before Eq. 1 and shifted back after it;
* the guard exchange is defined by global index modulo the periodic global
  grid: the owner's valid value wins (edges, corners and periodic wrap).

Parity pins: FD weights against exact rational moment solutions; the FFT
wrapper against a brute-force DFT; the per-mode update against the matrix
exponential of the Maxwell ODE with constant J; real-space plane waves against
the closed-form solution (dispersion); energy and Gauss invariants; the two
Gauss-diagnostic sums against N times real-space sums of (div_p E' - rho)^2 and
rho^2 (an order-p stencil evaluated without transforms, and Parseval); local
equals global when the padded box is one global period; guard-truncation error
decreasing with the guard count.  The magnitude of the guard-truncation error
is parity unpinned (its model is in another paper).
"""
from __future__ import annotations

import math
import os
from fractions import Fraction  # noqa: F401  (documented in the pins)
from typing import Dict, List, Sequence, Tuple

import numpy as np
import scipy.fft as sfft

EB = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
STAGGER = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Bx": (0.0, 0.5, 0.5), "By": (0.5, 0.0, 0.5), "Bz": (0.5, 0.5, 0.0),
    "Jx": (0.5, 0.0, 0.0), "Jy": (0.0, 0.5, 0.0), "Jz": (0.0, 0.0, 0.5),
    "rho": (0.0, 0.0, 0.0),
}


def _workers() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


WORKERS = _workers()


# ---------------------------------------------------------------------------
# Sec. 3.1: order-p modified wavenumber
# ---------------------------------------------------------------------------
def fd_weights_nodal(p: int) -> np.ndarray:
    """w_1..w_{p/2} of the centred order-p first derivative on a nodal grid,
    f'(x) ~ sum_j w_j (f(x+j du) - f(x-j du)) / du.

    Closed form w_j = (-1)^{j+1} (m!)^2 / (j (m-j)! (m+j)!), m = p/2, evaluated
    by the ratio of consecutive terms so that large p does not overflow."""
    assert p >= 2 and p % 2 == 0
    m = p // 2
    w = np.empty(m)
    w[0] = m / (m + 1.0)
    for j in range(1, m):
        w[j] = -w[j - 1] * j * (m - j) / ((j + 1.0) * (m + j + 1.0))
    return w


def fd_weights_staggered(p: int) -> np.ndarray:
    """c_1..c_{p/2} of the order-p staggered first derivative,
    f'(x) ~ sum_j c_j (f(x+(j-1/2) du) - f(x-(j-1/2) du)) / du.

    Closed form c_j = (-1)^{j+1} ((2m-1)!!)^2 / ((2j-1)^2 (m-j)! (m+j-1)! 4^{m-1}),
    evaluated by the ratio c_{j+1}/c_j = -(2j-1)^2 (m-j) / ((2j+1)^2 (m+j))."""
    assert p >= 2 and p % 2 == 0
    m = p // 2
    # log c_1 = 2 log((2m-1)!!) - log((m-1)!) - log(m!) - (m-1) log 4
    log_dfact = sum(math.log(2 * i - 1) for i in range(1, m + 1))
    logc1 = 2 * log_dfact - math.lgamma(m) - math.lgamma(m + 1) - (m - 1) * math.log(4.0)
    c = np.empty(m)
    c[0] = math.exp(logc1)
    for j in range(1, m):
        c[j] = -c[j - 1] * (2 * j - 1) ** 2 * (m - j) / ((2 * j + 1) ** 2 * (m + j))
    return c


def k_exact(L: int, du: float) -> np.ndarray:
    """Exact wavenumbers of the L-point DFT in FFT order; index L/2 of an even
    axis carries -pi/du."""
    n = np.arange(L)
    n = np.where(n < (L + 1) // 2, n, n - L)
    return 2.0 * math.pi * n / (L * du)


def modified_k(L: int, du: float, p: int, staggered: bool) -> np.ndarray:
    """[k]_u for every index of an L-point axis (FFT order), Sec. 3.1.

    nodal:     [k] = sum_j w_j sin(j k du) / (du/2)
    staggered: [k] = sum_j c_j 2 sin((2j-1) k du/2) / du
    p == 0:    [k] = k (infinite order)
    The Nyquist index of an even axis is set to 0 for every order."""
    k = k_exact(L, du)
    if p == 0:
        km = k.copy()
    elif not staggered:
        w = fd_weights_nodal(p)
        km = np.zeros(L)
        for j in range(1, len(w) + 1):
            km += w[j - 1] * np.sin(j * k * du) / (du / 2.0)
    else:
        c = fd_weights_staggered(p)
        km = np.zeros(L)
        for j in range(1, len(c) + 1):
            km += c[j - 1] * 2.0 * np.sin((2 * j - 1) * k * du / 2.0) / du
    if L % 2 == 0:
        km[L // 2] = 0.0
    return km


# ---------------------------------------------------------------------------
# Sec. 3.1, Eq. 1a/1b: the per-mode PSATD update
# ---------------------------------------------------------------------------
def eq1_coefficients(kmag: np.ndarray, dt: float) -> Dict[str, np.ndarray]:
    """C, S, S/k, 1-C, (1-C)/k, S/k - dt for |[k]| = kmag (k = 0 by limits)."""
    x = kmag * dt
    C = np.cos(x)
    S = np.sin(x)
    omc = 2.0 * np.sin(x / 2.0) ** 2                    # 1 - C without cancellation
    nz = kmag > 0
    safe = np.where(nz, kmag, 1.0)
    S_k = np.where(nz, S / safe, dt)
    omc_k = np.where(nz, omc / safe, 0.0)
    small = x < 1e-3
    xs = np.where(small, x, 0.0)
    series = dt * (-xs ** 2 / 6.0 + xs ** 4 / 120.0)   # dt (sin x / x - 1)
    dk = np.where(small, series, S_k - dt)
    return {"C": C, "S": S, "S_k": S_k, "omC": omc, "omC_k": omc_k, "Sk_dt": dk}


def eq1_update(E, B, J, kvec, dt):
    """Eq. 1a/1b on arrays of modes.

    E, B, J: tuples of three complex arrays (field spectra at n, n, n+1/2);
    kvec: tuple of three real arrays, the (modified) wavenumber components.
    Returns (E', B')."""
    kx, ky, kz = kvec
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    co = eq1_coefficients(kmag, dt)
    inv = np.where(kmag > 0, 1.0 / np.where(kmag > 0, kmag, 1.0), 0.0)
    h = (kx * inv, ky * inv, kz * inv)                  # khat (0 at k = 0)

    def cross(a, b):
        return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])

    def dot(a, b):
        return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]

    hxB, hxE, hxJ = cross(h, B), cross(h, E), cross(h, J)
    hE, hJ = dot(h, E), dot(h, J)
    E1 = tuple(co["C"] * E[a] + 1j * co["S"] * hxB[a] - co["S_k"] * J[a]
               + co["omC"] * h[a] * hE + h[a] * hJ * co["Sk_dt"] for a in range(3))
    B1 = tuple(co["C"] * B[a] - 1j * co["S"] * hxE[a] + 1j * co["omC_k"] * hxJ[a]
               for a in range(3))
    return E1, B1


# ---------------------------------------------------------------------------
# local FFTs over a padded box (Sec. 3.2)
# ---------------------------------------------------------------------------
def r2c(f: np.ndarray) -> np.ndarray:
    """Unnormalised forward real FFT of an [Lz][Ly][Lx] array -> [Lz][Ly][Lx/2+1]."""
    return sfft.rfftn(f, axes=(0, 1, 2), workers=WORKERS)


def c2r(F: np.ndarray, shape) -> np.ndarray:
    """Inverse of r2c with 1/(Lx Ly Lz), shape = (Lz, Ly, Lx)."""
    return sfft.irfftn(F, s=shape, axes=(0, 1, 2), workers=WORKERS)


def brute_dft3(f: np.ndarray) -> np.ndarray:
    """Direct triple sum F[kz,ky,kx] = sum_{z,y,x} f e^{-2 pi i (kz z/Lz + ky y/Ly + kx x/Lx)}
    for tiny grids (O(N^2) in the number of cells)."""
    Lz, Ly, Lx = f.shape
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    out = np.empty((Lz, Ly, Lx), dtype=complex)
    for kz in range(Lz):
        for ky in range(Ly):
            for kx in range(Lx):
                ph = -2j * math.pi * (kz * z / Lz + ky * y / Ly + kx * x / Lx)
                out[kz, ky, kx] = np.sum(f * np.exp(ph))
    return out


def local_kvectors(L: Sequence[int], dx: Sequence[float], p: int, staggered: bool):
    """Broadcastable modified and exact wavenumber arrays on the half spectrum."""
    Lx, Ly, Lz = L
    kmx = modified_k(Lx, dx[0], p, staggered)[: Lx // 2 + 1]
    kex = k_exact(Lx, dx[0])[: Lx // 2 + 1]
    kmod = (kmx[None, None, :], modified_k(Ly, dx[1], p, staggered)[None, :, None],
            modified_k(Lz, dx[2], p, staggered)[:, None, None])
    kex3 = (kex[None, None, :], k_exact(Ly, dx[1])[None, :, None], k_exact(Lz, dx[2])[:, None, None])
    return kmod, kex3


def _phase(name, kex, dx):
    s = STAGGER[name]
    return np.exp(-1j * (kex[0] * s[0] * dx[0] + kex[1] * s[1] * dx[1] + kex[2] * s[2] * dx[2]))


def half_weights(Lx: int) -> np.ndarray:
    """Multiplicity of each kx column of a half spectrum in the full spectrum."""
    w = np.full(Lx // 2 + 1, 2.0)
    w[0] = 1.0
    if Lx % 2 == 0:
        w[-1] = 1.0
    return w


def local_push(fields: Dict[str, np.ndarray], L, dx, p: int, c_dt: float, staggered: bool):
    """One PSATD push of one padded local box (Sec. 3.2 with Eq. 1).

    fields: the ten local arrays [Lz][Ly][Lx] (E, B at n; J at n+1/2; rho at n+1).
    Returns (E', B' on the whole padded box, (gauss_res2, rho2)) where
    gauss_res2 = sum over all modes of |i [k].E' - rho~|^2 and rho2 = sum |rho~|^2
    (full-spectrum sums, E' in nodal position), both on unnormalised spectra."""
    Lx, Ly, Lz = L
    kmod, kex = local_kvectors(L, dx, p, staggered)
    spec = {}
    for n in EB + ("Jx", "Jy", "Jz"):
        F = r2c(fields[n])
        if staggered:
            F = F * _phase(n, kex, dx)
        spec[n] = F
    E1, B1 = eq1_update(tuple(spec[n] for n in EB[:3]), tuple(spec[n] for n in EB[3:]),
                        tuple(spec[n] for n in ("Jx", "Jy", "Jz")), kmod, c_dt)
    rho = r2c(fields["rho"])
    res = 1j * (kmod[0] * E1[0] + kmod[1] * E1[1] + kmod[2] * E1[2]) - rho
    w = half_weights(Lx)[None, None, :]
    gauss = (float(np.sum(w * np.abs(res) ** 2)), float(np.sum(w * np.abs(rho) ** 2)))
    out = {}
    for n, F in zip(EB, E1 + B1):
        if staggered:
            F = F / _phase(n, kex, dx)
        out[n] = c2r(F, (Lz, Ly, Lx))
    return out, gauss


# ---------------------------------------------------------------------------
# decomposition, guard extraction and exchange (Sec. 3.2, Fig. 3)
# ---------------------------------------------------------------------------
def _guards(ng):
    """Guard widths (x, y, z) from an int or a 3-tuple."""
    return tuple(ng) if isinstance(ng, (tuple, list)) else (ng, ng, ng)


def sub_guards(sd):
    """Guard widths (x, y, z) of a subdomain (none along z in 2D problems)."""
    return tuple(getattr(sd, "guards", (sd.ng, sd.ng, sd.ng)))


def extract_box(G: np.ndarray, lo, L, ng) -> np.ndarray:
    """Padded box of a subdomain read from the periodic global array by global
    index modulo the grid (this is also the guard exchange: every local cell
    holds the owner's valid value).  ng: guard width, or (gx, gy, gz)."""
    Nz, Ny, Nx = G.shape
    gx, gy, gz = _guards(ng)
    ix = (np.arange(L[0]) + lo[0] - gx) % Nx
    iy = (np.arange(L[1]) + lo[1] - gy) % Ny
    iz = (np.arange(L[2]) + lo[2] - gz) % Nz
    return G[np.ix_(iz, iy, ix)]


def owner_map(global_n, subs) -> np.ndarray:
    """Index of the subdomain owning each global cell; asserts an exact tiling."""
    Nx, Ny, Nz = global_n
    own = np.full((Nz, Ny, Nx), -1, dtype=np.int64)
    for s, sd in enumerate(subs):
        (x0, y0, z0), (nx, ny, nz) = sd.lo, sd.n
        blk = own[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx]
        assert blk.shape == (nz, ny, nx) and np.all(blk == -1), "subdomains overlap or leave the grid"
        blk[...] = s
    assert np.all(own >= 0), "subdomains do not cover the grid"
    return own


def step(glob: Dict[str, np.ndarray], wl, gauss_out: List | None = None) -> Dict[str, np.ndarray]:
    """One step of the local-FFT method on the whole grid.

    For each subdomain: extract the padded box from the global valid field,
    push it, keep its valid cells.  The next extraction then refills every guard
    from its owner, which is the exchange of Fig. 3 step 3."""
    new = {n: np.empty_like(glob[n]) for n in EB}
    for sd in wl.subs:
        L = sd.local
        gx, gy, gz = sub_guards(sd)
        loc = {n: extract_box(glob[n], sd.lo, L, (gx, gy, gz)) for n in glob}
        out, gauss = local_push(loc, L, wl.dx, sd.p, wl.c_dt, wl.staggered)
        if gauss_out is not None:
            gauss_out.append(gauss)
        (x0, y0, z0), (nx, ny, nz) = sd.lo, sd.n
        for n in EB:
            new[n][z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] = out[n][gz:gz + nz, gy:gy + ny, gx:gx + nx]
    for n in glob:
        if n not in new:
            new[n] = glob[n]
    return new


def run(glob: Dict[str, np.ndarray], wl, steps: int) -> Dict[str, np.ndarray]:
    for _ in range(steps):
        glob = step(glob, wl)
    return glob


def local_arena(glob: Dict[str, np.ndarray], wl, name: str) -> List[np.ndarray]:
    """Padded boxes of every subdomain for one field (guards from the owners)."""
    return [extract_box(glob[name], sd.lo, sd.local, sub_guards(sd)) for sd in wl.subs]


def global_push(glob: Dict[str, np.ndarray], p: int, dx, c_dt: float, staggered: bool):
    """PSATD on the whole periodic grid with one global FFT (the comparison
    system of Sec. 3.2 / Fig. 2b); returns E', B'."""
    Nz, Ny, Nx = glob["Ex"].shape
    out, _ = local_push(glob, (Nx, Ny, Nz), dx, p, c_dt, staggered)
    return out


# ---------------------------------------------------------------------------
# error metric and invariants
# ---------------------------------------------------------------------------
def rel_l2(a: Dict[str, np.ndarray], b: Dict[str, np.ndarray], names=EB) -> float:
    """||a - b||_2 / ||b||_2 over the listed components stacked."""
    num = sum(float(np.sum((np.asarray(a[n], dtype=np.float64) - b[n]) ** 2)) for n in names)
    den = sum(float(np.sum(np.asarray(b[n], dtype=np.float64) ** 2)) for n in names)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


def energy(glob: Dict[str, np.ndarray]) -> float:
    return 0.5 * sum(float(np.sum(glob[n] ** 2)) for n in EB)


def spectral_divergence(fx, fy, fz, dx, p, staggered=False, names=("Ex", "Ey", "Ez")):
    """i [k].F~ on the half spectrum of a single periodic box (F in nodal position)."""
    Nz, Ny, Nx = fx.shape
    kmod, kex = local_kvectors((Nx, Ny, Nz), dx, p, staggered)
    acc = 0
    for a, (n, f) in enumerate(zip(names, (fx, fy, fz))):
        F = r2c(f)
        if staggered:
            F = F * _phase(n, kex, dx)
        acc = acc + 1j * kmod[a] * F
    return acc
