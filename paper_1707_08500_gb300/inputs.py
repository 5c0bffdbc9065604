"""Seeded synthetic workloads for the local-FFT PSATD push.

This module only *describes* workloads (grid, decomposition, order p, time
step) and *synthesises* the initial fields.  It contains none of the solver's
arithmetic: no modified wavenumber, no Eq. 1 coefficient, no local FFT.  Both
the CUDA path's harness and the FP64 oracle read their inputs from here.

Random draws use a counter-based generator (the ``lowbias32`` integer hash
published by C. Wellons, 2018) keyed by (seed, stream, global cell index), so
that any sub-box of any field can be evaluated on any device with bit-identical
results.  All arithmetic of the hash is done in int64 with 16-bit split
multiplies so that no intermediate overflows.

Conventions shared by everything in this repository:

* global arrays are shaped ``[Nz][Ny][Nx]`` (x fastest); sizes and subdomain
  corners are given as (x, y, z) tuples;
* units are c = 1, eps0 = 1 (the paper's form of Ampere's law, Sec. 2 Eq. 2b);
* field order is Ex, Ey, Ez, Bx, By, Bz, Jx, Jy, Jz, rho.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import torch

FIELD_NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz", "rho")
EB_NAMES = FIELD_NAMES[:6]

# Spatial stagger of each component, in cells along (x, y, z), used when a
# workload is Yee-staggered.  E and J sit on cell edges, B on cell faces, rho
# on nodes.
STAGGER = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Bx": (0.0, 0.5, 0.5), "By": (0.5, 0.0, 0.5), "Bz": (0.5, 0.5, 0.0),
    "Jx": (0.5, 0.0, 0.0), "Jy": (0.0, 0.5, 0.0), "Jz": (0.0, 0.0, 0.5),
    "rho": (0.0, 0.0, 0.0),
}


@dataclasses.dataclass(frozen=True)
class Sub:
    """One subdomain: valid box [lo, lo+n) of the global grid, padded by ng
    guard cells on every side (none along z when zguard is False, as in 2D
    problems), solved at stencil order p (0 = infinite)."""
    lo: Tuple[int, int, int]
    n: Tuple[int, int, int]
    ng: int
    p: int
    zguard: bool = True

    @property
    def guards(self) -> Tuple[int, int, int]:
        return (self.ng, self.ng, self.ng if self.zguard else 0)

    @property
    def local(self) -> Tuple[int, int, int]:
        return tuple(int(v) + 2 * g for v, g in zip(self.n, self.guards))


@dataclasses.dataclass
class Workload:
    name: str
    global_n: Tuple[int, int, int]
    subs: List[Sub]
    fields: str                      # "wavepacket" | "broadband" | "laser_slab"
    steps: int
    precision: str                   # "f64" | "f32"
    seed: int
    dx: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    c_dt: float = 0.5
    staggered: bool = False
    two_d: bool = False

    @property
    def valid_cells(self) -> int:
        return int(self.global_n[0]) * int(self.global_n[1]) * int(self.global_n[2])

    @property
    def local_cells(self) -> int:
        return sum(s.local[0] * s.local[1] * s.local[2] for s in self.subs)


# ---------------------------------------------------------------------------
# counter-based uniform generator
# ---------------------------------------------------------------------------
_M32 = 0xFFFFFFFF


def _mul32(x: torch.Tensor, m: int) -> torch.Tensor:
    """(x * m) mod 2^32 for 0 <= x, m < 2^32, without int64 overflow."""
    mh, ml = m >> 16, m & 0xFFFF
    return ((x * ml) + (((x * mh) & 0xFFFF) << 16)) & _M32


def lowbias32(x: torch.Tensor) -> torch.Tensor:
    x = x & _M32
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    x = x ^ (x >> 16)
    return x


def _key(seed: int, stream: int) -> int:
    t = torch.tensor([(seed * 1000003 + stream * 7919 + 12345) & _M32], dtype=torch.int64)
    return int(lowbias32(lowbias32(t))[0])


def uniform(seed: int, stream: int, index: torch.Tensor) -> torch.Tensor:
    """U[0,1) with 24 random bits (exact in FP32 and FP64) for each int64 index."""
    k = _key(seed, stream)
    h = lowbias32((index + k) & _M32)
    h = lowbias32(h ^ ((k * 3) & _M32))
    return (h >> 8).to(torch.float64) * (1.0 / 16777216.0)


def _global_index(global_n, lo, shape, device) -> torch.Tensor:
    """Linear global index (z*Ny + y)*Nx + x of the box [lo, lo+shape), periodic."""
    nx, ny, nz = (int(v) for v in global_n)
    x = (torch.arange(shape[0], device=device, dtype=torch.int64) + lo[0]) % nx
    y = (torch.arange(shape[1], device=device, dtype=torch.int64) + lo[1]) % ny
    z = (torch.arange(shape[2], device=device, dtype=torch.int64) + lo[2]) % nz
    return (z[:, None, None] * ny + y[None, :, None]) * nx + x[None, None, :]


# ---------------------------------------------------------------------------
# decompositions
# ---------------------------------------------------------------------------
def tensor_decomposition(cuts_x: Sequence[int], cuts_y: Sequence[int], cuts_z: Sequence[int],
                         ng, p) -> List[Sub]:
    """Cartesian product of per-axis cuts; subdomain index runs x fastest.
    ``ng`` and ``p`` are ints or callables (ix, iy, iz) -> int."""
    subs = []
    oz = 0
    for iz, wz in enumerate(cuts_z):
        oy = 0
        for iy, wy in enumerate(cuts_y):
            ox = 0
            for ix, wx in enumerate(cuts_x):
                g = ng(ix, iy, iz) if callable(ng) else ng
                pp = p(ix, iy, iz) if callable(p) else p
                subs.append(Sub((ox, oy, oz), (wx, wy, wz), int(g), int(pp)))
                ox += wx
            oy += wy
        oz += wz
    return subs


def _seeded_permutation(values: Sequence[int], seed: int, stream: int) -> List[int]:
    u = uniform(seed, stream, torch.arange(len(values), dtype=torch.int64))
    order = torch.argsort(u, stable=True).tolist()
    return [values[i] for i in order]


# ---------------------------------------------------------------------------
# the five workloads (and scaled-down variants for tests)
# ---------------------------------------------------------------------------
def workload(name: str) -> Workload:
    """Workloads named after what they are.

    plain32      : 32^3 periodic, 1 subdomain, no guards, p=inf, FP64, 100 steps
    yee64        : 64^3 periodic, 2x2x2 x 32^3, ng=8, p=32 staggered, FP64, 200 steps
    broadband256 : 256^3, 4x4x4 x 64^3, ng=16, p=64, FP32, 100 steps
    uneven48     : 192x144x192, 48 uneven subdomains, ng in {8,16}, p in {16,32,64}, FP32, 50 steps
    mirror1024   : 1024x512x512, 16x8x8 x 64^3, ng=16, p=100, FP32, 100 steps (plasma-mirror shaped)
    global256    : broadband256 as one 256^3 box without guards (the global solver), FP32
    broadband2d  : 4096^2 (2D), 64x64 x 64^2, ng=16, p=64, FP32
    """
    if name == "plain32":
        return Workload(name, (32, 32, 32), tensor_decomposition([32], [32], [32], 0, 0),
                        "wavepacket", 100, "f64", 1707 + 1)
    if name == "yee64":
        return Workload(name, (64, 64, 64), tensor_decomposition([32] * 2, [32] * 2, [32] * 2, 8, 32),
                        "wavepacket", 200, "f64", 1707 + 2, staggered=True)
    if name == "broadband256":
        return Workload(name, (256, 256, 256), tensor_decomposition([64] * 4, [64] * 4, [64] * 4, 16, 64),
                        "broadband", 100, "f32", 1707 + 3)
    if name == "uneven48":
        seed = 1707 + 4
        cx = _seeded_permutation([24, 40, 56, 72], seed, 101)
        cy = _seeded_permutation([32, 48, 64], seed, 102)
        cz = _seeded_permutation([32, 48, 48, 64], seed, 103)

        def draw(stream, choices):
            def f(ix, iy, iz):
                u = uniform(seed, stream, torch.tensor([(iz * 3 + iy) * 4 + ix]))
                return choices[min(int(float(u[0]) * len(choices)), len(choices) - 1)]
            return f
        subs = tensor_decomposition(cx, cy, cz, draw(104, [8, 16]), draw(105, [16, 32, 64]))
        return Workload(name, (sum(cx), sum(cy), sum(cz)), subs, "broadband", 50, "f32", seed)
    if name == "mirror1024":
        return Workload(name, (1024, 512, 512),
                        tensor_decomposition([64] * 16, [64] * 8, [64] * 8, 16, 100),
                        "laser_slab", 100, "f32", 1707 + 5)
    if name == "global256":
        # broadband256's grid and fields as one box without guards: the global
        # solver (Fig. 2b) on one GPU
        return Workload(name, (256, 256, 256), [Sub((0, 0, 0), (256, 256, 256), 0, 64)],
                        "broadband", 100, "f32", 1707 + 3)
    if name == "broadband2d":
        # a 2D problem: 4096^2 cells in 64 x 64 subdomains of 64^2, 16 guards
        subs = [dataclasses.replace(sd, zguard=False)
                for sd in tensor_decomposition([64] * 64, [64] * 64, [1], 16, 64)]
        return Workload(name, (4096, 4096, 1), subs, "broadband", 100, "f32", 1707 + 6, two_d=True)
    raise KeyError(name)


WORKLOADS = ("plain32", "yee64", "broadband256", "uneven48", "mirror1024")
EXTRA_WORKLOADS = ("global256", "broadband2d")     # the global solver and a 2D problem


def custom(name, global_n, cuts, ng, p, fields="broadband", steps=1, precision="f32",
           seed=1707, staggered=False, c_dt=0.5, two_d=False) -> Workload:
    """A workload with explicit per-axis cuts ((cx...), (cy...), (cz...)).
    two_d: a 2D (x, y) problem, global_n[2] == 1 and no guards along z."""
    subs = tensor_decomposition(cuts[0], cuts[1], cuts[2], ng, p)
    if two_d:
        assert global_n[2] == 1
        subs = [dataclasses.replace(sd, zguard=False) for sd in subs]
    assert tuple(sum(c) for c in cuts) == tuple(global_n)
    return Workload(name, tuple(global_n), subs, fields, steps, precision, seed,
                    staggered=staggered, c_dt=c_dt, two_d=two_d)


# ---------------------------------------------------------------------------
# field synthesis
# ---------------------------------------------------------------------------
def _freqs(n: int, d: float, device, half=False) -> torch.Tensor:
    if half:
        return torch.fft.rfftfreq(n, d=d, device=device, dtype=torch.float64) * (2 * math.pi)
    return torch.fft.fftfreq(n, d=d, device=device, dtype=torch.float64) * (2 * math.pi)


def _kgrid_half(global_n, dx, device):
    nx, ny, nz = global_n
    kx = _freqs(nx, dx[0], device, half=True)[None, None, :]
    ky = _freqs(ny, dx[1], device)[None, :, None]
    kz = _freqs(nz, dx[2], device)[:, None, None]
    return kx, ky, kz


def _nyquist_mask(global_n, device):
    """1 everywhere except on the Nyquist plane of every even axis."""
    nx, ny, nz = global_n
    m = torch.ones((nz, ny, nx // 2 + 1), dtype=torch.float64, device=device)
    if nx % 2 == 0:
        m[:, :, nx // 2] = 0
    if ny % 2 == 0:
        m[:, ny // 2, :] = 0
    if nz % 2 == 0:
        m[nz // 2, :, :] = 0
    return m


def _shift_to(spec, comp, kx, ky, kz, dx, staggered):
    """Resample a nodal band-limited field at the component's staggered position."""
    if not staggered:
        return spec
    s = STAGGER[comp]
    ph = kx * (s[0] * dx[0]) + ky * (s[1] * dx[1]) + kz * (s[2] * dx[2])
    return spec * torch.exp(1j * ph)


def _transverse_pair(e_spec, kx, ky, kz):
    """Remove the longitudinal part of a vector spectrum (exact k) and build the
    matching forward-going magnetic field khat x E."""
    k2 = kx * kx + ky * ky + kz * kz
    inv = torch.where(k2 > 0, 1.0 / torch.sqrt(torch.where(k2 > 0, k2, torch.ones_like(k2))),
                      torch.zeros_like(k2))
    hx, hy, hz = kx * inv, ky * inv, kz * inv
    ex, ey, ez = e_spec
    d = hx * ex + hy * ey + hz * ez
    ex, ey, ez = ex - hx * d, ey - hy * d, ez - hz * d
    bx = hy * ez - hz * ey
    by = hz * ex - hx * ez
    bz = hx * ey - hy * ex
    return (ex, ey, ez), (bx, by, bz)


def _random_fields(wl: Workload, device, j_amp: float, rho_amp: float) -> Dict[str, torch.Tensor]:
    nx, ny, nz = wl.global_n
    idx = _global_index(wl.global_n, (0, 0, 0), (nx, ny, nz), device)
    out = {}
    for c, name in enumerate(("Jx", "Jy", "Jz")):
        out[name] = j_amp * (2.0 * uniform(wl.seed, 10 + c, idx) - 1.0)
    out["rho"] = rho_amp * (2.0 * uniform(wl.seed, 13, idx) - 1.0)
    return out


def _wavepacket(wl: Workload, device) -> Dict[str, torch.Tensor]:
    """Gaussian-envelope plane wave along x: Ey = cos(k0 x) exp(-|r-rc|^2/w^2),
    k0 = 2 pi/8, w = 6 cells, projected transverse (exact k) with B = khat x E."""
    nx, ny, nz = wl.global_n
    x = torch.arange(nx, dtype=torch.float64, device=device)[None, None, :] * wl.dx[0]
    y = torch.arange(ny, dtype=torch.float64, device=device)[None, :, None] * wl.dx[1]
    z = torch.arange(nz, dtype=torch.float64, device=device)[:, None, None] * wl.dx[2]
    cx, cy, cz = nx * wl.dx[0] / 2, ny * wl.dx[1] / 2, nz * wl.dx[2] / 2
    k0, w = 2 * math.pi / (8 * wl.dx[0]), 6.0 * wl.dx[0]
    ey = torch.cos(k0 * x) * torch.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / w ** 2)
    kx, ky, kz = _kgrid_half(wl.global_n, wl.dx, device)
    mask = _nyquist_mask(wl.global_n, device)
    zero = torch.zeros((nz, ny, nx // 2 + 1), dtype=torch.complex128, device=device)
    e_spec = (zero, torch.fft.rfftn(ey, dim=(0, 1, 2)) * mask, zero)
    (ex, ey_, ez), (bx, by, bz) = _transverse_pair(e_spec, kx, ky, kz)
    out = {}
    for name, spec in zip(EB_NAMES, (ex, ey_, ez, bx, by, bz)):
        spec = _shift_to(spec, name, kx, ky, kz, wl.dx, wl.staggered)
        out[name] = torch.fft.irfftn(spec, s=(nz, ny, nx), dim=(0, 1, 2))
    out.update(_random_fields(wl, device, 1e-3, 1e-3))
    return out


def _unit_transverse(seed, stream, mode_idx, kx, ky, kz):
    """Random unit polarisation perpendicular to k (exact k)."""
    v = [2.0 * uniform(seed, stream + a, mode_idx) - 1.0 for a in range(3)]
    k2 = kx * kx + ky * ky + kz * kz
    inv = torch.where(k2 > 0, 1.0 / torch.sqrt(torch.where(k2 > 0, k2, torch.ones_like(k2))),
                      torch.zeros_like(k2))
    hx, hy, hz = kx * inv, ky * inv, kz * inv
    d = hx * v[0] + hy * v[1] + hz * v[2]
    v = [v[0] - hx * d, v[1] - hy * d, v[2] - hz * d]
    nrm = torch.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    nrm = torch.where(nrm > 1e-12, nrm, torch.ones_like(nrm))
    return [c / nrm for c in v]


def _broadband(wl: Workload, device) -> Dict[str, torch.Tensor]:
    """Every mode with |k| <= 0.8 pi/dx: unit amplitude, uniform random phase and
    random transverse polarisation; an independent transverse B built the same
    way; J = rho = 0 (vacuum).  Scaled to unit RMS of E."""
    nx, ny, nz = wl.global_n
    kx, ky, kz = _kgrid_half(wl.global_n, wl.dx, device)
    kx, ky, kz = (t.expand(nz, ny, nx // 2 + 1) for t in (kx, ky, kz))
    kmag = torch.sqrt(kx * kx + ky * ky + kz * kz)
    band = (kmag <= 0.8 * math.pi / max(wl.dx)) & (kmag > 0)
    mode = (torch.arange(nz, device=device)[:, None, None] * ny
            + torch.arange(ny, device=device)[None, :, None]) * (nx // 2 + 1) \
        + torch.arange(nx // 2 + 1, device=device)[None, None, :]
    out = {}
    for base, names in ((20, ("Ex", "Ey", "Ez")), (30, ("Bx", "By", "Bz"))):
        pol = _unit_transverse(wl.seed, base, mode, kx, ky, kz)
        phase = 2 * math.pi * uniform(wl.seed, base + 5, mode)
        amp = band.to(torch.float64) * torch.exp(1j * phase)
        for name, c in zip(names, pol):
            out[name] = torch.fft.irfftn(amp * c, s=(nz, ny, nx), dim=(0, 1, 2))
    rms = torch.sqrt(sum((out[n] ** 2).mean() for n in ("Ex", "Ey", "Ez")) / 3)
    for n in EB_NAMES:
        out[n] = out[n] / rms
    for n in ("Jx", "Jy", "Jz", "rho"):
        out[n] = torch.zeros((nz, ny, nx), dtype=torch.float64, device=device)
    return out


def laser_slab_box(wl: Workload, lo, shape, device) -> Dict[str, torch.Tensor]:
    """Plasma-mirror-shaped fields on the periodic box [lo, lo+shape) (x, y, z).

    Laser: p-polarised in the (x, z) plane, k at 45 deg to x, lambda = 32 cells,
    waist 64, longitudinal Gaussian half-length 64, E0 = a0 * 2 pi / lambda with
    a0 = 10, centred at (320, Ny/2, Nz/2); B = khat0 x E (plane-wave relation).
    Slab: normal along x, exponential ramp exp(-d/4) over the 20 cells before
    x = 640, then a 16-cell plateau; J = 0.1 * U[-1, 1] * profile per component,
    rho = U[-1, 1] * profile."""
    nx, ny, nz = wl.global_n
    f64 = torch.float64
    gx = ((torch.arange(shape[0], device=device, dtype=torch.int64) + lo[0]) % nx).to(f64)[None, None, :]
    gy = ((torch.arange(shape[1], device=device, dtype=torch.int64) + lo[1]) % ny).to(f64)[None, :, None]
    gz = ((torch.arange(shape[2], device=device, dtype=torch.int64) + lo[2]) % nz).to(f64)[:, None, None]
    lam, w0, ll, a0 = 32.0, 64.0, 64.0, 10.0
    e0 = a0 * 2 * math.pi / lam
    c45 = math.cos(math.pi / 4)
    khat = (c45, 0.0, c45)
    pol = (-c45, 0.0, c45)
    rx, ry, rz = gx - 320.0, gy - ny / 2, gz - nz / 2
    xi = rx * khat[0] + ry * khat[1] + rz * khat[2]
    r2 = rx * rx + ry * ry + rz * rz
    perp2 = torch.clamp(r2 - xi * xi, min=0.0)
    env = e0 * torch.exp(-(xi * xi) / (ll * ll) - perp2 / (w0 * w0)) * torch.cos(2 * math.pi / lam * xi)
    e = [env * pol[a] for a in range(3)]
    b = [khat[1] * e[2] - khat[2] * e[1], khat[2] * e[0] - khat[0] * e[2], khat[0] * e[1] - khat[1] * e[0]]
    prof = torch.where((gx >= 620) & (gx < 640), torch.exp(-(640.0 - gx) / 4.0),
                       torch.where((gx >= 640) & (gx < 656), torch.ones_like(gx), torch.zeros_like(gx)))
    idx = _global_index(wl.global_n, lo, shape, device)
    out = {}
    full = (len(shape), shape[2], shape[1], shape[0])
    for name, t in zip(EB_NAMES, e + b):
        out[name] = t.expand(full[1:]).clone()
    for c, name in enumerate(("Jx", "Jy", "Jz")):
        out[name] = 0.1 * (2.0 * uniform(wl.seed, 40 + c, idx) - 1.0) * prof
    out["rho"] = (2.0 * uniform(wl.seed, 43, idx) - 1.0) * prof
    return out


def random_fields(global_n, seed: int, names=FIELD_NAMES[:9], device="cpu",
                  dtype=torch.float64) -> Dict[str, torch.Tensor]:
    """Independent U[-1, 1) values per cell for each named field, [Nz][Ny][Nx]
    (one counter-based stream per field name)."""
    nx, ny, nz = global_n
    idx = torch.arange(nx * ny * nz, dtype=torch.int64, device=device)
    out = {}
    for i, n in enumerate(names):
        out[n] = (2.0 * uniform(seed, 200 + FIELD_NAMES.index(n), idx) - 1.0).to(dtype).reshape(nz, ny, nx)
    return out


def global_fields(wl: Workload, device="cpu") -> Dict[str, torch.Tensor]:
    """All ten global fields, FP64, shaped [Nz][Ny][Nx]."""
    if wl.fields == "wavepacket":
        return _wavepacket(wl, device)
    if wl.fields == "broadband":
        return _broadband(wl, device)
    if wl.fields == "laser_slab":
        nx, ny, nz = wl.global_n
        return laser_slab_box(wl, (0, 0, 0), (nx, ny, nz), device)
    raise KeyError(wl.fields)


def box_fields(wl: Workload, sub: Sub, device="cpu") -> Dict[str, torch.Tensor]:
    """The ten fields on one subdomain's padded box, read from the global field
    by periodic index (used to sample a few subdomains of a large workload)."""
    lo = tuple(sub.lo[a] - sub.guards[a] for a in range(3))
    if wl.fields == "laser_slab":
        return laser_slab_box(wl, lo, sub.local, device)
    g = global_fields(wl, device)
    nx, ny, nz = wl.global_n
    ix = (torch.arange(sub.local[0]) + lo[0]) % nx
    iy = (torch.arange(sub.local[1]) + lo[1]) % ny
    iz = (torch.arange(sub.local[2]) + lo[2]) % nz
    return {k: v[iz][:, iy][:, :, ix] for k, v in g.items()}
