"""Plain FP64 CPU oracle of the local-FFT heat-equation step.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/`` and by the CPU-baseline leg
of ``bench.py``; the product path never imports, links or calls it, and it
shares no code with the CUDA path.

What it computes.  Sec. 5 of Vincenti & Vay (arXiv:1707.08500) states that
the local-FFT decomposition of Sec. 3.2 applies to other initial-value
problems solved by FFT-based pseudo-spectral methods and that the authors
tested it on the heat equation.  The paper gives no equations for it; the
readings here (listed with their reasons in the design notes) are:

* the equation dT/dt = D lap T + Q, advanced by its exact per-mode solution
  over one step, the analogue of Eq. 1 for Maxwell's equations:
      T~' = exp(-x) T~ + (1 - exp(-x)) / x * S~,   x = D dt |[k]|^2,
  where S = Q dt is the heat added per cell over the step (held constant
  over it) and the factor tends to 1 at x = 0;
* the Laplacian symbol is -sum_u [k_u]^2 with [k_u] the order-p STAGGERED
  modified wavenumber of Sec. 3.1 (p = 0: the exact k), i.e. the order-p
  staggered first difference applied twice (div of grad in flux form; p = 2
  gives the textbook 3-point Laplacian 4 sin^2(k du/2)/du^2).  Unlike the
  Maxwell reading, the Nyquist index keeps its value (k = pi/du): only the
  square enters, which is even in k, and a centred NODAL first difference
  applied twice would leave the Nyquist mode undamped;
* the decomposition is that of Sec. 3.2 / Fig. 3: padded local boxes, local
  FFTs over the padded box, valid cells kept, guards refilled from their
  owners.  Unlike light, heat has no finite propagation speed: the guard
  truncation error is set by the diffusion length sqrt(2 D dt) against the
  guard width, and its size is not fixed by the paper (parity unpinned: only
  its fall with the guard count and the exact one-period case are pinned).

Pins (tests/test_heat_pins.py): the periodic Gaussian heat kernel in closed
form (p = 0, one box), the decay of single Fourier modes by exp(-D dt [k]^2),
the conservation of the mean (and its growth by the mean of S), local equals
global when the padded box is one period, and the guard-truncation error
falling with the guard count.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

from . import psatd_oracle as _po


def heat_k2(L: int, du: float, p: int) -> np.ndarray:
    """[k]^2 of every index of an L-point axis (FFT order): the square of the
    order-p staggered first-difference symbol sum_j c_j 2 sin((2j-1) k du/2)/du
    (p = 0: k^2), Nyquist included."""
    n = np.arange(L)
    n = np.where(n < (L + 1) // 2, n, n - L)
    k = 2.0 * np.pi * n / (L * du)
    if p == 0:
        return k * k
    c = _po.fd_weights_staggered(p)
    s = np.zeros(L)
    for j in range(1, len(c) + 1):
        s += c[j - 1] * 2.0 * np.sin((2 * j - 1) * k * du / 2.0) / du
    return s * s


def heat_factors(k2, d_dt: float):
    """(exp(-x), (1 - exp(-x))/x) with x = D dt |[k]|^2 (1 at x = 0)."""
    x = d_dt * k2
    a = np.exp(-x)
    safe = np.where(x > 0, x, 1.0)
    b = np.where(x > 0, -np.expm1(-x) / safe, 1.0)
    return a, b


def local_heat_push(T: np.ndarray, S: np.ndarray | None, L, dx, p: int, d_dt: float) -> np.ndarray:
    """One exact step of one padded local box [Lz][Ly][Lx]; S is the heat
    added per cell over the step (None: no source)."""
    Lx, Ly, Lz = L
    k2 = (heat_k2(Lx, dx[0], p)[: Lx // 2 + 1][None, None, :] + heat_k2(Ly, dx[1], p)[None, :, None] +
          heat_k2(Lz, dx[2], p)[:, None, None])
    a, b = heat_factors(k2, d_dt)
    F = a * _po.r2c(T)
    if S is not None:
        F = F + b * _po.r2c(S)
    return _po.c2r(F, (Lz, Ly, Lx))


def heat_step(glob: Dict[str, np.ndarray], wl, d_dt: float) -> Dict[str, np.ndarray]:
    """One local-FFT step over all subdomains.  glob: 'T' and optionally 'S'
    global arrays [Nz][Ny][Nx]; returns the dict with T advanced."""
    T = np.empty_like(glob["T"])
    for sd in wl.subs:
        g = _po.sub_guards(sd)
        loc = _po.extract_box(glob["T"], sd.lo, sd.local, g)
        src = _po.extract_box(glob["S"], sd.lo, sd.local, g) if "S" in glob else None
        out = local_heat_push(loc, src, sd.local, wl.dx, sd.p, d_dt)
        (x0, y0, z0), (nx, ny, nz) = sd.lo, sd.n
        gx, gy, gz = g
        T[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] = out[gz:gz + nz, gy:gy + ny, gx:gx + nx]
    return dict(glob, T=T)


def heat_run(glob: Dict[str, np.ndarray], wl, d_dt: float, steps: int) -> Dict[str, np.ndarray]:
    for _ in range(steps):
        glob = heat_step(glob, wl, d_dt)
    return glob


def heat_global_push(T: np.ndarray, S: np.ndarray | None, p: int, dx: Sequence[float], d_dt: float) -> np.ndarray:
    """The same step with one FFT over the whole periodic grid."""
    Nz, Ny, Nx = T.shape
    return local_heat_push(T, S, (Nx, Ny, Nz), dx, p, d_dt)


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))
