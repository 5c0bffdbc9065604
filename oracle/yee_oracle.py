"""Plain FP64 CPU oracle of the Yee FDTD Maxwell step.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/`` and by the CPU-baseline leg
of ``bench.py``; the product path never imports, links or calls it, and it
shares no code with the CUDA path.

What it computes (Vincenti & Vay, arXiv:1707.08500, Sec. 2, Eqs. 2a/2b): the
finite-difference time-domain solver that the paper compares PSATD against,

    D_t B = -curl E          (Faraday)
    D_t E =  curl B - J      (Ampere)

with D_t the centred time difference over one step and D_x, D_y, D_z centred
differences over one cell (c = eps0 = 1).  Readings where the paper is silent:

* the Yee mesh: Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2),
  Bx at (i, j+1/2, k+1/2), By at (i+1/2, j, k+1/2), Bz at (i+1/2, j+1/2, k);
  array element [k, j, i] of a component holds its value at that position;
* time centring of Eq. 2a at step n and of Eq. 2b at n+1/2: the state is
  (E^n, B^{n-1/2}) and J is taken at n+1/2, so one step is
  B^{n+1/2} = B^{n-1/2} - dt curl E^n, then
  E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2});
* the grid is periodic: differences wrap around every axis.

Pins (tests/test_yee_pins.py): a discrete plane wave with the Yee dispersion
relation (sin(w dt/2)/dt)^2 = sum_u (sin(k_u du/2)/du)^2 is reproduced to
rounding; div B is preserved; the J term enters E as -dt J.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

E_NAMES = ("Ex", "Ey", "Ez")
B_NAMES = ("Bx", "By", "Bz")

# staggered position (x, y, z offsets in cells) of each component on the Yee mesh
YEE_STAGGER = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Bx": (0.0, 0.5, 0.5), "By": (0.5, 0.0, 0.5), "Bz": (0.5, 0.5, 0.0),
    "Jx": (0.5, 0.0, 0.0), "Jy": (0.0, 0.5, 0.0), "Jz": (0.0, 0.0, 0.5),
}

# array axis of each spatial direction for [z][y][x] arrays
_AXIS = {"x": 2, "y": 1, "z": 0}


def d_fwd(f: np.ndarray, ax: str, du: float) -> np.ndarray:
    """(f[u+1] - f[u]) / du: the centred difference D_u evaluated half a cell
    above the position of f (periodic)."""
    return (np.roll(f, -1, axis=_AXIS[ax]) - f) / du


def d_bwd(f: np.ndarray, ax: str, du: float) -> np.ndarray:
    """(f[u] - f[u-1]) / du: the centred difference D_u evaluated half a cell
    below the position of f (periodic)."""
    return (f - np.roll(f, 1, axis=_AXIS[ax])) / du


def curl_e(E: Dict[str, np.ndarray], dx: Sequence[float]) -> Dict[str, np.ndarray]:
    """curl E at the B positions (Eq. 2a right-hand side, without the sign)."""
    ddx, ddy, ddz = dx
    return {
        "Bx": d_fwd(E["Ez"], "y", ddy) - d_fwd(E["Ey"], "z", ddz),
        "By": d_fwd(E["Ex"], "z", ddz) - d_fwd(E["Ez"], "x", ddx),
        "Bz": d_fwd(E["Ey"], "x", ddx) - d_fwd(E["Ex"], "y", ddy),
    }


def curl_b(B: Dict[str, np.ndarray], dx: Sequence[float]) -> Dict[str, np.ndarray]:
    """curl B at the E positions (Eq. 2b right-hand side, without J)."""
    ddx, ddy, ddz = dx
    return {
        "Ex": d_bwd(B["Bz"], "y", ddy) - d_bwd(B["By"], "z", ddz),
        "Ey": d_bwd(B["Bx"], "z", ddz) - d_bwd(B["Bz"], "x", ddx),
        "Ez": d_bwd(B["By"], "x", ddx) - d_bwd(B["Bx"], "y", ddy),
    }


def yee_step(f: Dict[str, np.ndarray], dx: Sequence[float], dt: float) -> Dict[str, np.ndarray]:
    """One step of Eqs. 2a/2b: (E^n, B^{n-1/2}, J^{n+1/2}) -> (E^{n+1}, B^{n+1/2}).
    Returns a new dict with the six updated components (J, rho passed through)."""
    out = dict(f)
    ce = curl_e(f, dx)
    for n in B_NAMES:
        out[n] = f[n] - dt * ce[n]
    cb = curl_b(out, dx)
    for n, j in zip(E_NAMES, ("Jx", "Jy", "Jz")):
        out[n] = f[n] + dt * (cb[n] - f[j])
    return out


def yee_run(f: Dict[str, np.ndarray], dx: Sequence[float], dt: float, steps: int) -> Dict[str, np.ndarray]:
    for _ in range(steps):
        f = yee_step(f, dx, dt)
    return f


def divergence_b(B: Dict[str, np.ndarray], dx: Sequence[float]) -> np.ndarray:
    """Discrete div B at the cell centres (i+1/2, j+1/2, k+1/2)."""
    return d_fwd(B["Bx"], "x", dx[0]) + d_fwd(B["By"], "y", dx[1]) + d_fwd(B["Bz"], "z", dx[2])


def courant_limit(dx: Sequence[float]) -> float:
    """Largest stable c dt of the Yee scheme: 1 / sqrt(sum 1/du^2)."""
    return 1.0 / float(np.sqrt(sum(1.0 / d ** 2 for d in dx)))
