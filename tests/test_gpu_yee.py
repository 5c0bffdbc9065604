"""Parity of the Yee FDTD kernel (through the C ABI) with the FP64 Yee oracle
(Sec. 2, Eqs. 2a/2b): both copy paths (16-byte tile rows when Nx is a
multiple of 32, single elements otherwise), ragged tiles and z chunks, tiny
and 2D grids, anisotropic cells, FP64 to 1e-12 and FP32 to 1e-5 after 100
steps, plus the closed-form Yee plane wave on the GPU."""
import math

import numpy as np
import pytest
import torch

from oracle import yee_oracle as Y
from paper_1707_08500_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_08500_gb300 import build
    build.build()
    from paper_1707_08500_gb300 import fdtd
    return fdtd


def _rel(a, b, names):
    num = sum(float(((a[n] - b[n]) ** 2).sum()) for n in names)
    den = sum(float((b[n] ** 2).sum()) for n in names)
    return math.sqrt(num / den)


@pytest.mark.parametrize("shape,dx,steps,prec,tol", [
    ((48, 40, 36), (1.0, 1.0, 1.0), 10, "f64", 1e-12),       # ragged x tile and z chunk
    ((20, 13, 5), (1.0, 0.8, 1.25), 7, "f64", 1e-12),        # smaller than one tile, anisotropic
    ((64, 48, 1), (1.0, 1.0, 1.0), 12, "f64", 1e-12),        # 2D
    ((1, 1, 70), (1.0, 1.0, 1.0), 5, "f64", 1e-12),          # one column: x and y wrap onto themselves
    ((33, 9, 65), (0.9, 1.1, 1.0), 4, "f64", 1e-12),         # one past a tile on every axis
    ((64, 13, 9), (1.0, 0.8, 1.25), 6, "f64", 1e-12),        # full x tiles (16-byte rows), ragged y tile
    ((128, 24, 40), (1.0, 1.0, 1.0), 5, "f64", 1e-12),       # full x tiles, ragged z chunk
    ((96, 64, 70), (1.0, 1.0, 1.0), 100, "f32", 1e-5),       # FP32 over many steps (full x tiles)
    ((100, 30, 20), (1.0, 1.0, 1.0), 50, "f32", 1e-5),       # FP32, element copies
])
def test_yee_matches_oracle(F, shape, dx, steps, prec, tol):
    glob = I.random_fields(shape, 1707 + 50, names=Y.E_NAMES + Y.B_NAMES + ("Jx", "Jy", "Jz"))
    # keep J small so that the fields stay O(1) over the run
    for n in ("Jx", "Jy", "Jz"):
        glob[n] = glob[n] * 0.01
    dt = 0.95 * Y.courant_limit(dx)
    sol = F.YeeSolver(shape, dt, dx, precision=prec)
    sol.load(glob)
    for _ in range(steps):
        sol.step()
    torch.cuda.synchronize()
    got = {k: v.numpy() for k, v in sol.gather().items()}
    ref = Y.yee_run({k: v.numpy() for k, v in glob.items()}, dx, dt, steps)
    err = _rel(got, ref, Y.E_NAMES + Y.B_NAMES)
    print(f"Yee {shape} {prec} {steps} steps: rel L2 {err:.3e}")
    assert err < tol


def test_yee_plane_wave_closed_form_f64(F):
    """The exact discrete plane wave of the Yee dispersion relation."""
    N, DX, m = (24, 20, 16), (1.0, 0.8, 1.25), (3, -2, 1)
    dt = 0.9 * Y.courant_limit(DX)
    k = np.array([2 * math.pi * m[a] / (N[a] * DX[a]) for a in range(3)])
    kt = np.array([2 * math.sin(k[a] * DX[a] / 2) / DX[a] for a in range(3)])
    w = 2.0 / dt * math.asin(np.linalg.norm(kt) * dt / 2)
    E0 = np.cross(kt, (0.3, -1.0, 0.7))
    E0 /= np.linalg.norm(E0)
    B0 = np.cross(kt, E0) / np.linalg.norm(kt)

    def fields(tE, tB):
        out = {}
        for c, (n, amp, t) in enumerate(zip(Y.E_NAMES + Y.B_NAMES, list(E0) + list(B0), [tE] * 3 + [tB] * 3)):
            sx, sy, sz = Y.YEE_STAGGER[n]
            z, y, x = np.meshgrid((np.arange(N[2]) + sz) * DX[2], (np.arange(N[1]) + sy) * DX[1],
                                  (np.arange(N[0]) + sx) * DX[0], indexing="ij")
            out[n] = amp * np.cos(k[0] * x + k[1] * y + k[2] * z - w * t)
        return out
    sol = F.YeeSolver(N, dt, DX, precision="f64")
    sol.load({n: torch.from_numpy(v) for n, v in fields(0.0, -0.5 * dt).items()})
    steps = 40
    for _ in range(steps):
        sol.step()
    torch.cuda.synchronize()
    got = sol.gather()
    exp = fields(steps * dt, (steps - 0.5) * dt)
    err = max(float(np.abs(got[n].numpy() - exp[n]).max()) for n in exp)
    assert err < 1e-11, err
