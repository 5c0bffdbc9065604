"""Pins of the Yee FDTD oracle (Sec. 2, Eqs. 2a/2b) against what the
mathematics fixes: the exact discrete plane wave of the Yee dispersion
relation, the discrete identities div curl = 0 (div B preserved, Gauss's law
with a continuity-consistent J), and the J term of Eq. 2b.  CPU only."""
import math

import numpy as np
import pytest

from oracle import yee_oracle as Y

N = (24, 20, 16)
DX = (1.0, 0.8, 1.25)


def _positions(name, shape, dx):
    nz, ny, nx = shape
    sx, sy, sz = Y.YEE_STAGGER[name]
    z, y, x = np.meshgrid((np.arange(nz) + sz) * dx[2], (np.arange(ny) + sy) * dx[1],
                          (np.arange(nx) + sx) * dx[0], indexing="ij")
    return x, y, z


def _plane_wave(m, dt, amp_seed):
    """Closed-form Yee plane wave: wavevector k = 2 pi m / (N du), discrete
    wavevector kt_u = 2 sin(k_u du / 2) / du, frequency w with
    2 sin(w dt / 2) / dt = |kt|, E0 perpendicular to kt, B0 = kt x E0 / |kt|.
    Returns (k, w, E0, B0)."""
    k = np.array([2 * math.pi * m[a] / (N[a] * DX[a]) for a in range(3)])
    kt = np.array([2 * math.sin(k[a] * DX[a] / 2) / DX[a] for a in range(3)])
    wt = float(np.linalg.norm(kt))
    w = 2.0 / dt * math.asin(wt * dt / 2)
    a = np.random.default_rng(amp_seed).standard_normal(3)
    E0 = np.cross(kt, a)
    E0 /= np.linalg.norm(E0)
    B0 = np.cross(kt, E0) / wt
    return k, w, E0, B0


def _wave_fields(k, w, E0, B0, tE, tB):
    shape = (N[2], N[1], N[0])
    f = {}
    for c, n in enumerate(Y.E_NAMES):
        x, y, z = _positions(n, shape, DX)
        f[n] = E0[c] * np.cos(k[0] * x + k[1] * y + k[2] * z - w * tE)
    for c, n in enumerate(Y.B_NAMES):
        x, y, z = _positions(n, shape, DX)
        f[n] = B0[c] * np.cos(k[0] * x + k[1] * y + k[2] * z - w * tB)
    for n in ("Jx", "Jy", "Jz"):
        f[n] = np.zeros(shape)
    return f


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 3, 0), (0, 0, 2), (3, -2, 1), (11, 9, 7)])
def test_discrete_plane_wave_follows_yee_dispersion(m):
    dt = 0.9 * Y.courant_limit(DX)
    k, w, E0, B0 = _plane_wave(m, dt, 5)
    steps = 40
    f = _wave_fields(k, w, E0, B0, 0.0, -0.5 * dt)
    got = Y.yee_run(f, DX, dt, steps)
    exp = _wave_fields(k, w, E0, B0, steps * dt, (steps - 0.5) * dt)
    err = max(np.abs(got[n] - exp[n]).max() for n in Y.E_NAMES + Y.B_NAMES)
    assert err < 1e-11, err
    # the exact-k frequency (no numerical dispersion) is measurably wrong
    if m == (11, 9, 7):
        wrong = _wave_fields(k, float(np.linalg.norm(k)), E0, B0, steps * dt, (steps - 0.5) * dt)
        assert max(np.abs(got[n] - wrong[n]).max() for n in Y.E_NAMES) > 1e-2


def test_div_b_is_preserved():
    rng = np.random.default_rng(7)
    shape = (N[2], N[1], N[0])
    f = {n: rng.standard_normal(shape) for n in Y.E_NAMES + Y.B_NAMES + ("Jx", "Jy", "Jz")}
    d0 = Y.divergence_b(f, DX)
    g = Y.yee_run(f, DX, 0.5, 10)
    assert np.abs(Y.divergence_b(g, DX) - d0).max() < 1e-11


def test_gauss_law_with_continuity_current():
    """div E (at the nodes, backward differences) changes by -dt div J in one
    step, for any B: the discrete div curl B vanishes."""
    rng = np.random.default_rng(8)
    shape = (N[2], N[1], N[0])
    f = {n: rng.standard_normal(shape) for n in Y.E_NAMES + Y.B_NAMES + ("Jx", "Jy", "Jz")}

    def div_node(a, b, c):
        return Y.d_bwd(a, "x", DX[0]) + Y.d_bwd(b, "y", DX[1]) + Y.d_bwd(c, "z", DX[2])
    dt = 0.4
    g = Y.yee_step(f, DX, dt)
    lhs = div_node(g["Ex"], g["Ey"], g["Ez"]) - div_node(f["Ex"], f["Ey"], f["Ez"])
    rhs = -dt * div_node(f["Jx"], f["Jy"], f["Jz"])
    assert np.abs(lhs - rhs).max() < 1e-11


def test_current_enters_e_as_minus_dt_j():
    rng = np.random.default_rng(9)
    shape = (N[2], N[1], N[0])
    f = {n: rng.standard_normal(shape) for n in Y.E_NAMES + Y.B_NAMES}
    f0 = dict(f, **{n: np.zeros(shape) for n in ("Jx", "Jy", "Jz")})
    J = {n: rng.standard_normal(shape) for n in ("Jx", "Jy", "Jz")}
    a = Y.yee_step(f0, DX, 0.3)
    b = Y.yee_step(dict(f, **J), DX, 0.3)
    for n, j in zip(Y.E_NAMES, ("Jx", "Jy", "Jz")):
        np.testing.assert_allclose(b[n] - a[n], -0.3 * J[j], atol=1e-13)
    for n in Y.B_NAMES:
        assert np.array_equal(a[n], b[n])


def test_courant_limit_textbook():
    assert abs(Y.courant_limit((1.0, 1.0, 1.0)) - 1 / math.sqrt(3)) < 1e-15
    assert abs(Y.courant_limit((1.0, 1e9, 1e9)) - 1.0) < 1e-12


# --------------------------------------------------------------------------
# planted mistakes: each plausible error in the oracle fails a pin above
# --------------------------------------------------------------------------
def _plane_wave_error(m=(3, -2, 1), steps=20):
    dt = 0.9 * Y.courant_limit(DX)
    k, w, E0, B0 = _plane_wave(m, dt, 5)
    got = Y.yee_run(_wave_fields(k, w, E0, B0, 0.0, -0.5 * dt), DX, dt, steps)
    exp = _wave_fields(k, w, E0, B0, steps * dt, (steps - 0.5) * dt)
    return max(np.abs(got[n] - exp[n]).max() for n in Y.E_NAMES + Y.B_NAMES)


def _mutant(name):
    bwd, ce, cb = Y.d_bwd, Y.curl_e, Y.curl_b
    if name == "forward_as_backward":       # a difference taken in the wrong direction
        return "d_fwd", lambda f, ax, du: bwd(f, ax, du)
    if name == "curl_e_sign":               # Faraday with the wrong sign
        return "curl_e", lambda E, dx: {k: -v for k, v in ce(E, dx).items()}
    if name == "swapped_cell_sizes":        # dx and dz exchanged in curl B
        return "curl_b", lambda B, dx: cb(B, (dx[2], dx[1], dx[0]))
    if name == "half_curl_b":               # Ampere's curl term halved
        return "curl_b", lambda B, dx: {k: 0.5 * v for k, v in cb(B, dx).items()}
    raise ValueError(name)


@pytest.mark.parametrize("name", ["forward_as_backward", "curl_e_sign", "swapped_cell_sizes", "half_curl_b"])
def test_plane_wave_pin_catches_planted_mistakes(monkeypatch, name):
    assert _plane_wave_error() < 1e-11
    attr, fn = _mutant(name)
    monkeypatch.setattr(Y, attr, fn)
    assert _plane_wave_error() > 1e-3
