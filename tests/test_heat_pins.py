"""Pins of the local-FFT heat-equation oracle against what the mathematics
fixes: the periodic Gaussian heat kernel, textbook single-mode decay at
orders 2 and 4, conservation of the mean, the exact source response, the
exact one-period special case of the decomposition, and the guard-truncation
error falling with the guard count.  CPU only."""
import itertools
import math

import numpy as np
import pytest

from oracle import heat_oracle as H
from paper_1707_08500_gb300 import inputs as I

N = (32, 24, 20)
DX = (1.0, 0.8, 1.25)


def _grid(shape_xyz, dx):
    nx, ny, nz = shape_xyz
    z, y, x = np.meshgrid(np.arange(nz) * dx[2], np.arange(ny) * dx[1], np.arange(nx) * dx[0], indexing="ij")
    return x, y, z


def _periodic_gaussian(var, centre, shape_xyz, dx):
    """sum over periodic images of (s0^2 / var)^{3/2} exp(-|r - c|^2 / (2 var))."""
    x, y, z = _grid(shape_xyz, dx)
    box = [shape_xyz[a] * dx[a] for a in range(3)]
    out = np.zeros(x.shape)
    for i, j, k in itertools.product(range(-2, 3), repeat=3):
        r2 = ((x - centre[0] - i * box[0]) ** 2 + (y - centre[1] - j * box[1]) ** 2 +
              (z - centre[2] - k * box[2]) ** 2)
        out += np.exp(-r2 / (2 * var))
    return out


def test_periodic_gaussian_heat_kernel_closed_form():
    s0, d_dt, steps = 2.5, 0.3, 5
    c = (14.3, 9.1, 12.0)
    T = _periodic_gaussian(s0 ** 2, c, N, DX)
    wl = I.custom("g", N, ((N[0],), (N[1],), (N[2],)), 0, 0, fields="wavepacket", precision="f64")
    wl = I.Workload(wl.name, wl.global_n, wl.subs, wl.fields, 1, "f64", 1, dx=DX)
    out = H.heat_run({"T": T}, wl, d_dt, steps)["T"]
    var = s0 ** 2 + 2 * d_dt * steps
    exp = (s0 ** 2 / var) ** 1.5 * _periodic_gaussian(var, c, N, DX)
    assert np.abs(out - exp).max() < 1e-12


@pytest.mark.parametrize("p", [2, 4])
def test_single_mode_decay_textbook_orders(p):
    """cos(k.x) decays by exp(-D dt |[k]|^2) with the textbook order-2
    Laplacian symbol 4 sin^2(k du/2)/du^2 and the square of the order-4
    staggered first difference (9/8, -1/24)."""
    m = (3, -2, 5)
    k = [2 * math.pi * m[a] / (N[a] * DX[a]) for a in range(3)]
    if p == 2:
        kk = [2 * math.sin(k[a] * DX[a] / 2) / DX[a] for a in range(3)]
    else:
        kk = [(9 / 8) * 2 * math.sin(k[a] * DX[a] / 2) / DX[a] - (1 / 24) * 2 * math.sin(3 * k[a] * DX[a] / 2) / DX[a]
              for a in range(3)]
    x, y, z = _grid(N, DX)
    T = np.cos(k[0] * x + k[1] * y + k[2] * z)
    d_dt = 0.7
    out = H.heat_global_push(T, None, p, DX, d_dt)
    assert np.abs(out - math.exp(-d_dt * sum(v * v for v in kk)) * T).max() < 1e-13


def test_source_response_and_mean():
    rng = np.random.default_rng(3)
    shape = (N[2], N[1], N[0])
    T = rng.standard_normal(shape)
    S = rng.standard_normal(shape)
    out = H.heat_global_push(T, S, 8, DX, 0.4)
    assert abs(out.sum() - (T.sum() + S.sum())) < 1e-9
    # a uniform source is added as it is
    c = np.full(shape, 0.37)
    np.testing.assert_allclose(H.heat_global_push(np.zeros(shape), c, 8, DX, 0.4), c, atol=1e-14)
    # a single source mode is scaled by (1 - exp(-x)) / x at order 2
    m = (1, 2, 3)
    k = [2 * math.pi * m[a] / (N[a] * DX[a]) for a in range(3)]
    x, y, z = _grid(N, DX)
    Sm = np.cos(k[0] * x + k[1] * y + k[2] * z)
    xx = 0.4 * sum((2 * math.sin(k[a] * DX[a] / 2) / DX[a]) ** 2 for a in range(3))
    np.testing.assert_allclose(H.heat_global_push(np.zeros(shape), Sm, 2, DX, 0.4), -math.expm1(-xx) / xx * Sm,
                               atol=1e-13)


@pytest.mark.parametrize("p", [0, 8])
def test_local_equals_global_when_padded_box_is_one_period(p):
    n = 16
    wl = I.custom("sp", (n, n, n), ((8, 8),) * 3, 4, p)
    rng = np.random.default_rng(5)
    T = rng.standard_normal((n, n, n))
    S = rng.standard_normal((n, n, n))
    a = H.heat_run({"T": T, "S": S}, wl, 0.6, 3)["T"]
    b = T
    for _ in range(3):
        b = H.heat_global_push(b, S, p, (1.0, 1.0, 1.0), 0.6)
    assert H.rel_l2(a, b) < 1e-13


def test_guard_truncation_error_falls_with_guard_count():
    """No finite propagation speed: the error is set by the diffusion length
    sqrt(2 D dt) against the guard width (at p = 8 it falls by about two
    orders of magnitude per two guard cells; at p = 0 the spectrum cut at
    Nyquist leaves slowly decaying tails and it falls much more slowly)."""
    n, p, steps, d_dt = 48, 8, 4, 0.5
    x, y, z = _grid((n, n, n), (1.0, 1.0, 1.0))
    T = np.exp(-((x - 23.5) ** 2 + (y - 22.0) ** 2 + (z - 25.0) ** 2) / (2 * 9.0))
    ref = T
    for _ in range(steps):
        ref = H.heat_global_push(ref, None, p, (1.0, 1.0, 1.0), d_dt)
    errs = []
    for ng in (2, 4, 6, 8):
        wl = I.custom("h", (n, n, n), ((24, 24),) * 3, ng, p)
        errs.append(H.rel_l2(H.heat_run({"T": T}, wl, d_dt, steps)["T"], ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5 * errs[0], errs


def test_nyquist_mode_decays():
    """The checkerboard (-1)^(i+j+k) is damped by exp(-D dt sum_u 4/du^2) at
    order 2 (the textbook 3-point Laplacian)."""
    x = np.indices((N[2], N[1], N[0])).sum(axis=0)
    T = (-1.0) ** x
    out = H.heat_global_push(T, None, 2, DX, 0.05)
    np.testing.assert_allclose(out, math.exp(-0.05 * sum(4 / d ** 2 for d in DX)) * T, atol=1e-14)


# --------------------------------------------------------------------------
# planted mistakes: each plausible error in the oracle fails a pin above
# --------------------------------------------------------------------------
def _pin_errors():
    """Largest deviation of each closed-form pin above, in one dict."""
    out = {}
    m = (3, -2, 5)
    k = [2 * math.pi * m[a] / (N[a] * DX[a]) for a in range(3)]
    x, y, z = _grid(N, DX)
    T = np.cos(k[0] * x + k[1] * y + k[2] * z)
    kk = [2 * math.sin(k[a] * DX[a] / 2) / DX[a] for a in range(3)]
    xx = 0.7 * sum(v * v for v in kk)
    out["mode"] = float(np.abs(H.heat_global_push(T, None, 2, DX, 0.7) - math.exp(-xx) * T).max())
    out["source"] = float(np.abs(H.heat_global_push(np.zeros_like(T), T, 2, DX, 0.7) + math.expm1(-xx) / xx * T).max())
    chk = (-1.0) ** np.indices(T.shape).sum(axis=0)
    out["nyquist"] = float(np.abs(H.heat_global_push(chk, None, 2, DX, 0.05) -
                                  math.exp(-0.05 * sum(4 / d ** 2 for d in DX)) * chk).max())
    return out


def _mutant(name):
    k2, fac = H.heat_k2, H.heat_factors
    if name == "ignored_cell_size":
        return "heat_k2", lambda L, du, p: k2(L, 1.0, p)
    if name == "doubled_dt":
        return "heat_factors", lambda kk, d_dt: fac(kk, 2 * d_dt)
    if name == "dropped_source_factor":
        return "heat_factors", lambda kk, d_dt: (fac(kk, d_dt)[0], np.ones_like(kk))
    if name == "nodal_weights":
        from oracle import psatd_oracle as O

        def nodal(L, du, p):
            km = O.modified_k(L, du, p, False)
            return km * km
        return "heat_k2", nodal
    raise ValueError(name)


@pytest.mark.parametrize("name", ["ignored_cell_size", "doubled_dt", "dropped_source_factor", "nodal_weights"])
def test_pins_catch_planted_mistakes(monkeypatch, name):
    assert max(_pin_errors().values()) < 1e-12
    attr, fn = _mutant(name)
    monkeypatch.setattr(H, attr, fn)
    assert max(_pin_errors().values()) > 1e-3
