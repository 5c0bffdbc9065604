"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative L2 over the valid cells of E and B stacked, 1e-12 for
the FP64 path and 2e-6 per step (1e-5 over many steps) for the FP32 path; the
exchange is bit-exact (it is a copy)."""
import math

import numpy as np
import pytest
import torch

from oracle import psatd_oracle as O
from paper_1707_08500_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_08500_gb300 import build
    build.build()
    from paper_1707_08500_gb300 import psatd
    return psatd


def _np(d):
    return {k: v.numpy() if isinstance(v, torch.Tensor) else v for k, v in d.items()}


def _run_gpu(P, wl, glob, steps, plain=False, gauss=False, precision=None, split=False):
    sol = P.Solver(wl, precision=precision, plain=plain, gauss=gauss,
                   extra_flags=P.PSATD_SPLIT_PLANES if split else 0)
    sol.load_global(glob, names=I.EB_NAMES, guards=False)
    sol.load_global(glob, names=("Jx", "Jy", "Jz", "rho"), guards=True)
    sol.exchange()
    sums = []
    for _ in range(steps):
        sol.push()
        if gauss:
            torch.cuda.synchronize()
            sums.append(sol.gauss_sums().copy())
    torch.cuda.synchronize()
    return sol, sums


def _oracle(wl, glob, steps):
    g = _np(glob)
    sums = []
    for _ in range(steps):
        gs = []
        g = O.step(g, wl, gauss_out=gs)
        sums.append(np.array(gs))
    return g, sums


MIXED = dict(global_n=(32, 27, 35), cuts=((12, 20), (14, 13), (18, 17)))  # radices 2,3,5,7,11,13


def _mixed(precision, staggered=False, ng=4):
    p = lambda ix, iy, iz: (4, 8, 0, 12)[(ix + 2 * iy + iz) % 4]
    subs = I.tensor_decomposition(*MIXED["cuts"], ng, p)
    return I.Workload("mixed", MIXED["global_n"], subs, "wavepacket", 3, precision, 1707 + 9,
                      staggered=staggered, c_dt=0.7)


CASES = {
    "plain32_f64": (lambda: I.custom("p32", (32, 32, 32), ((32,),) * 3, 0, 0, fields="wavepacket",
                                     precision="f64"), 4, 1e-12),
    "yee_small_f64": (lambda: I.custom("yee", (32, 32, 32), ((16, 16),) * 3, 4, 8, fields="wavepacket",
                                       precision="f64", staggered=True), 3, 1e-12),
    "mixed_f64": (lambda: _mixed("f64"), 2, 1e-12),
    "mixed_stag_f64": (lambda: _mixed("f64", staggered=True), 2, 1e-12),
    "mixed_f32": (lambda: _mixed("f32"), 2, 4e-6),
    "broadband_f32": (lambda: I.custom("bb", (64, 64, 64), ((32, 32),) * 3, 8, 16, fields="broadband",
                                       precision="f32"), 5, 1e-5),
    "wide_guard_f64": (lambda: I.custom("wg", (40, 16, 16), ((8, 32), (16,), (16,)), 10, 6,
                                        fields="wavepacket", precision="f64"), 2, 1e-12),
    # 2D problems: one cell along z, no guards along z
    "twod_f64": (lambda: I.custom("2d", (48, 30, 1), ((30, 18), (16, 14), (1,)), 6, 16, fields="wavepacket",
                                  precision="f64", two_d=True), 3, 1e-12),
    "twod_stag_f64": (lambda: I.custom("2ds", (40, 36, 1), ((24, 16), (20, 16), (1,)), 4, 8, fields="wavepacket",
                                       precision="f64", staggered=True, two_d=True), 3, 1e-12),
    "twod_f32": (lambda: I.custom("2df", (64, 64, 1), ((32, 32), (32, 32), (1,)), 8, 16, fields="broadband",
                                  precision="f32", two_d=True), 5, 1e-5),
    "twod_global_f64": (lambda: I.custom("2dg", (128, 96, 1), ((128,), (96,), (1,)), 0, 0, fields="wavepacket",
                                         precision="f64", two_d=True), 2, 1e-12),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("schedule", ["batched", "plain", "split", "split_plain"])
def test_push_matches_oracle(P, name, schedule):
    make, steps, tol = CASES[name]
    wl = make()
    glob = I.global_fields(wl)
    sol, _ = _run_gpu(P, wl, glob, steps, plain="plain" in schedule, split="split" in schedule)
    ref, _ = _oracle(wl, glob, steps)
    got = _np(sol.gather_global())
    err = O.rel_l2(got, ref)
    assert err < tol, f"{name}: rel L2 {err:.3e}"
    # guards hold the owners' values after the step (fused or separate
    # exchange): bit for bit the owners' valid cells on the GPU (the gathered
    # global arrays), and close to the oracle's
    for s in range(len(wl.subs)):
        for n in I.EB_NAMES:
            exp = O.extract_box(ref[n], wl.subs[s].lo, wl.subs[s].local, O.sub_guards(wl.subs[s]))
            own = O.extract_box(got[n], wl.subs[s].lo, wl.subs[s].local, O.sub_guards(wl.subs[s]))
            box = sol.box(n, s).double().cpu().numpy()
            assert np.array_equal(box, own.astype(np.float64)), (name, s, n)
            scale = max(np.abs(exp).max(), 1e-30)
            assert np.abs(box - exp).max() / scale < 50 * tol, (name, s, n)


def test_exchange_is_exact_copy(P):
    wl = _mixed("f32", ng=4)
    glob = I.global_fields(wl)
    sol = P.Solver(wl)
    sol.load_global(glob, names=I.EB_NAMES, guards=False)
    sol.exchange()
    torch.cuda.synchronize()
    for s, sd in enumerate(wl.subs):
        for n in I.EB_NAMES:
            exp = O.extract_box(glob[n].numpy().astype(np.float32), sd.lo, sd.local, sd.ng)
            assert np.array_equal(sol.box(n, s).cpu().numpy(), exp), (s, n)


def _twod(precision):
    return I.custom("2dg", (48, 30, 1), ((30, 18), (16, 14), (1,)), 6, 16, fields="wavepacket",
                    precision=precision, two_d=True)


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("shape", ["3d", "2d"])
@pytest.mark.parametrize("precision,tol", [("f64", 1e-9), ("f32", 1e-3)])
def test_gauss_partials_match_oracle(P, precision, tol, shape, split):
    wl = _mixed(precision) if shape == "3d" else _twod(precision)
    glob = I.global_fields(wl)
    _, gsum = _run_gpu(P, wl, glob, 2, gauss=True, split=split)
    _, osum = _oracle(wl, glob, 2)
    for a, b in zip(gsum, osum):
        np.testing.assert_allclose(a[:, 1], b[:, 1], rtol=tol)        # |rho~|^2
        np.testing.assert_allclose(a[:, 0], b[:, 0], rtol=tol)        # |i[k].E - rho|^2


def test_repeat_is_deterministic(P):
    wl = _mixed("f32")
    glob = I.global_fields(wl)
    a, _ = _run_gpu(P, wl, glob, 3)
    b, _ = _run_gpu(P, wl, glob, 3)
    for n in I.EB_NAMES:
        assert torch.equal(a.arenas[n], b.arenas[n])
    # persistent launches of both runs drew exactly their own tickets, and
    # every item was decoded inside its subdomain
    assert P.psatd_check(a.plan) == 0 and P.psatd_check(b.plan) == 0


def test_f32_error_over_many_steps(P):
    """FP32 batched path over 100 steps of a broadband vacuum field against the
    FP64 oracle (2x2x2 subdomains of 32^3, 16 guards, p = 64)."""
    wl = I.custom("bb100", (64, 64, 64), ((32, 32),) * 3, 16, 64, fields="broadband", precision="f32")
    glob = I.global_fields(wl)
    sol, _ = _run_gpu(P, wl, glob, 100)
    ref, _ = _oracle(wl, glob, 100)
    err = O.rel_l2(_np(sol.gather_global()), ref)
    print(f"FP32 100-step relative L2 error: {err:.3e}")
    assert err < 1e-5


@pytest.mark.parametrize("chunk", [1, 3, 5, 6])
def test_pass_b_chunk_widths(P, chunk):
    """Any chunk width of the z/Eq. 1 stage, odd ones included (element
    copies instead of 16-byte pairs), against the oracle."""
    wl = _mixed("f32")
    glob = I.global_fields(wl)
    sol = P.Solver(wl, tuning={"chunk_b": chunk, "f1": [0, 0, 0]})
    sol.load_global(glob, names=I.EB_NAMES, guards=False)
    sol.load_global(glob, names=("Jx", "Jy", "Jz", "rho"), guards=True)
    sol.exchange()
    for _ in range(2):
        sol.push()
    torch.cuda.synchronize()
    ref, _ = _oracle(wl, glob, 2)
    assert O.rel_l2(_np(sol.gather_global()), ref) < 4e-6
    assert P.psatd_check(sol.plan) == 0


@pytest.mark.parametrize("case", ["mixed_f32", "mixed_f64", "twod_f64", "wide_guard_f64"])
def test_scatter_gather_global_are_exact_copies(P, case):
    """psatd_scatter_global fills every padded box from the periodic global
    grid (valid cells and guard images, bit-exact against the oracle's box
    extraction); psatd_gather_global writes the valid cells back."""
    wl = {"mixed_f32": lambda: _mixed("f32"), "mixed_f64": lambda: _mixed("f64"),
          "twod_f64": lambda: CASES["twod_f64"][0](), "wide_guard_f64": lambda: CASES["wide_guard_f64"][0]()}[case]()
    glob = I.global_fields(wl)
    sol = P.Solver(wl)
    names = I.FIELD_NAMES
    dev = {n: glob[n].to("cuda", sol.dtype).contiguous() for n in names}
    P.psatd_scatter_global(sol.plan, [dev[n] for n in names], [sol.arenas[n] for n in names])
    torch.cuda.synchronize()
    for s, sd in enumerate(wl.subs):
        for n in names:
            exp = O.extract_box(dev[n].double().cpu().numpy(), sd.lo, sd.local, O.sub_guards(sd))
            assert np.array_equal(sol.box(n, s).double().cpu().numpy(), exp), (s, n)
    out = {n: torch.full_like(dev[n], float("nan")) for n in I.EB_NAMES}
    P.psatd_gather_global(sol.plan, [sol.arenas[n] for n in I.EB_NAMES], [out[n] for n in I.EB_NAMES])
    torch.cuda.synchronize()
    for n in I.EB_NAMES:
        assert torch.equal(out[n], dev[n]), n
