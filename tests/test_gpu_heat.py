"""Parity of the local-FFT heat equation (PSATD_HEAT, through the C ABI) with
the FP64 heat oracle: uneven mixed-radix decompositions with and without a
source, infinite and finite order, 2D, the plain and split-plane schedules,
FP64 to 1e-12 and FP32 to 1e-5; the guards hold the owners' values."""
import numpy as np
import pytest
import torch

from oracle import heat_oracle as H
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


def _mixed(precision, two_d=False):
    if two_d:
        return I.custom("h2", (48, 30, 1), ((30, 18), (16, 14), (1,)), 6, 8, precision=precision, two_d=True)
    p = lambda ix, iy, iz: (4, 8, 0, 12)[(ix + 2 * iy + iz) % 4]
    subs = I.tensor_decomposition((12, 20), (14, 13), (18, 17), 4, p)
    return I.Workload("hmix", (32, 27, 35), subs, "broadband", 3, precision, 1707 + 70, dx=(1.0, 0.9, 1.1))


CASES = [
    ("mixed_f64_src", lambda: _mixed("f64"), True, 3, 1e-12),
    ("mixed_f64", lambda: _mixed("f64"), False, 3, 1e-12),
    ("mixed_f32_src", lambda: _mixed("f32"), True, 3, 1e-5),
    ("twod_f64_src", lambda: _mixed("f64", two_d=True), True, 4, 1e-12),
    ("box_f64_exact_k", lambda: I.custom("hb", (32, 24, 20), ((16, 16), (24,), (20,)), 8, 0, precision="f64"),
     True, 3, 1e-12),
]


@pytest.mark.parametrize("name,make,source,steps,tol", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("schedule", ["batched", "plain", "split"])
def test_heat_matches_oracle(P, name, make, source, steps, tol, schedule):
    wl = make()
    d_dt = 0.45
    nx, ny, nz = wl.global_n
    g = I.random_fields(wl.global_n, 1707 + 71, names=("Jx", "Jy"))
    glob = {"T": g["Jx"], "S": 0.1 * g["Jy"]} if source else {"T": g["Jx"]}
    sol = P.HeatSolver(wl, d_dt, source=source, plain=schedule == "plain",
                       extra_flags=P.PSATD_SPLIT_PLANES if schedule == "split" else 0)
    sol.load_global(glob, names=tuple(glob), guards=True)
    for _ in range(steps):
        sol.push()
    torch.cuda.synchronize()
    got = sol.gather_global(names=("T",))["T"].numpy()
    ref = H.heat_run({k: v.numpy() for k, v in glob.items()}, wl, d_dt, steps)
    err = H.rel_l2(got, ref["T"])
    print(f"heat {name} {schedule}: rel L2 {err:.3e}")
    assert err < tol
    for s, sd in enumerate(wl.subs):
        exp = O.extract_box(ref["T"], sd.lo, sd.local, O.sub_guards(sd))
        box = sol.box("T", s).double().cpu().numpy()
        assert np.abs(box - exp).max() < 50 * tol * max(np.abs(exp).max(), 1e-30), (s,)
