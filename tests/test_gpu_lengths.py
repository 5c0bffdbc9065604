"""Local lengths that have no split into two factors <= 16 and are done in
three (n = f1 f2 f3, e.g. 216 = 12 x 6 x 3, 512 = 16 x 8 x 4 for a 1024-long
real x axis), against the FP64 oracle through the C ABI: along x (the real
split walks the three-factor position order), y and z, in FP64 and FP32,
batched, plain and split-plane schedules."""
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


CASES = {
    # local y = 200 + 2*8 = 216 on both subdomains
    "y216": lambda prec: I.custom("y216", (32, 400, 16), ((32,), (200, 200), (16,)), 8, 8, fields="wavepacket",
                                  precision=prec),
    # local z = 216
    "z216": lambda prec: I.custom("z216", (32, 16, 400), ((32,), (16,), (200, 200)), 8, 8, fields="wavepacket",
                                  precision=prec),
    # one periodic box, x = 1024 (packed half length 512), no guards
    "x1024": lambda prec: I.custom("x1024", (1024, 8, 8), ((1024,), (8,), (8,)), 0, 0, fields="broadband",
                                   precision=prec),
    # local x = 416 + 2*8 = 432 (half length 216)
    "x432": lambda prec: I.custom("x432", (416, 16, 16), ((416,), (16,), (16,)), 8, 16, fields="wavepacket",
                                  precision=prec),
}


@pytest.mark.parametrize("schedule", ["batched", "plain", "split"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 4e-6)])
@pytest.mark.parametrize("name", list(CASES))
def test_three_factor_lengths_match_oracle(P, name, prec, tol, schedule):
    wl = CASES[name](prec)
    glob = I.global_fields(wl)
    flags = P.PSATD_SPLIT_PLANES if schedule == "split" else 0
    sol = P.Solver(wl, plain=schedule == "plain", extra_flags=flags)
    sol.load_global(glob, names=I.EB_NAMES, guards=False)
    sol.load_global(glob, names=("Jx", "Jy", "Jz", "rho"), guards=True)
    sol.exchange()
    for _ in range(2):
        sol.push()
    torch.cuda.synchronize()
    assert P.psatd_check(sol.plan) == 0
    ref = _np(glob)
    for _ in range(2):
        ref = O.step(ref, wl)
    err = O.rel_l2(_np(sol.gather_global()), ref)
    assert err < tol, (name, prec, schedule, err)
