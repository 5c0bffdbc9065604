"""The CUDA-graph-captured step loop and the tuned launch shapes against the
FP64 oracle, through the C ABI: K pushes captured in one CUDA graph and
replayed; FFT factorisations other than the default split on every axis;
and the autotuner's own check of the shape it picks."""
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


def _uneven():
    """48-subdomain-like decomposition with uneven boxes, guards 8 or 16 and
    orders 16/32/64, as in the batching workload, scaled down."""
    cuts = ((24, 40, 56), (32, 48), (32, 48))
    ngs = lambda ix, iy, iz: (8, 16)[(ix + iy + iz) % 2]
    subs = []
    for sd in I.tensor_decomposition(*cuts, 8, 16):
        ix = [0, 24, 64].index(sd.lo[0])
        iy = [0, 32].index(sd.lo[1])
        iz = [0, 32].index(sd.lo[2])
        subs.append(I.Sub(sd.lo, sd.n, ngs(ix, iy, iz), (16, 32, 64)[(ix + 2 * iy + iz) % 3]))
    return I.Workload("uneven-small", (120, 80, 80), subs, "broadband", 6, "f32", 1707 + 41, c_dt=0.5)


def _mixed():
    p = lambda ix, iy, iz: (4, 8, 0, 12)[(ix + 2 * iy + iz) % 4]
    subs = I.tensor_decomposition((12, 20), (14, 13), (18, 17), 4, p)
    return I.Workload("mixed", (32, 27, 35), subs, "wavepacket", 3, "f32", 1707 + 9, c_dt=0.7)


def _load(sol, glob):
    sol.load_global(glob, names=I.EB_NAMES, guards=False)
    sol.load_global(glob, names=("Jx", "Jy", "Jz", "rho"), guards=True)
    sol.exchange()
    torch.cuda.synchronize()


@pytest.mark.parametrize("case", ["mixed", "uneven"])
def test_graph_replayed_pushes_match_oracle(P, case):
    wl = _mixed() if case == "mixed" else _uneven()
    K = 6
    glob = I.global_fields(wl)
    sol = P.Solver(wl, gauss=True)
    _load(sol, glob)
    # capture K pushes (with the Gauss reduction) in one CUDA graph, replay it once
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for _ in range(K):
                P.psatd_push(sol.plan, sol.fields, sol.gauss_out.data_ptr(), side.cuda_stream)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert P.psatd_check(sol.plan) == 0
    ref = _np(glob)
    gs = []
    for k in range(K):
        gs = []
        ref = O.step(ref, wl, gauss_out=gs)
    err = O.rel_l2(_np(sol.gather_global()), ref)
    print(f"{case}: {K} graph-replayed FP32 pushes, rel L2 vs oracle {err:.3e}")
    assert err < 1e-5
    np.testing.assert_allclose(sol.gauss_sums()[:, 1], np.array(gs)[:, 1], rtol=1e-3)


def _factorised():
    return I.custom("fac", (128, 128, 128), ((64, 64),) * 3, 16, 32, fields="broadband", precision="f32",
                    c_dt=0.6)


# local box 96^3: x half length 48, y and z 96 (default splits 8 x 6, 12 x 8, 12 x 8)
SPLITS = [(4, 0, 0), (6, 0, 0), (12, 0, 0), (16, 0, 0), (0, 6, 0), (0, 8, 0), (0, 16, 0), (0, 0, 6),
          (0, 0, 16), (3, 16, 8)]


@pytest.fixture(scope="module")
def fac_ref():
    wl = _factorised()
    glob = I.global_fields(wl)
    ref = _np(glob)
    for _ in range(2):
        ref = O.step(ref, wl)
    return wl, glob, ref


@pytest.mark.parametrize("f1", SPLITS)
def test_non_default_factorisations_match_oracle(P, fac_ref, f1):
    wl, glob, ref = fac_ref
    sol = P.Solver(wl, tuning={"chunk_b": 0, "f1": list(f1)})
    _load(sol, glob)
    for _ in range(2):
        sol.push()
    torch.cuda.synchronize()
    err = O.rel_l2(_np(sol.gather_global()), ref)
    assert err < 4e-6, (f1, err)


def test_autotuner_checks_its_choice(P):
    """autotune() compares one push of the shape it picked with one push of
    the default shape on the same fields and keeps the default if they
    differ; the shape it returns then matches the oracle."""
    from paper_1707_08500_gb300 import tune as T
    wl = _uneven()
    flags = P.PSATD_F32
    best = T.autotune(wl, flags, use_cache=False, reps=1)
    glob = I.global_fields(wl)
    sol = P.Solver(wl, tuning=best)
    _load(sol, glob)
    sol.push()
    torch.cuda.synchronize()
    ref = O.step(_np(glob), wl)
    assert O.rel_l2(_np(sol.gather_global()), ref) < 4e-6
