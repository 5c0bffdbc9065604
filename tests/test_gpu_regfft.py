"""The FP32 plane stages with thread-private transforms of compile-time
length (psatd_plane_engine == 1) against the FP64 oracle and against the
generic plane stages (PSATD_GENERIC_PLANES), on decompositions whose local x
and y lengths are all compiled in: uneven boxes, both guard widths, ragged
valid rows, per-subdomain orders, 2D, the plain schedule and the heat
equation.  Through the C ABI."""
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


def _np(d):
    return {k: v.numpy() if isinstance(v, torch.Tensor) else v for k, v in d.items()}


def _uneven(ng, cuts, nz, two_d=False):
    p = lambda ix, iy, iz: (8, 16, 0, 32)[(ix + 2 * iy + iz) % 4]
    zc = (1,) if two_d else nz
    subs = I.tensor_decomposition(cuts[0], cuts[1], zc, ng, p)
    if two_d:
        import dataclasses
        subs = [dataclasses.replace(sd, zguard=False) for sd in subs]
    g = (sum(cuts[0]), sum(cuts[1]), sum(zc))
    return I.Workload("reg", g, subs, "broadband", 2, "f32", 1707 + 31, c_dt=0.6, two_d=two_d)


# local x lengths n + 2 ng and y lengths all in the compiled sets (engine
# bit 1); in the "z" cases the local z lengths too, run with PSATD_PACKED_Z
# (bit 2: the packed z/Eq. 1 stage)
CASES = {
    "ng8": (lambda: _uneven(8, ((24, 40, 56, 72, 88), (16, 32, 48, 64, 80)), (17, 23)), 1),
    "ng16": (lambda: _uneven(16, ((16, 24, 32, 40, 56, 64, 72), (16, 32, 48, 64)), (20,)), 1),
    "twod": (lambda: _uneven(8, ((40, 24, 88), (80, 16, 32)), None, two_d=True), 1),
    "ng8z": (lambda: _uneven(8, ((24, 40), (16, 32)), (16, 32, 48)), 3),
    "ng16z": (lambda: _uneven(16, ((32, 64), (16, 48)), (16, 32, 48, 64)), 3),
}


def _run(P, wl, glob, steps, generic, plain=False, engine=1, gauss=False):
    flags = P.PSATD_GENERIC_PLANES if generic else (P.PSATD_PACKED_Z if engine & 2 else 0)
    sol = P.Solver(wl, plain=plain, extra_flags=flags, gauss=gauss)
    assert P.psatd_plane_engine(sol.plan) == (0 if generic else engine)
    sol.load_global(glob, names=I.EB_NAMES, guards=False)
    sol.load_global(glob, names=("Jx", "Jy", "Jz", "rho"), guards=True)
    sol.exchange()
    for _ in range(steps):
        sol.push()
    torch.cuda.synchronize()
    assert P.psatd_check(sol.plan) == 0
    return sol


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("name", list(CASES))
def test_compiled_length_planes_match_oracle_and_generic(P, name, plain):
    make, engine = CASES[name]
    wl = make()
    glob = I.global_fields(wl)
    steps = 2
    reg = _run(P, wl, glob, steps, generic=False, plain=plain, engine=engine)
    gen = _run(P, wl, glob, steps, generic=True, plain=plain)
    ref = _np(glob)
    for _ in range(steps):
        ref = O.step(ref, wl)
    err = O.rel_l2(_np(reg.gather_global()), ref)
    err_gen = O.rel_l2(_np(gen.gather_global()), ref)
    print(f"{name} plain={plain}: compiled-length {err:.3e}, generic {err_gen:.3e}")
    assert err < 4e-6 and err_gen < 4e-6
    # guard images hold the owners' values on both engines
    for s, sd in enumerate(wl.subs):
        for n in I.EB_NAMES:
            exp = O.extract_box(ref[n], sd.lo, sd.local, O.sub_guards(sd))
            scale = np.abs(exp).max()
            for sol in (reg, gen):
                assert np.abs(sol.box(n, s).double().cpu().numpy() - exp).max() < 4e-5 * scale, (name, s, n)


def test_compiled_length_planes_are_deterministic(P):
    wl = CASES["ng8z"][0]()
    glob = I.global_fields(wl)
    a = _run(P, wl, glob, 3, generic=False, engine=3)
    b = _run(P, wl, glob, 3, generic=False, engine=3)
    for n in I.EB_NAMES:
        assert torch.equal(a.arenas[n], b.arenas[n])


@pytest.mark.parametrize("source", [False, True])
def test_compiled_length_planes_heat(P, source):
    wl = _uneven(8, ((24, 40, 56), (16, 48)), (20,))
    g = I.random_fields(wl.global_n, 11, names=("Jx", "Jy"))
    hs = P.HeatSolver(wl, 0.45, source=source)
    assert P.psatd_plane_engine(hs.plan) == 1
    names = ("T", "S") if source else ("T",)
    hs.load_global({"T": g["Jx"], "S": 0.1 * g["Jy"]}, names=names, guards=True)
    for _ in range(2):
        hs.push()
    torch.cuda.synchronize()
    ref = {"T": g["Jx"].numpy()}
    if source:
        ref["S"] = 0.1 * g["Jy"].numpy()
    ref = H.heat_run(ref, wl, 0.45, 2)["T"]
    err = H.rel_l2(hs.gather_global(names=("T",))["T"].numpy(), ref)
    assert err < 4e-6, err


@pytest.mark.parametrize("staggered", [False, True])
def test_compiled_length_z_stage_gauss_and_stagger(P, staggered):
    """The packed z/Eq. 1 stage (PSATD_PACKED_Z) with the Gauss diagnostic
    (ten fields) and with Yee-staggered components (phase shifts inside
    Eq. 1), against the oracle: fields and per-subdomain Gauss sums."""
    import dataclasses
    wl = dataclasses.replace(_uneven(8, ((24, 40), (16, 32)), (16, 32)), staggered=staggered, fields="wavepacket")
    glob = I.global_fields(wl)
    sol = _run(P, wl, glob, 0, generic=False, engine=3, gauss=True)
    sums = []
    for _ in range(2):
        sol.push()
        torch.cuda.synchronize()
        sums.append(sol.gauss_sums().copy())
    ref = _np(glob)
    osum = []
    for _ in range(2):
        gs = []
        ref = O.step(ref, wl, gauss_out=gs)
        osum.append(np.array(gs))
    err = O.rel_l2(_np(sol.gather_global()), ref)
    assert err < 4e-6, err
    for a, b in zip(sums, osum):
        np.testing.assert_allclose(a[:, 1], b[:, 1], rtol=1e-3)
        np.testing.assert_allclose(a[:, 0], b[:, 0], rtol=1e-3)
