"""Full-size FP32 trajectories against the FP64 oracle, through the C ABI, in
the launch configuration bench.py times (batched, persistent grids).

* uneven48 (the batching workload): 50 FP32 steps on the GPU against 50
  oracle steps of the whole grid.
* broadband256 (the precision workload): 100 FP32 steps against the
  oracle's 100-step trajectory at 2048 sampled cells per component, written
  by tests/golden/make_trajectory_golden.py (oracle only).
* mirror1024 (the plasma-mirror-shaped workload): the GPU's FP32 state at
  steps 50 and 99, pushed once more by the oracle on sampled subdomains and
  compared with the GPU's next step.

Each reports the stacked relative L2 error of the six E/B components and,
per component, the largest error relative to that component's largest
magnitude (Sec. 3.1 Eq. 1 advanced with the decomposition of Sec. 3.2 /
Fig. 3)."""
import os

import numpy as np
import pytest
import torch

from oracle import psatd_oracle as O
from paper_1707_08500_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "broadband256_trajectory.txt")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_08500_gb300 import build
    build.build()
    from paper_1707_08500_gb300 import psatd
    return psatd


def _np(d):
    return {k: v.numpy() for k, v in d.items()}


def _errors(got, ref):
    """(stacked relative L2, {component: max |got - ref| / max |ref|})."""
    num = sum(float(np.sum((np.asarray(got[n], np.float64) - ref[n]) ** 2)) for n in I.EB_NAMES)
    den = sum(float(np.sum(np.asarray(ref[n], np.float64) ** 2)) for n in I.EB_NAMES)
    comp = {n: float(np.abs(np.asarray(got[n], np.float64) - ref[n]).max() / np.abs(ref[n]).max())
            for n in I.EB_NAMES}
    return (num / den) ** 0.5, comp


def _run_gpu(P, wl, glob, steps):
    sol = P.Solver(wl, gauss=True)
    sol.load_global(glob, names=I.EB_NAMES, guards=False)
    sol.load_global(glob, names=("Jx", "Jy", "Jz", "rho"), guards=True)
    sol.exchange()
    for _ in range(steps):
        sol.push()
    torch.cuda.synchronize()
    assert P.psatd_check(sol.plan) == 0
    return sol


def test_uneven48_50_steps_f32(P):
    wl = I.workload("uneven48")
    glob = I.global_fields(wl)
    sol = _run_gpu(P, wl, glob, 50)
    ref = O.run(_np(glob), wl, 50)
    l2, comp = _errors(_np(sol.gather_global()), ref)
    print(f"uneven48 FP32 after 50 steps: rel L2 {l2:.3e}; per-component max "
          + ", ".join(f"{n} {v:.2e}" for n, v in comp.items()))
    assert l2 < 1e-5
    assert max(comp.values()) < 1e-4


def test_broadband256_100_steps_f32_sampled(P):
    wl = I.workload("broadband256")
    with open(GOLDEN) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    steps = int(rows[0][1])
    data = np.array([[float(v) for v in r] for r in rows[1:]])
    z, y, x = (data[:, i].astype(int) for i in range(3))
    ref = {n: data[:, 3 + i] for i, n in enumerate(I.EB_NAMES)}
    glob = I.global_fields(wl)
    sol = _run_gpu(P, wl, glob, steps)
    g = sol.gather_global()
    got = {n: g[n].numpy()[z, y, x] for n in I.EB_NAMES}
    l2, comp = _errors(got, ref)
    print(f"broadband256 FP32 after {steps} steps at {len(z)} sampled cells: rel L2 {l2:.3e}; per-component max "
          + ", ".join(f"{n} {v:.2e}" for n, v in comp.items()))
    assert steps == 100
    assert l2 < 1e-5
    assert max(comp.values()) < 1e-4


def test_mirror1024_one_oracle_step_from_gpu_states(P):
    """At steps 50 and 99 of the GPU's FP32 trajectory, the oracle pushes the
    GPU's padded boxes of sampled subdomains (in the laser, in the slab, at
    the periodic corner) once; the GPU's next step must agree on their valid
    cells (error normalised by the pushed box, as in the one-step checks)."""
    wl = I.workload("mirror1024")
    dev = torch.device("cuda")
    sol = P.Solver(wl, gauss=True)
    for s, sd in enumerate(wl.subs):
        b = I.box_fields(wl, sd, device=dev)
        for n in I.FIELD_NAMES:
            sol.box(n, s).copy_(b[n])
        del b
    laser = next(s for s, sd in enumerate(wl.subs) if sd.lo == (256, 192, 192))
    slab = next(s for s, sd in enumerate(wl.subs) if sd.lo == (640, 256, 256))
    samples = [0, laser, slab]
    done = 0
    for at in (50, 99):
        while done < at:
            sol.push()
            done += 1
        torch.cuda.synchronize()
        boxes = {s: {n: sol.box(n, s).double().cpu().numpy() for n in I.FIELD_NAMES} for s in samples}
        sol.push()
        done += 1
        torch.cuda.synchronize()
        for s in samples:
            sd = wl.subs[s]
            out, _ = O.local_push(boxes[s], sd.local, wl.dx, sd.p, wl.c_dt, wl.staggered)
            g = O.sub_guards(sd)
            sel = np.s_[g[2]:g[2] + sd.n[2], g[1]:g[1] + sd.n[1], g[0]:g[0] + sd.n[0]]
            got = {n: sol.box(n, s).double().cpu().numpy()[sel] for n in I.EB_NAMES}
            num = sum(float(((got[n] - out[n][sel]) ** 2).sum()) for n in I.EB_NAMES)
            den = sum(float((out[n] ** 2).sum()) for n in I.EB_NAMES)
            err = (num / den) ** 0.5
            print(f"mirror1024 step {at} -> {at + 1}, subdomain {s}: rel L2 {err:.3e}")
            assert err < 2e-6, (at, s, err)
    assert P.psatd_check(sol.plan) == 0
