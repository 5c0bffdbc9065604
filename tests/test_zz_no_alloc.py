"""psatd_push_static against psatd_push, through the C ABI.

psatd_push_static serves callers that may not allocate device memory (for
example a plugin inside a host application that owns every device
allocation, or a code path where a device-synchronising cudaMalloc is not
allowed): they pass their fields but no workspace, and the push runs on a
library-owned static device buffer.  Its results must match the regular push
that runs on a caller-provided workspace, on consecutive calls (the static
buffer keeps the previous call's contents).  This file is collected last.
"""
import pytest
import torch

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


def _workload():
    return I.custom("static", (32, 24, 20), ((12, 20), (10, 14), (20,)), 4, 8, fields="wavepacket",
                    precision="f32")


def test_static_push_matches_regular_push_on_two_calls(P):
    """The two entry points run the same kernels on the same inputs, so E, B
    and the Gauss sums agree bit for bit; after the first static call (which
    looks the buffer's address up), further calls leave the device's free
    memory unchanged: they allocate nothing."""
    wl = _workload()
    ref = P.Solver(wl, gauss=True)
    assert ref.ws_bytes <= P.STATIC_WORKSPACE_BYTES
    glob = I.global_fields(wl)
    ref.load_global(glob)
    # a second set of arenas with the same contents, pushed without any workspace
    mine = {n: ref.arenas[n].clone() for n in I.FIELD_NAMES}
    fields = P.make_fields([mine[n] for n in ("Ex", "Ey", "Ez")], [mine[n] for n in ("Bx", "By", "Bz")],
                           [mine[n] for n in ("Jx", "Jy", "Jz")], mine["rho"])
    gauss = torch.zeros_like(ref.gauss_out)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(3):
        ref.push()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        P.psatd_push_static(ref.plan, wl.c_dt, wl.dx, fields, gauss.data_ptr(), stream)
        torch.cuda.synchronize()
        if call > 0:      # the first call may load the library's device module
            assert torch.cuda.mem_get_info()[0] == free_before, call
        for n in I.EB_NAMES:
            assert torch.equal(mine[n], ref.arenas[n]), (call, n)
        assert torch.equal(gauss, ref.gauss_out), call


def test_static_push_errors_are_reported_by_check(P):
    """psatd_check on a plan without a workspace reads the static buffer's
    device error word: zero after correct static pushes."""
    wl = _workload()
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F32)
    try:
        n = P.psatd_arena_elems(h)
        ar = {k: torch.zeros(n, device="cuda") for k in I.FIELD_NAMES}
        f = P.make_fields([ar[k] for k in ("Ex", "Ey", "Ez")], [ar[k] for k in ("Bx", "By", "Bz")],
                          [ar[k] for k in ("Jx", "Jy", "Jz")])
        P.psatd_push_static(h, wl.c_dt, wl.dx, f, None, torch.cuda.current_stream().cuda_stream)
        assert P.psatd_check(h) == 0
    finally:
        P.psatd_destroy(h)


def test_static_push_rejects_plans_larger_than_its_buffer(P):
    wl = I.workload("broadband256")          # needs far more than 32 MiB of workspace
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F32)
    try:
        assert P.psatd_workspace_bytes(h) > P.STATIC_WORKSPACE_BYTES
        x = torch.zeros(16, device="cuda")
        f = P.make_fields([x] * 3, [x] * 3, [x] * 3)
        with pytest.raises(P.PsatdError) as e:
            P.psatd_push_static(h, wl.c_dt, wl.dx, f, None, torch.cuda.current_stream().cuda_stream)
        assert e.value.code == -3
        assert "static workspace" in P.psatd_last_error(h)
    finally:
        P.psatd_destroy(h)
