"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every symbol declared in include/psatd.h, and plan creation validates the
decomposition (Sec. 3.2) without touching a device."""
import os
import re
import subprocess

import pytest

from paper_1707_08500_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1707_08500_gb300 import build
    build.build()
    from paper_1707_08500_gb300 import psatd
    psatd.lib()
    return psatd


def _declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"\b(psatd_[a-z_]+)\s*\(", src)))


def test_header_declarations_are_exported(P):
    names = _declared()
    assert "psatd_push" in names and "psatd_plan_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (psatd_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(P.lib(), n)
    assert set(P.EXPORTS) == set(names)


def test_plan_counts_for_every_workload(P):
    for name in I.WORKLOADS:
        wl = I.workload(name)
        flags = P.PSATD_F64 if wl.precision == "f64" else P.PSATD_F32
        if wl.staggered:
            flags |= P.PSATD_STAGGERED
        h = P.psatd_plan_create(wl.global_n, wl.subs, flags)
        try:
            n = P.psatd_arena_elems(h)
            assert n >= wl.local_cells
            for s in (0, len(wl.subs) - 1):
                off, ln = P.psatd_layout(h, s)
                assert ln == wl.subs[s].local
                assert off % 64 == 0 and off + ln[0] * ln[1] * ln[2] <= n
            assert P.psatd_workspace_bytes(h) > 0
            assert P.psatd_push_launches(h) in (3, 4)
        finally:
            P.psatd_destroy(h)


def test_plain_schedule_launch_count(P):
    wl = I.workload("yee64")
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F64 | P.PSATD_STAGGERED | P.PSATD_PLAIN)
    assert P.psatd_push_launches(h) == 3 * 8 + 1
    P.psatd_destroy(h)


@pytest.mark.parametrize("case,code", [
    ("overlap", -2), ("gap", -2), ("outside", -2), ("odd_order", -2),
    ("odd_local_x", -5), ("big_prime", -5), ("no_precision", -1), ("both_precisions", -1), ("no_subdomains", -1),
    ("unknown_flag", -1), ("negative_guard", -2), ("empty_global", -2), ("empty_subdomain", -2),
    ("negative_global", -2), ("two_d_with_z", -2),
])
def test_plan_rejects_bad_input(P, case, code):
    g = (32, 32, 32)
    subs = I.tensor_decomposition([16, 16], [32], [32], 4, 8)
    flags = P.PSATD_F32
    if case == "overlap":
        subs = [subs[0], I.Sub((8, 0, 0), (24, 32, 32), 4, 8)]
    elif case == "gap":
        subs = [subs[0]]
    elif case == "outside":
        subs = [subs[0], I.Sub((16, 0, 0), (17, 32, 32), 4, 8)]
    elif case == "odd_order":
        subs = [I.Sub(s.lo, s.n, s.ng, 7) for s in subs]
    elif case == "odd_local_x":
        subs = I.tensor_decomposition([15, 17], [32], [32], 4, 8)
    elif case == "big_prime":
        g = (32, 34, 32)
        subs = I.tensor_decomposition([16, 16], [34], [32], 4, 8)     # 42 = 2*3*7 ok, use 17 below
        subs = [I.Sub(s.lo, s.n, 0, 8) for s in subs]                 # local y = 34 = 2*17: no split
    elif case == "no_precision":
        flags = 0
    elif case == "both_precisions":
        flags = P.PSATD_F32 | P.PSATD_F64
    elif case == "no_subdomains":
        subs = []
    elif case == "unknown_flag":
        flags = P.PSATD_F32 | 0x4000
    elif case == "negative_guard":
        subs = [I.Sub(s.lo, s.n, -1, 8) for s in subs]
    elif case == "empty_global":
        g = (0, 32, 32)
    elif case == "empty_subdomain":
        subs = [I.Sub((0, 0, 0), (32, 32, 0), 0, 8)]
    elif case == "negative_global":
        g = (-4, 32, 32)
    elif case == "two_d_with_z":
        flags |= P.PSATD_2D
    with pytest.raises(P.PsatdError) as e:
        P.psatd_plan_create(g, subs, flags)
    assert e.value.code == code


def test_status_strings(P):
    for c in (0, -1, -2, -3, -4, -5, -6, -7):
        assert P.psatd_status_string(c)
    assert P.psatd_status_string(-99) == "unknown status"


def test_state_errors_without_gpu(P):
    wl = I.workload("plain32")
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F64)
    f = P.FieldsT()
    with pytest.raises(P.PsatdError) as e:
        P.psatd_push(h, f)
    assert e.value.code == -6            # no workspace yet
    with pytest.raises(P.PsatdError) as e:
        P.psatd_set_coeffs(h, 0.5, (1.0, 1.0, 1.0))
    assert e.value.code == -6
    with pytest.raises(P.PsatdError) as e:
        P.psatd_check(h)                            # no workspace to read the error word from
    assert e.value.code == -6
    with pytest.raises(P.PsatdError) as e:
        P.psatd_set_workspace(h, 0x1001, 1 << 30)   # misaligned: rejected before any copy
    assert e.value.code == -1
    with pytest.raises(P.PsatdError) as e:
        P.psatd_set_workspace(h, 0x1000, 16)        # too small
    assert e.value.code == -3
    P.psatd_destroy(h)


def test_exchange_segments_cover_every_local_cell_once(P):
    """Host bookkeeping of the guard exchange: the plan's arena size and the
    tiling checks accept guard widths larger than a neighbour's width."""
    g = (40, 16, 16)
    subs = I.tensor_decomposition([8, 32], [16], [16], 10, 4)
    h = P.psatd_plan_create(g, subs, P.PSATD_F32)
    assert P.psatd_layout(h, 0)[1] == (28, 36, 36)
    P.psatd_destroy(h)


def test_fixed_geometry_kernels_are_selected_for_cubic_boxes(P):
    G = P.PSATD_GENERIC_PLANES      # the FP32 generic kernels (the compiled-length ones take 6 modes per item)
    cases = [("mirror1024", P.PSATD_F32 | G, 0), ("broadband256", P.PSATD_F32 | G, 0), ("mirror1024", P.PSATD_F64, 0),
             ("yee64", P.PSATD_F64 | P.PSATD_STAGGERED, 1), ("plain32", P.PSATD_F64, 2), ("uneven48", P.PSATD_F32 | G, -2)]
    for name, flags, want in cases:
        wl = I.workload(name)
        h = P.psatd_plan_create(wl.global_n, wl.subs, flags)
        try:
            assert P.psatd_geometry_variant(h) == want, name
        finally:
            P.psatd_destroy(h)
    # a non-default split falls back to the descriptor-driven kernels (with
    # the default chunk width compiled in), a non-default chunk width to the
    # fully descriptor-driven ones
    wl = I.workload("broadband256")
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F32 | G, {"chunk_b": 8, "f1": [4, 0, 0]})
    assert P.psatd_geometry_variant(h) == -2
    P.psatd_destroy(h)
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F32 | G, {"chunk_b": 6, "f1": [4, 0, 0]})
    assert P.psatd_geometry_variant(h) == -1
    P.psatd_destroy(h)


def test_two_d_plans(P):
    """PSATD_2D: one cell along z, no guards along z (the local box is
    (nx + 2 ng, ny + 2 ng, 1)); a 3D global grid is rejected."""
    wl = I.custom("p2", (64, 32, 1), ((40, 24), (32,), (1,)), 8, 32, two_d=True)
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F32 | P.PSATD_2D)
    try:
        assert P.psatd_layout(h, 0)[1] == (56, 48, 1)
        assert P.psatd_layout(h, 1)[1] == (40, 48, 1)
        assert P.psatd_geometry_variant(h) == -1
    finally:
        P.psatd_destroy(h)
    subs = I.tensor_decomposition([16, 16], [32], [32], 4, 8)
    with pytest.raises(P.PsatdError) as e:
        P.psatd_plan_create((32, 32, 32), subs, P.PSATD_F32 | P.PSATD_2D)
    assert e.value.code == -2


def test_split_plane_schedule_is_chosen_for_large_planes(P):
    """One box over a 256^3 grid (PSATD-global, Fig. 2b): its (x, y) plane
    does not fit in shared memory, so the plan takes the five-stage
    split-plane schedule; a 64^3 box takes it only when forced."""
    g = (256, 256, 256)
    subs = [I.Sub((0, 0, 0), g, 0, 64)]
    for flags, want in ((P.PSATD_F32, 5), (P.PSATD_F64, 5), (P.PSATD_F32 | P.PSATD_GAUSS_DIAG, 6),
                        (P.PSATD_F32 | P.PSATD_PLAIN, 5)):
        h = P.psatd_plan_create(g, subs, flags)
        try:
            assert P.psatd_push_launches(h) == want
            assert P.psatd_geometry_variant(h) == -1
            assert P.psatd_layout(h, 0)[1] == g
        finally:
            P.psatd_destroy(h)
    wl = I.workload("broadband256")
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F32)
    assert P.psatd_push_launches(h) == 3
    P.psatd_destroy(h)
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F32 | P.PSATD_SPLIT_PLANES)
    assert P.psatd_push_launches(h) == 5 and P.psatd_geometry_variant(h) == -1
    P.psatd_destroy(h)
    # lengths beyond 16 x 16 take three factors: a 1024-long x axis is
    # accepted; a length with a prime factor above 16 is not
    h = P.psatd_plan_create((1024, 256, 256), [I.Sub((0, 0, 0), (1024, 256, 256), 0, 0)], P.PSATD_F32)
    P.psatd_destroy(h)
    with pytest.raises(P.PsatdError) as e:
        P.psatd_plan_create((1024, 34 * 8, 256), [I.Sub((0, 0, 0), (1024, 34 * 8, 256), 0, 0)], P.PSATD_F32)
    assert e.value.code == -5


@pytest.mark.parametrize("case", ["flags", "both", "shape", "dx", "null", "misaligned", "overlap_in", "overlap_out",
                                  "too_tall"])
def test_yee_step_rejects_bad_arguments(P, case):
    """Argument checks of psatd_yee_step run before any CUDA call."""
    n, flags, dx = [16, 16, 16], P.PSATD_F32, [1.0, 1.0, 1.0]
    bytes_ = 16 * 16 * 16 * 4
    base = 1 << 40
    fin, fout = P.FieldsT(), P.FieldsT()
    for a in range(3):
        fin.E[a], fin.B[a], fin.J[a] = base + a * bytes_, base + (3 + a) * bytes_, base + (6 + a) * bytes_
        fout.E[a], fout.B[a] = base + (9 + a) * bytes_, base + (12 + a) * bytes_
    if case == "flags":
        flags |= P.PSATD_STAGGERED
    elif case == "both":
        flags = P.PSATD_F32 | P.PSATD_F64
    elif case == "shape":
        n[1] = 0
    elif case == "dx":
        dx[2] = -1.0
    elif case == "null":
        fin.J[2] = None
    elif case == "misaligned":
        fout.B[1] += 4
    elif case == "overlap_in":
        fout.E[0] = fin.B[2] + 64
    elif case == "overlap_out":
        fout.B[2] = fout.E[1]
    elif case == "too_tall":
        n = [1, 1 << 20, 1]
    with pytest.raises(P.PsatdError) as e:
        P.psatd_yee_step(n, flags, 0.5, dx, fin, fout)
    assert e.value.code == (-2 if case in ("shape", "too_tall") else -1)
    assert P.psatd_yee_launches() == 1


def test_heat_plans(P):
    """PSATD_HEAT: one field in (two with a source), one out; the Maxwell-only
    flags are rejected."""
    g = (32, 32, 32)
    subs = I.tensor_decomposition([16, 16], [32], [32], 4, 8)
    for flags in (P.PSATD_F32 | P.PSATD_HEAT, P.PSATD_F64 | P.PSATD_HEAT | P.PSATD_HEAT_SOURCE,
                  P.PSATD_F32 | P.PSATD_HEAT | P.PSATD_PLAIN, P.PSATD_F32 | P.PSATD_HEAT | P.PSATD_SPLIT_PLANES):
        h = P.psatd_plan_create(g, subs, flags)
        try:
            assert P.psatd_layout(h, 0)[1] == (24, 40, 40)
            maxwell = P.psatd_plan_create(g, subs, flags & ~(P.PSATD_HEAT | P.PSATD_HEAT_SOURCE))
            assert P.psatd_workspace_bytes(h) < P.psatd_workspace_bytes(maxwell)
            assert P.psatd_push_launches(h) == P.psatd_push_launches(maxwell)
            P.psatd_destroy(maxwell)
        finally:
            P.psatd_destroy(h)
    for flags in (P.PSATD_F32 | P.PSATD_HEAT_SOURCE, P.PSATD_F32 | P.PSATD_HEAT | P.PSATD_STAGGERED,
                  P.PSATD_F32 | P.PSATD_HEAT | P.PSATD_GAUSS_DIAG):
        with pytest.raises(P.PsatdError) as e:
            P.psatd_plan_create(g, subs, flags)
        assert e.value.code == -1


def test_scatter_gather_argument_checks(P):
    wl = I.workload("plain32")
    h = P.psatd_plan_create(wl.global_n, wl.subs, P.PSATD_F64)
    try:
        with pytest.raises(P.PsatdError) as e:
            P.psatd_scatter_global(h, [0x1000], [0x2000])     # no workspace yet
        assert e.value.code == -6
        with pytest.raises(P.PsatdError) as e:
            P.psatd_gather_global(h, [0x1000] * 11, [0x2000] * 11)
        assert e.value.code == -1
    finally:
        P.psatd_destroy(h)


@pytest.mark.parametrize("name", ["mixed", "wide_guard", "two_d", "uneven48", "one_box", "thin", "guard_wider_than_grid"])
def test_exchange_segments_write_every_local_cell_once_from_its_owner(P, name):
    """Host check of the plan's guard exchange (Fig. 3 step 3): every local
    cell of every padded box is the destination of exactly one segment cell,
    whose source is a valid cell of the subdomain that owns the same global
    cell (global index modulo the periodic grid)."""
    import numpy as np
    from oracle import psatd_oracle as O
    two_d = False
    if name == "mixed":
        g, subs = (32, 27, 35), I.tensor_decomposition((12, 20), (14, 13), (18, 17), 4, 8)
    elif name == "wide_guard":
        g, subs = (40, 16, 16), I.tensor_decomposition([8, 32], [16], [16], 10, 6)
    elif name == "two_d":
        wl = I.custom("t2", (48, 30, 1), ((30, 18), (16, 14), (1,)), 6, 16, two_d=True)
        g, subs, two_d = wl.global_n, wl.subs, True
    elif name == "uneven48":
        wl = I.workload("uneven48")
        g, subs = wl.global_n, wl.subs
    elif name == "one_box":
        g, subs = (16, 12, 8), [I.Sub((0, 0, 0), (16, 12, 8), 3, 8)]
    elif name == "thin":
        g, subs = (20, 12, 12), I.tensor_decomposition([2, 18], [12], [12], 3, 6)
    else:                        # guards wrap around the periodic grid more than once
        g, subs = (8, 6, 4), I.tensor_decomposition([4, 4], [6], [4], 10, 4)
    h = P.psatd_plan_create(g, subs, P.PSATD_F32 | (P.PSATD_2D if two_d else 0))
    try:
        segs = P.psatd_exchange_segments(h)
    finally:
        P.psatd_destroy(h)
    owner = O.owner_map(g, subs)                     # [Nz][Ny][Nx] -> owning subdomain
    guards = [O.sub_guards(sd) for sd in subs]
    cover = [np.zeros(sd.local[::-1], dtype=np.int32) for sd in subs]
    for (src, dst, x0, y0, z0, ex, ey, ez, dx, dy, dz, ident) in segs:
        s, d = subs[src], subs[dst]
        gs, gd = guards[src], guards[dst]
        # source cells are valid cells of the source subdomain
        assert gs[0] <= x0 and x0 + ex <= gs[0] + s.n[0]
        assert gs[1] <= y0 and y0 + ey <= gs[1] + s.n[1]
        assert gs[2] <= z0 and z0 + ez <= gs[2] + s.n[2]
        assert not ident or (src == dst and (dx, dy, dz) == (0, 0, 0))
        zz, yy, xx = np.meshgrid(np.arange(z0, z0 + ez), np.arange(y0, y0 + ey), np.arange(x0, x0 + ex), indexing="ij")
        # the destination cell images the same global cell, which the source owns
        gsx, gsy, gsz = (s.lo[0] - gs[0] + xx) % g[0], (s.lo[1] - gs[1] + yy) % g[1], (s.lo[2] - gs[2] + zz) % g[2]
        tx, ty, tz = xx + dx, yy + dy, zz + dz
        gdx, gdy, gdz = (d.lo[0] - gd[0] + tx) % g[0], (d.lo[1] - gd[1] + ty) % g[1], (d.lo[2] - gd[2] + tz) % g[2]
        assert np.array_equal(gsx, gdx) and np.array_equal(gsy, gdy) and np.array_equal(gsz, gdz)
        assert (owner[gsz, gsy, gsx] == src).all()
        np.add.at(cover[dst], (tz, ty, tx), 1)
    for c in cover:
        assert (c == 1).all()


@pytest.mark.parametrize("p_order,staggered", [(8, False), (4, True), (0, False)])
def test_coefficient_tables_match_the_oracle(P, p_order, staggered):
    """Host check of the Eq. 1 tables the plan builds (Sec. 3.1): the FP64
    image for one 12 x 10 x 8 box with explicit FFT splits, read back in the
    forward transforms' position order and mapped to natural indices, against
    the oracle's modified wavenumbers and Eq. 1 coefficients."""
    import numpy as np
    from oracle import psatd_oracle as O
    L, f1 = (12, 10, 8), (2, 5, 4)
    dx, c_dt = (1.0, 0.8, 1.25), 0.45
    flags = P.PSATD_F64 | (P.PSATD_STAGGERED if staggered else 0)
    h = P.psatd_plan_create(L, [I.Sub((0, 0, 0), L, 0, p_order)], flags, {"chunk_b": 0, "f1": list(f1)})
    try:
        img = np.frombuffer(P.psatd_debug_tables(h, c_dt, dx), dtype=np.float64)
    finally:
        P.psatd_destroy(h)
    hx = L[0] // 2
    lxh = hx + 1
    n = (hx, L[1], L[2])

    def nat(a, P_):
        f2 = n[a] // f1[a]
        return hx if (a == 0 and P_ == hx) else P_ // f2 + f1[a] * (P_ % f2)
    natx = np.array([nat(0, q) for q in range(lxh)])
    naty = np.array([nat(1, q) for q in range(L[1])])
    natz = np.array([nat(2, q) for q in range(L[2])])
    km = [O.modified_k(L[a], dx[a], p_order, staggered) for a in range(3)]
    kx, ky, kz = km[0][natx], km[1][naty], km[2][natz]
    NM = L[2] * L[1] * lxh
    koff = (7 * NM + 63) // 64 * 64
    assert np.allclose(img[koff:koff + lxh], kx, rtol=1e-14, atol=1e-14)
    assert np.allclose(img[koff + lxh:koff + lxh + L[1]], ky, rtol=1e-14, atol=1e-14)
    assert np.allclose(img[koff + lxh + L[1]:koff + lxh + L[1] + L[2]], kz, rtol=1e-14, atol=1e-14)
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    kmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2).transpose(2, 1, 0)      # [z][y][x] positions
    co = O.eq1_coefficients(kmag, c_dt)
    inv = np.where(kmag > 0, 1.0 / np.where(kmag > 0, kmag, 1.0), 0.0)
    invN = 1.0 / (L[0] * L[1] * L[2])
    want = [co["C"] * invN, co["S"] * invN, co["S_k"] * invN, co["omC"] * invN, co["omC_k"] * invN,
            co["Sk_dt"] * invN, inv]
    for t, w in enumerate(want):
        got = img[t * NM:(t + 1) * NM].reshape(L[2], L[1], lxh)
        np.testing.assert_allclose(got, w, rtol=1e-12, atol=1e-15 * (1.0 if t < 6 else 10.0), err_msg=str(t))


def test_compiled_length_plane_engine_selection(P):
    """FP32 plans whose local x and y lengths are all compiled in take the
    plane stages with thread-private transforms (bit 1); with PSATD_PACKED_Z,
    those whose z lengths are compiled in take the packed z/Eq. 1 stage
    (bit 2).  FP64, odd or uncompiled lengths, non-default factorisations and
    PSATD_GENERIC_PLANES take the generic kernels; the split-plane schedule
    keeps only the z/Eq. 1 one."""
    G, Z = P.PSATD_GENERIC_PLANES, P.PSATD_PACKED_Z
    cases = [("mirror1024", P.PSATD_F32, None, 1), ("broadband256", P.PSATD_F32, None, 1),
             ("uneven48", P.PSATD_F32, None, 1), ("broadband2d", P.PSATD_F32 | P.PSATD_2D, None, 1),
             ("broadband256", P.PSATD_F32 | Z, None, 3), ("uneven48", P.PSATD_F32 | Z, None, 3),
             ("broadband2d", P.PSATD_F32 | P.PSATD_2D | Z, None, 1),
             ("mirror1024", P.PSATD_F64 | Z, None, 0), ("broadband256", P.PSATD_F32 | G | Z, None, 0),
             ("broadband256", P.PSATD_F32 | P.PSATD_SPLIT_PLANES | Z, None, 2),
             ("broadband256", P.PSATD_F32 | Z, {"chunk_b": 0, "f1": [6, 0, 0]}, 2),
             ("broadband256", P.PSATD_F32 | Z, {"chunk_b": 0, "f1": [0, 0, 6]}, 1),
             ("broadband256", P.PSATD_F32 | Z, {"chunk_b": 8, "f1": [0, 0, 0]}, 1)]
    for name, flags, tuning, want in cases:
        wl = I.workload(name)
        h = P.psatd_plan_create(wl.global_n, wl.subs, flags, tuning)
        try:
            assert P.psatd_plane_engine(h) == want, (name, flags, tuning)
        finally:
            P.psatd_destroy(h)
    subs = I.tensor_decomposition([12, 20], [14, 13], [18, 17], 4, 8)     # odd local lengths
    h = P.psatd_plan_create((32, 27, 35), subs, P.PSATD_F32 | Z)
    assert P.psatd_plane_engine(h) == 0
    P.psatd_destroy(h)


def test_three_factor_lengths_are_accepted(P):
    """Lengths with no two-factor split but a three-factor one (216, 432 along
    x, a 1024-long x axis, the 1024 x 512 x 512 grid as one global box) are
    accepted; a length with a prime factor above 16 is still rejected."""
    ok = [((32, 400, 16), I.tensor_decomposition([32], [200, 200], [16], 8, 8)),
          ((416, 16, 16), I.tensor_decomposition([416], [16], [16], 8, 8)),
          ((1024, 8, 8), I.tensor_decomposition([1024], [8], [8], 0, 0)),
          ((1024, 512, 512), I.tensor_decomposition([1024], [512], [512], 0, 0))]
    for g, subs in ok:
        for flags in (P.PSATD_F32, P.PSATD_F64):
            h = P.psatd_plan_create(g, subs, flags)
            assert P.psatd_layout(h, 0)[1] == subs[0].local
            P.psatd_destroy(h)
    with pytest.raises(P.PsatdError) as e:
        P.psatd_plan_create((32, 34 * 16, 16), I.tensor_decomposition([32], [34 * 16], [16], 0, 8), P.PSATD_F32)
    assert e.value.code == -5
