"""ctypes binding of libpsatd.so (argument marshalling only) plus a small
harness class that owns torch-allocated arenas and workspace.

Every function here calls straight into the C ABI of ``include/psatd.h``;
all arithmetic of the solver runs in the library's CUDA kernels.  There is no
CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import torch

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PSATD_LIB") or os.path.join(_HERE, "libpsatd.so")

PSATD_F32 = 0x01
PSATD_F64 = 0x02
PSATD_STAGGERED = 0x04
PSATD_GAUSS_DIAG = 0x08
PSATD_PLAIN = 0x10
PSATD_GRID_PER_ITEM = 0x20
PSATD_2D = 0x40
PSATD_SPLIT_PLANES = 0x80
PSATD_HEAT = 0x100
PSATD_HEAT_SOURCE = 0x200
PSATD_GENERIC_PLANES = 0x400
PSATD_PACKED_Z = 0x800

STATUS = {0: "PSATD_OK", -1: "PSATD_E_ARG", -2: "PSATD_E_SHAPE", -3: "PSATD_E_NOMEM",
          -4: "PSATD_E_CUDA", -5: "PSATD_E_UNSUPPORTED", -6: "PSATD_E_STATE", -7: "PSATD_E_TIMEOUT"}

EXPORTS = ("psatd_plan", "psatd_plan_create", "psatd_layout", "psatd_arena_elems", "psatd_workspace_bytes",
           "psatd_set_workspace", "psatd_set_coeffs", "psatd_push", "psatd_exchange_guards",
           "psatd_destroy", "psatd_status_string", "psatd_last_error", "psatd_push_launches",
           "psatd_push_profiled", "psatd_plan_create_tuned", "psatd_push_static", "psatd_geometry_variant",
           "psatd_yee_step", "psatd_yee_launches", "psatd_check", "psatd_scatter_global",
           "psatd_gather_global", "psatd_exchange_segments", "psatd_debug_tables", "psatd_plane_engine")

STATIC_WORKSPACE_BYTES = 32 * 1024 * 1024


class PsatdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class SubT(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int32 * 3), ("n", ctypes.c_int32 * 3),
                ("ng", ctypes.c_int32), ("order", ctypes.c_int32)]


class TuningT(ctypes.Structure):
    _fields_ = [("chunk_b", ctypes.c_int32), ("f1", ctypes.c_int32 * 3)]


class FieldsT(ctypes.Structure):
    _fields_ = [("E", ctypes.c_void_p * 3), ("B", ctypes.c_void_p * 3),
                ("J", ctypes.c_void_p * 3), ("rho", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libpsatd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1707_08500_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, VP = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.psatd_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(I32), ctypes.POINTER(SubT), I32, I32]
        L.psatd_plan.argtypes = [ctypes.POINTER(P), ctypes.POINTER(I32), ctypes.POINTER(SubT), I32, I32, VP]
        L.psatd_plan_create_tuned.argtypes = [ctypes.POINTER(P), ctypes.POINTER(I32), ctypes.POINTER(SubT), I32, I32,
                                              ctypes.POINTER(TuningT)]
        L.psatd_layout.argtypes = [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I32)]
        L.psatd_arena_elems.argtypes = [P, ctypes.POINTER(I64)]
        L.psatd_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.psatd_set_workspace.argtypes = [P, VP, ctypes.c_size_t]
        L.psatd_set_coeffs.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        L.psatd_push.argtypes = [P, ctypes.POINTER(FieldsT), VP, VP]
        L.psatd_push_profiled.argtypes = [P, ctypes.POINTER(FieldsT), VP, VP, ctypes.POINTER(VP)]
        L.psatd_push_static.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(FieldsT),
                                         VP, VP]
        L.psatd_exchange_guards.argtypes = [P, ctypes.POINTER(FieldsT), VP]
        L.psatd_destroy.argtypes = [P]
        L.psatd_status_string.argtypes = [ctypes.c_int]
        L.psatd_status_string.restype = ctypes.c_char_p
        L.psatd_last_error.argtypes = [P]
        L.psatd_last_error.restype = ctypes.c_char_p
        L.psatd_push_launches.argtypes = [P, ctypes.POINTER(I32)]
        L.psatd_geometry_variant.argtypes = [P, ctypes.POINTER(I32)]
        L.psatd_plane_engine.argtypes = [P, ctypes.POINTER(I32)]
        for name in EXPORTS:
            if name not in ("psatd_status_string", "psatd_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(code: int, plan=None):
    if code != 0:
        msg = lib().psatd_last_error(plan).decode() if plan else lib().psatd_status_string(code).decode()
        raise PsatdError(code, msg)


# ---- thin wrappers with the C names -------------------------------------------
def psatd_plan_create(global_n: Sequence[int], subs: Sequence, flags: int, tuning: Optional[dict] = None) -> ctypes.c_void_p:
    """tuning: None or {"chunk_b": M, "f1": (fx, fy, fz)} (0 = default)."""
    arr = (SubT * max(len(subs), 1))()
    for i, s in enumerate(subs):
        arr[i].lo[:] = list(s.lo)
        arr[i].n[:] = list(s.n)
        arr[i].ng = s.ng
        arr[i].order = s.p
    g = (ctypes.c_int32 * 3)(*global_n)
    h = ctypes.c_void_p()
    if tuning is None:
        code = lib().psatd_plan_create(ctypes.byref(h), g, arr, len(subs), flags)
    else:
        t = TuningT()
        t.chunk_b = int(tuning.get("chunk_b", 0))
        t.f1[:] = [int(v) for v in tuning.get("f1", (0, 0, 0))]
        code = lib().psatd_plan_create_tuned(ctypes.byref(h), g, arr, len(subs), flags, ctypes.byref(t))
    if code != 0:
        raise PsatdError(code, lib().psatd_status_string(code).decode())
    return h


def psatd_plan(global_n: Sequence[int], subs: Sequence, flags: int, stream: Optional[int] = None) -> ctypes.c_void_p:
    """psatd_plan_create with a bound set-up stream (raw cudaStream_t or None)."""
    arr = (SubT * max(len(subs), 1))()
    for i, s in enumerate(subs):
        arr[i].lo[:] = list(s.lo)
        arr[i].n[:] = list(s.n)
        arr[i].ng = s.ng
        arr[i].order = s.p
    g = (ctypes.c_int32 * 3)(*global_n)
    h = ctypes.c_void_p()
    code = lib().psatd_plan(ctypes.byref(h), g, arr, len(subs), flags, ctypes.c_void_p(stream or 0))
    if code != 0:
        raise PsatdError(code, lib().psatd_status_string(code).decode())
    return h


def psatd_layout(plan, sub: int):
    off = ctypes.c_int64()
    ln = (ctypes.c_int32 * 3)()
    _check(lib().psatd_layout(plan, sub, ctypes.byref(off), ln), plan)
    return off.value, tuple(ln)


def psatd_arena_elems(plan) -> int:
    n = ctypes.c_int64()
    _check(lib().psatd_arena_elems(plan, ctypes.byref(n)), plan)
    return n.value


def psatd_workspace_bytes(plan) -> int:
    n = ctypes.c_size_t()
    _check(lib().psatd_workspace_bytes(plan, ctypes.byref(n)), plan)
    return n.value


def psatd_set_workspace(plan, ptr: int, nbytes: int):
    _check(lib().psatd_set_workspace(plan, ctypes.c_void_p(ptr), nbytes), plan)


def psatd_set_coeffs(plan, c_dt: float, dx: Sequence[float]):
    d = (ctypes.c_double * 3)(*dx)
    _check(lib().psatd_set_coeffs(plan, c_dt, d), plan)


def psatd_push(plan, fields: FieldsT, gauss_ptr: Optional[int] = None, stream: Optional[int] = None):
    _check(lib().psatd_push(plan, ctypes.byref(fields), ctypes.c_void_p(gauss_ptr or 0),
                            ctypes.c_void_p(stream or 0)), plan)


def psatd_push_profiled(plan, fields: FieldsT, gauss_ptr, stream, events):
    """events: four raw cudaEvent_t handles (ints) or None."""
    ev = (ctypes.c_void_p * 4)(*[e or None for e in events])
    _check(lib().psatd_push_profiled(plan, ctypes.byref(fields), ctypes.c_void_p(gauss_ptr or 0),
                                     ctypes.c_void_p(stream or 0), ev), plan)


def psatd_push_static(plan, c_dt: float, dx: Sequence[float], fields: FieldsT, gauss_ptr: Optional[int] = None,
                      stream: Optional[int] = None):
    """The push on the library's static device workspace (no allocation by
    the caller or the library; see include/psatd.h)."""
    d = (ctypes.c_double * 3)(*dx)
    _check(lib().psatd_push_static(plan, c_dt, d, ctypes.byref(fields), ctypes.c_void_p(gauss_ptr or 0),
                                   ctypes.c_void_p(stream or 0)), plan)


def psatd_exchange_guards(plan, fields: FieldsT, stream: Optional[int] = None):
    _check(lib().psatd_exchange_guards(plan, ctypes.byref(fields), ctypes.c_void_p(stream or 0)), plan)


def psatd_yee_step(global_n: Sequence[int], flags: int, c_dt: float, dx: Sequence[float], fin: FieldsT,
                   fout: FieldsT, stream: Optional[int] = None):
    """One Yee FDTD step (Eqs. 2a/2b): fin = (E^n, B^{n-1/2}, J^{n+1/2}) ->
    fout = (E^{n+1}, B^{n+1/2}); dense [Nz][Ny][Nx] device arrays."""
    n = (ctypes.c_int32 * 3)(*global_n)
    d = (ctypes.c_double * 3)(*dx)
    _check(lib().psatd_yee_step(n, ctypes.c_int32(flags), ctypes.c_double(c_dt), d, ctypes.byref(fin),
                                ctypes.byref(fout), ctypes.c_void_p(stream or 0)))


def psatd_yee_launches() -> int:
    v = ctypes.c_int32()
    _check(lib().psatd_yee_launches(ctypes.byref(v)))
    return v.value


def _ptrs(ts) -> "ctypes.Array":
    return (ctypes.c_void_p * len(ts))(*[t if isinstance(t, int) else t.data_ptr() for t in ts])


def psatd_scatter_global(plan, global_in: Sequence, arenas: Sequence, stream: Optional[int] = None):
    """Fill every padded box (valid cells and guards) of each arena from a
    global [Nz][Ny][Nx] device array (tensors or raw pointers)."""
    assert len(global_in) == len(arenas)
    _check(lib().psatd_scatter_global(plan, _ptrs(global_in), _ptrs(arenas), ctypes.c_int32(len(arenas)),
                                      ctypes.c_void_p(stream or 0)), plan)


def psatd_gather_global(plan, arenas: Sequence, global_out: Sequence, stream: Optional[int] = None):
    """Write each box's valid cells of each arena into a global device array."""
    assert len(global_out) == len(arenas)
    _check(lib().psatd_gather_global(plan, _ptrs(arenas), _ptrs(global_out), ctypes.c_int32(len(arenas)),
                                     ctypes.c_void_p(stream or 0)), plan)


def psatd_debug_tables(plan, c_dt: float, dx: Sequence[float]) -> bytes:
    """The real coefficient-table image the plan would upload (host only)."""
    d = (ctypes.c_double * 3)(*dx)
    n = ctypes.c_size_t(0)
    _check(lib().psatd_debug_tables(plan, ctypes.c_double(c_dt), d, None, ctypes.byref(n)), plan)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().psatd_debug_tables(plan, ctypes.c_double(c_dt), d, buf, ctypes.byref(n)), plan)
    return buf.raw


def psatd_exchange_segments(plan):
    """The plan's guard-exchange copy segments as a list of 12-int tuples
    (src, dst, x0, y0, z0, ex, ey, ez, dx, dy, dz, identity)."""
    n = ctypes.c_int32()
    _check(lib().psatd_exchange_segments(plan, ctypes.byref(n), None), plan)
    buf = (ctypes.c_int32 * (12 * n.value))()
    _check(lib().psatd_exchange_segments(plan, ctypes.byref(n), buf), plan)
    return [tuple(buf[12 * i:12 * i + 12]) for i in range(n.value)]


def psatd_check(plan) -> int:
    """Synchronise the device and return (and clear) the plan's device error bits."""
    v = ctypes.c_int32()
    _check(lib().psatd_check(plan, ctypes.byref(v)), plan)
    return v.value


def psatd_destroy(plan):
    lib().psatd_destroy(plan)


def psatd_status_string(code: int) -> str:
    return lib().psatd_status_string(code).decode()


def psatd_last_error(plan) -> str:
    return lib().psatd_last_error(plan).decode()


def psatd_push_launches(plan) -> int:
    n = ctypes.c_int32()
    _check(lib().psatd_push_launches(plan, ctypes.byref(n)), plan)
    return n.value


def psatd_geometry_variant(plan) -> int:
    n = ctypes.c_int32()
    _check(lib().psatd_geometry_variant(plan, ctypes.byref(n)), plan)
    return n.value


def psatd_plane_engine(plan) -> int:
    n = ctypes.c_int32()
    _check(lib().psatd_plane_engine(plan, ctypes.byref(n)), plan)
    return n.value


def make_fields(E, B, J, rho=None) -> FieldsT:
    f = FieldsT()
    for a in range(3):
        f.E[a] = E[a].data_ptr()
        f.B[a] = B[a].data_ptr()
        f.J[a] = J[a].data_ptr()
    f.rho = rho.data_ptr() if rho is not None else None
    return f


# ---- harness -------------------------------------------------------------------
class Solver:
    """Owns the ten field arenas and the workspace of one plan (torch memory).

    Arenas are flat tensors of ``psatd_arena_elems`` elements; subdomain s sits
    at ``layout[s][0]`` as a dense [Lz][Ly][Lx] box."""

    def __init__(self, wl: "_inputs.Workload", precision: Optional[str] = None, plain: bool = False,
                 gauss: bool = False, device="cuda", tuning: Optional[dict] = None, extra_flags: int = 0):
        self.wl = wl
        self.precision = precision or wl.precision
        self.dtype = torch.float64 if self.precision == "f64" else torch.float32
        flags = PSATD_F64 if self.precision == "f64" else PSATD_F32
        if wl.staggered:
            flags |= PSATD_STAGGERED
        if wl.two_d:
            flags |= PSATD_2D
        if gauss:
            flags |= PSATD_GAUSS_DIAG
        if plain:
            flags |= PSATD_PLAIN
        flags |= extra_flags
        self.flags = flags
        self.gauss = gauss
        self.device = torch.device(device)
        self.tuning = tuning
        self.plan = psatd_plan_create(wl.global_n, wl.subs, flags, tuning)
        self.layout = [psatd_layout(self.plan, s) for s in range(len(wl.subs))]
        self.arena_elems = psatd_arena_elems(self.plan)
        self.ws_bytes = psatd_workspace_bytes(self.plan)
        self.arenas = {n: torch.zeros(self.arena_elems, dtype=self.dtype, device=self.device)
                       for n in _inputs.FIELD_NAMES}
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        psatd_set_workspace(self.plan, self.ws_ptr, self.ws_bytes)
        psatd_set_coeffs(self.plan, wl.c_dt, wl.dx)
        self.gauss_out = torch.zeros(2 * len(wl.subs), dtype=torch.float64, device=self.device) if gauss else None
        self.fields = make_fields([self.arenas[n] for n in ("Ex", "Ey", "Ez")],
                                  [self.arenas[n] for n in ("Bx", "By", "Bz")],
                                  [self.arenas[n] for n in ("Jx", "Jy", "Jz")],
                                  self.arenas["rho"])

    def __del__(self):
        try:
            if getattr(self, "plan", None):
                psatd_destroy(self.plan)
                self.plan = None
        except Exception:
            pass

    # -- layout helpers (pure data movement) --
    def box(self, name: str, s: int) -> torch.Tensor:
        off, (lx, ly, lz) = self.layout[s]
        return self.arenas[name][off:off + lx * ly * lz].view(lz, ly, lx)

    def load_global(self, glob: Dict[str, torch.Tensor], names=None, guards=True):
        """Write every subdomain's padded box (guards=True) or only its valid
        box from global arrays [Nz][Ny][Nx] (periodic indexing)."""
        names = names or _inputs.FIELD_NAMES
        nx, ny, nz = self.wl.global_n
        dev = {n: glob[n].to(self.device) for n in names}
        for s, sd in enumerate(self.wl.subs):
            for n in names:
                g = dev[n]
                b = self.box(n, s)
                gx, gy, gz = sd.guards
                if guards:
                    ix = (torch.arange(sd.local[0], device=self.device) + sd.lo[0] - gx) % nx
                    iy = (torch.arange(sd.local[1], device=self.device) + sd.lo[1] - gy) % ny
                    iz = (torch.arange(sd.local[2], device=self.device) + sd.lo[2] - gz) % nz
                    b.copy_(g[iz][:, iy][:, :, ix].to(self.dtype))
                else:
                    x0, y0, z0 = sd.lo
                    vx, vy, vz = sd.n
                    b[gz:gz + vz, gy:gy + vy, gx:gx + vx].copy_(g[z0:z0 + vz, y0:y0 + vy, x0:x0 + vx].to(self.dtype))

    def load_boxes(self, boxes: Dict[int, Dict[str, torch.Tensor]]):
        for s, fl in boxes.items():
            for n, t in fl.items():
                self.box(n, s).copy_(t.to(self.device, self.dtype))

    def gather_global(self, names=_inputs.EB_NAMES) -> Dict[str, torch.Tensor]:
        """Valid cells of every subdomain assembled into global arrays (FP64, CPU)."""
        nx, ny, nz = self.wl.global_n
        out = {n: torch.empty((nz, ny, nx), dtype=torch.float64) for n in names}
        for s, sd in enumerate(self.wl.subs):
            x0, y0, z0 = sd.lo
            vx, vy, vz = sd.n
            gx, gy, gz = sd.guards
            for n in names:
                out[n][z0:z0 + vz, y0:y0 + vy, x0:x0 + vx] = \
                    self.box(n, s)[gz:gz + vz, gy:gy + vy, gx:gx + vx].to("cpu", torch.float64)
        return out

    # -- solver calls --
    def exchange(self, stream: Optional[int] = None):
        psatd_exchange_guards(self.plan, self.fields, stream if stream is not None else
                              torch.cuda.current_stream(self.device).cuda_stream)

    def push(self, stream: Optional[int] = None):
        psatd_push(self.plan, self.fields, self.gauss_out.data_ptr() if self.gauss else None,
                   stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream)

    def gauss_sums(self):
        return self.gauss_out.view(-1, 2).cpu().numpy()


class HeatSolver(Solver):
    """The local-FFT heat equation (PSATD_HEAT) on the decomposition of a
    workload: arenas "T" (advanced in place, guards included) and, with a
    source, "S" (heat added per cell over a step).  d_dt = D dt."""

    def __init__(self, wl: "_inputs.Workload", d_dt: float, source: bool = False, precision: Optional[str] = None,
                 plain: bool = False, device="cuda", tuning: Optional[dict] = None, extra_flags: int = 0):
        self.wl = wl
        self.precision = precision or wl.precision
        self.dtype = torch.float64 if self.precision == "f64" else torch.float32
        flags = (PSATD_F64 if self.precision == "f64" else PSATD_F32) | PSATD_HEAT
        if source:
            flags |= PSATD_HEAT_SOURCE
        if wl.two_d:
            flags |= PSATD_2D
        if plain:
            flags |= PSATD_PLAIN
        flags |= extra_flags
        self.flags, self.gauss, self.device, self.tuning = flags, False, torch.device(device), tuning
        self.gauss_out = None
        self.plan = psatd_plan_create(wl.global_n, wl.subs, flags, tuning)
        self.layout = [psatd_layout(self.plan, s) for s in range(len(wl.subs))]
        self.arena_elems = psatd_arena_elems(self.plan)
        self.ws_bytes = psatd_workspace_bytes(self.plan)
        names = ("T", "S") if source else ("T",)
        self.arenas = {n: torch.zeros(self.arena_elems, dtype=self.dtype, device=self.device) for n in names}
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        psatd_set_workspace(self.plan, self.ws_ptr, self.ws_bytes)
        psatd_set_coeffs(self.plan, d_dt, wl.dx)
        f = FieldsT()
        f.E[0] = self.arenas["T"].data_ptr()
        f.J[0] = self.arenas["S"].data_ptr() if source else None
        self.fields = f
