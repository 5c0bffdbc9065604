"""Yee FDTD solver (Sec. 2, Eqs. 2a/2b) over the C ABI: two device field sets
used in turn (the step writes the other set), J shared by both.

State: E^n and B^{n-1/2}; each ``step()`` advances to E^{n+1}, B^{n+1/2} with
the current J (J^{n+1/2}).  Arrays are dense [Nz][Ny][Nx] tensors."""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import torch

from . import psatd as P

E_NAMES = ("Ex", "Ey", "Ez")
B_NAMES = ("Bx", "By", "Bz")
J_NAMES = ("Jx", "Jy", "Jz")


class YeeSolver:
    def __init__(self, global_n: Sequence[int], c_dt: float, dx: Sequence[float] = (1.0, 1.0, 1.0),
                 precision: str = "f32", device="cuda"):
        self.global_n = tuple(int(v) for v in global_n)
        self.c_dt, self.dx = float(c_dt), tuple(float(v) for v in dx)
        self.flags = P.PSATD_F64 if precision == "f64" else P.PSATD_F32
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.device = torch.device(device)
        nx, ny, nz = self.global_n
        shape = (nz, ny, nx)
        self.sets = [{n: torch.zeros(shape, dtype=self.dtype, device=self.device) for n in E_NAMES + B_NAMES}
                     for _ in range(2)]
        self.J = {n: torch.zeros(shape, dtype=self.dtype, device=self.device) for n in J_NAMES}
        self.cur = 0
        self._fields = [self._make(s) for s in (0, 1)]

    def _make(self, s):
        f = self.sets[s]
        return P.make_fields([f[n] for n in E_NAMES], [f[n] for n in B_NAMES], [self.J[n] for n in J_NAMES], None)

    @property
    def fields(self) -> Dict[str, torch.Tensor]:
        """The current E^n, B^{n-1/2} (and J)."""
        return dict(self.sets[self.cur], **self.J)

    def load(self, glob: Dict[str, torch.Tensor]):
        for n in E_NAMES + B_NAMES:
            if n in glob:
                self.sets[self.cur][n].copy_(glob[n].to(self.device, self.dtype))
        for n in J_NAMES:
            if n in glob:
                self.J[n].copy_(glob[n].to(self.device, self.dtype))

    def step(self, stream: Optional[int] = None):
        st = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        P.psatd_yee_step(self.global_n, self.flags, self.c_dt, self.dx, self._fields[self.cur],
                         self._fields[self.cur ^ 1], st)
        self.cur ^= 1

    def gather(self) -> Dict[str, torch.Tensor]:
        return {n: t.to("cpu", torch.float64) for n, t in self.sets[self.cur].items()}
