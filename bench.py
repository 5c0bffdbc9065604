"""Throughput of the local-FFT PSATD push on one GB300 (arXiv:1707.08500, Sec. 3).

Default workload: the plasma-mirror-shaped grid, 1024x512x512 cells cut into
16x8x8 subdomains of 64^3 with 16 guards (96^3 local FFTs), order p = 100,
FP32 batched schedule with the Gauss diagnostic (10 fields in, 6 out).

One step = one psatd_push (passes A, B, C and the Gauss reduction) over all
1024 subdomains.  Inputs (906 M local cells x 10 fields, 36 GB) are far larger
than L2, so no flush is needed between steps.  The JSON line also carries the
per-stage roofline of the dominant kernel, the plain one-subdomain-per-launch
FP64 GPU path, an end-to-end number through the C ABI with per-step host
copies, and the FP64 CPU oracle timed on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-steps/s of local-FFT PSATD push, batched FP32 vs plain FP64; % HBM roof"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ------------------------------------------------------------------------------
def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest value over all ranks (timing only; no data-path collective)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(valid_cells: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput of `world` independent replicas (weak scaling):
    valid cells of all ranks per second, in Gcell-steps/s."""
    return valid_cells * world / (ms_per_step / 1e3) / 1e9


def stage_bytes(wl, nf: int, esz: int, nout: int = 6):
    """Algorithmic HBM bytes per launch of each stage (unique inputs + outputs):
    A reads nf real fields and writes nf half spectra; B reads nf spectra and
    writes 6 spectra on the valid z planes; C reads those and writes 6 real
    fields on every local cell (own box plus guard images)."""
    A = B = C = 0
    local = 0
    for sd in wl.subs:
        lx, ly, lz = sd.local
        cells = lx * ly * lz
        spec = lz * ly * (lx // 2 + 1) * 2 * esz
        vspec = sd.n[2] * ly * (lx // 2 + 1) * 2 * esz
        A += nf * (cells * esz + spec)
        B += nf * spec + nout * vspec
        C += nout * (vspec + cells * esz)
        local += cells
    return {"A": A, "B": B, "C": C}, local


KERNEL_SOURCES = ("psatd_kernels.cuh", "psatd_kernels_f32.cu", "small_dft.cuh", "psatd_internal.h", "psatd_regfft.cuh",
                  "psatd_regfft_f32.cu")


def kernels_sha256() -> str:
    """Hash of the stage-kernel sources (the profile summaries record it)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1707_08500_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources and this workload (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic_mirror1024.json")) as f:
            t = json.load(f)
        if t.get("kernels_sha256") != kernels_sha256() or t.get("workload") != workload:
            return None
        return t["bytes_per_launch"].get(kernel)
    except Exception:
        return None


def fill_solver(sol, wl, device):
    """Write every subdomain's padded box of all ten fields (FP64 synthesis on
    the device, cast to the solver's precision)."""
    from paper_1707_08500_gb300 import inputs as I
    import torch
    if wl.fields == "laser_slab":
        for s, sd in enumerate(wl.subs):
            b = I.box_fields(wl, sd, device=device)
            for n in I.FIELD_NAMES:
                sol.box(n, s).copy_(b[n])
            del b
    else:
        glob = I.global_fields(wl)
        sol.load_global(glob)
    torch.cuda.synchronize()


def cpu_oracle_sample(wl, budget_s: float):
    """FP64 oracle (as it stands) on whole subdomain steps until the budget is spent."""
    from oracle import psatd_oracle as O
    from paper_1707_08500_gb300 import inputs as I
    t_used, cells, nsub = 0.0, 0, 0
    for sd in wl.subs[:: max(1, len(wl.subs) // 64)]:
        b = {k: v.numpy() for k, v in I.box_fields(wl, sd, device="cpu").items()}
        t0 = time.perf_counter()
        O.local_push(b, sd.local, wl.dx, sd.p, wl.c_dt, wl.staggered)
        t_used += time.perf_counter() - t0
        cells += sd.n[0] * sd.n[1] * sd.n[2]
        nsub += 1
        if t_used > budget_s:
            break
    return {"value": cells / t_used / 1e9, "unit": "Gcell-steps/s", "cores": O.WORKERS, "kind": "oracle",
            "sample": f"{nsub} of {len(wl.subs)} subdomain steps ({cells} valid cells), {t_used:.1f} s"}


# ------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1707_08500_gb300 import build as B
    from paper_1707_08500_gb300 import inputs as I
    from paper_1707_08500_gb300 import psatd as P

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = I.workload(args.workload)
    gauss = not args.no_gauss
    prec = args.precision or ("f32" if wl.precision == "f32" else "f64")
    flags = (P.PSATD_F32 if prec == "f32" else P.PSATD_F64) | (P.PSATD_GAUSS_DIAG if gauss else 0)
    if wl.staggered:
        flags |= P.PSATD_STAGGERED
    if wl.two_d:
        flags |= P.PSATD_2D
    if args.chunk_b:
        tuning = {"chunk_b": args.chunk_b, "f1": [0, 0, 0]}
    elif not args.no_tune:
        from paper_1707_08500_gb300 import tune as T
        tuning = T.autotune(wl, flags, device=dev)
        torch.cuda.empty_cache()
    else:
        tuning = None
    sol = P.Solver(wl, precision=prec, gauss=gauss, device=dev, tuning=tuning,
                   extra_flags=(P.PSATD_GRID_PER_ITEM if args.grid_per_item else 0) |
                   (P.PSATD_GENERIC_PLANES if args.generic_planes else 0))
    fill_solver(sol, wl, dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def mkev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    for _ in range(args.warmup):
        sol.push(sp)
    torch.cuda.synchronize()
    evs = [[mkev() for _ in range(4)] for _ in range(args.steps)]
    t0, t1 = mkev(), mkev()
    torch.cuda.synchronize()
    gp = sol.gauss_out.data_ptr() if gauss else None
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(args.steps):
            P.psatd_push_profiled(sol.plan, sol.fields, gp, sp, [e.cuda_event for e in evs[k]])
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    graph_ms = None
    if not args.no_graph:
        # the same K steps captured as one CUDA graph and replayed (the stage
        # events above cannot be timed inside a graph, so this is reported beside)
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                cs = torch.cuda.current_stream(dev).cuda_stream
                for k in range(args.steps):
                    P.psatd_push(sol.plan, sol.fields, gp, cs)
            graph.replay()
            torch.cuda.synchronize()
            g0, g1 = mkev(), mkev()
            torch.cuda.synchronize()
            g0.record(stream)
            graph.replay()
            g1.record(stream)
            torch.cuda.synchronize()
            graph_ms = g0.elapsed_time(g1) / args.steps
            del graph
        except Exception as exc:
            print(f"graph capture unavailable: {exc}", file=sys.stderr)
            torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    stage_ms = {st: sum(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)) / args.steps
                for i, st in enumerate("ABC")}
    ms = max_over_ranks(ms, world, dev)
    ms_step = ms / args.steps
    valid = wl.valid_cells
    value = replica_value(valid, world, ms_step)
    nf = 10 if gauss else 9
    by, local = stage_bytes(wl, nf, 4 if prec == "f32" else 8)
    peak, peak_kind = _peaks()
    dom = max(stage_ms, key=stage_ms.get)
    split = P.psatd_push_launches(sol.plan) - (1 if gauss else 0) == 5
    engine = P.psatd_plane_engine(sol.plan)
    names = ({"A": "k_rows_fwd+k_cols", "B": "k_pass_b", "C": "k_cols+k_rows_inv"} if split
             else {"A": "k_pass_a_reg", "B": "k_pass_b", "C": "k_pass_c_reg"} if engine & 1
             else {"A": "k_pass_a", "B": "k_pass_b", "C": "k_pass_c"})
    if engine & 2:
        names["B"] = "k_pass_b_reg"
    stages = {st: {"kernel": names[st], "ms": round(stage_ms[st], 3), "alg_bytes": by[st],
                   "gbs": round(by[st] / (stage_ms[st] / 1e3) / 1e9, 1),
                   "frac": round(by[st] / (stage_ms[st] / 1e3) / 1e9 / peak, 4)} for st in "ABC"}
    achieved = by[dom] / (stage_ms[dom] / 1e3) / 1e9
    fused_bytes = (16 if gauss else 15) * (4 if prec == "f32" else 8) * local
    result = {
        "metric": METRIC,
        "value": round(value, 4), "unit": "Gcell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": wl.name, "global_n": list(wl.global_n), "subdomains": len(wl.subs),
                   "local_n": list(wl.subs[0].local), "guards": wl.subs[0].ng, "order": wl.subs[0].p,
                   "c_dt": wl.c_dt, "gauss_diag": gauss, "valid_cells": valid, "local_cells": local,
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "schedule": "split-plane (5 stages)" if split else "3 stages",
                   "l2": f"inputs ({local * nf * (4 if prec == 'f32' else 8) / 1e9:.1f} GB) larger than L2; no flush"},
        "local_gcell_steps": round(local * world / (ms_step / 1e3) / 1e9, 4),
        "stages": stages,
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": _traffic(names[dom], wl.name),
                     "peak_kind": peak_kind},
        "step_roofline": {"alg_bytes_per_step_fused": fused_bytes,
                          "frac_of_fused_floor": round(fused_bytes / (ms_step / 1e3) / 1e9 / peak, 4),
                          "three_pass_bytes_per_step": sum(by.values()),
                          "frac_three_pass": round(sum(by.values()) / (ms_step / 1e3) / 1e9 / peak, 4)},
        "gpu_launches": args.steps * P.psatd_push_launches(sol.plan),
        "kernels": {"geometry_variant": P.psatd_geometry_variant(sol.plan),
                    "engine": {"planes": "compiled-length" if engine & 1 else "generic",
                               "z_eq1": "compiled-length" if engine & 2 else "generic"},
                    "tuning": tuning,
                    "persistent": not args.grid_per_item, "cuda_graph_ms_per_step": None if graph_ms is None else round(graph_ms, 4)},
        "clocks": clk.summary(),
    }
    # ---- end to end through the C ABI with per-step host copies ----------------
    # Every step copies its sources (J, and rho with the Gauss diagnostic) as
    # global arrays of valid cells from pinned host memory, spreads them into
    # the padded boxes on the device (psatd_scatter_global: valid cells and
    # guard images), pushes, collects the valid E and B of every subdomain
    # into global arrays (psatd_gather_global) and copies them, with the Gauss
    # sums, back to pinned host memory.  The upload of step k+1 runs on a
    # second stream into a second device buffer while step k computes; the
    # read-backs run on a third stream from two alternating device buffers.
    # The same loop without the field read-back (fields stay resident on the
    # device, as in a particle-in-cell code whose particle push reads them
    # there) is reported as e2e_fields_resident.
    if not args.skip_e2e:
        names_in = ("Jx", "Jy", "Jz", "rho") if gauss else ("Jx", "Jy", "Jz")
        nx, ny, nz = wl.global_n
        gdev = [{n: torch.empty((nz, ny, nx), dtype=sol.dtype, device=dev) for n in names_in} for _ in range(2)]
        P.psatd_gather_global(sol.plan, [sol.arenas[n] for n in names_in], [gdev[0][n] for n in names_in], sp)
        host = {n: torch.empty((nz, ny, nx), dtype=sol.dtype, pin_memory=True) for n in names_in}
        for n in names_in:
            host[n].copy_(gdev[0][n])
        ksteps = max(3, min(args.steps, 10))
        # one small Gauss buffer per step (device and pinned host), so that no
        # push waits for an earlier step's read-back
        gh = [torch.empty(2 * len(wl.subs), dtype=torch.float64, pin_memory=True) for _ in range(ksteps)]
        gd = [torch.empty(2 * len(wl.subs), dtype=torch.float64, device=dev) for _ in range(ksteps)]
        fdev = [{n: torch.empty((nz, ny, nx), dtype=sol.dtype, device=dev) for n in I.EB_NAMES} for _ in range(2)]
        fhost = {n: torch.empty((nz, ny, nx), dtype=sol.dtype, pin_memory=True) for n in I.EB_NAMES}
        cs = torch.cuda.Stream(dev)
        ds = torch.cuda.Stream(dev)       # read-backs: kept off the compute stream, where they would
        pushed = [torch.cuda.Event() for _ in range(ksteps)]   # queue behind the uploads on the copy engines
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        read = [torch.cuda.Event() for _ in range(2)]
        arenas_in = [sol.arenas[n] for n in names_in]
        arenas_eb = [sol.arenas[n] for n in I.EB_NAMES]

        def upload(b):
            with torch.cuda.stream(cs):
                for n in names_in:
                    gdev[b][n].copy_(host[n], non_blocking=True)
                copied[b].record(cs)

        def step(b, gptr):
            stream.wait_event(copied[b])
            P.psatd_scatter_global(sol.plan, [gdev[b][n] for n in names_in], arenas_in, sp)
            used[b].record(stream)
            P.psatd_push(sol.plan, sol.fields, gptr, sp)

        def run_loop(fields_out):
            for e in read:
                e.record(ds)
            e0, e1 = mkev(), mkev()
            e0.record(stream)
            cs.wait_event(e0)
            upload(0)
            for k in range(ksteps):
                b = k % 2
                if k + 1 < ksteps:
                    if k >= 1:
                        cs.wait_event(used[b ^ 1])
                    upload(b ^ 1)
                step(b, gd[k].data_ptr() if gauss else None)
                if fields_out:
                    stream.wait_event(read[b])          # the read-back of step k-2 has left buffer b
                    P.psatd_gather_global(sol.plan, arenas_eb, [fdev[b][n] for n in I.EB_NAMES], sp)
                pushed[k].record(stream)
                ds.wait_event(pushed[k])
                with torch.cuda.stream(ds):
                    if gauss:
                        gh[k].copy_(gd[k], non_blocking=True)
                    if fields_out:
                        for n in I.EB_NAMES:
                            fhost[n].copy_(fdev[b][n], non_blocking=True)
                        read[b].record(ds)
            stream.wait_stream(ds)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / ksteps
        # warm-up of the copy path and of the pushes, outside the timed region;
        # then the upload, the scatter and the read-back alone, timed, for reference
        upload(0)
        upload(1)
        for b in (0, 1):
            step(b, gd[b].data_ptr() if gauss else None)
        torch.cuda.synchronize()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(cs)
        upload(0)
        u1.record(cs)
        torch.cuda.synchronize()
        upload_ms = u0.elapsed_time(u1)
        s0, s1 = mkev(), mkev()
        s0.record(stream)
        P.psatd_scatter_global(sol.plan, [gdev[0][n] for n in names_in], arenas_in, sp)
        s1.record(stream)
        torch.cuda.synchronize()
        scatter_ms = s0.elapsed_time(s1)
        with torch.cuda.stream(ds):           # first touch of the pinned buffers, untimed
            for n in I.EB_NAMES:
                fhost[n].copy_(fdev[0][n], non_blocking=True)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(ds)
        with torch.cuda.stream(ds):
            for n in I.EB_NAMES:
                fhost[n].copy_(fdev[0][n], non_blocking=True)
        r1.record(ds)
        torch.cuda.synchronize()
        readback_ms = r0.elapsed_time(r1)
        ems = max_over_ranks(run_loop(True), world, dev)
        rms = max_over_ranks(run_loop(False), world, dev)
        d2h_fields = sum(t.numel() * t.element_size() for t in fhost.values())
        d2h_gauss = gh[0].numel() * 8 if gauss else 0
        result["e2e"] = {"value": round(replica_value(valid, world, ems), 4), "unit": "Gcell-steps/s",
                         "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in host.values()),
                         "d2h_bytes_per_step": d2h_fields + d2h_gauss, "steps": ksteps,
                         "ms_per_step": round(ems, 3), "upload_alone_ms": round(upload_ms, 3),
                         "scatter_ms": round(scatter_ms, 3), "field_readback_alone_ms": round(readback_ms, 3),
                         "what": "per step: J (and rho) on the global grid copied from pinned host (the next "
                                 "step's copy overlapping this step), psatd_scatter_global into the padded "
                                 "boxes, psatd_push, psatd_gather_global of the valid E and B, and E, B and the "
                                 "Gauss sums copied back to pinned host (on a third stream)"}
        result["e2e_fields_resident"] = {
            "value": round(replica_value(valid, world, rms), 4), "unit": "Gcell-steps/s", "ms_per_step": round(rms, 3),
            "d2h_bytes_per_step": d2h_gauss,
            "what": "the same loop with E and B left on the device; only the Gauss sums are read back"}
        del host, gdev, fdev, fhost
        torch.cuda.empty_cache()
    # ---- plain FP64 GPU path and FP32-vs-FP64 agreement ------------------------
    if not args.skip_plain and rank == 0:
        del sol
        torch.cuda.empty_cache()
        s64 = P.Solver(wl, precision="f64", plain=True, gauss=gauss, device=dev)
        fill_solver(s64, wl, dev)
        s64.push(sp)
        torch.cuda.synchronize()
        nst = 2
        e0, e1 = mkev(), mkev()
        e0.record(stream)
        for _ in range(nst):
            s64.push(sp)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / nst
        launches = P.psatd_push_launches(s64.plan)
        del s64
        torch.cuda.empty_cache()
        # the FP32 batched path against FP64 after S steps of each (the FP64
        # reference runs batched: the same arithmetic as the plain FP64 path,
        # one launch per stage, so S = 100 fits in the run)
        S = args.plain_accuracy_steps
        s32 = P.Solver(wl, precision="f32", gauss=gauss, device=dev)
        fill_solver(s32, wl, dev)
        for _ in range(S):
            s32.push(sp)
        torch.cuda.synchronize()
        keep = {n: s32.arenas[n].clone() for n in I.EB_NAMES}
        del s32
        torch.cuda.empty_cache()
        s64 = P.Solver(wl, precision="f64", gauss=gauss, device=dev)
        fill_solver(s64, wl, dev)
        for _ in range(S):
            s64.push(sp)
        torch.cuda.synchronize()
        num = den = 0.0
        comp = {}
        for n in I.EB_NAMES:
            d = (keep[n].double() - s64.arenas[n])
            num += float((d * d).sum())
            den += float((s64.arenas[n] * s64.arenas[n]).sum())
            comp[n] = float(f"{float(d.abs().max() / s64.arenas[n].abs().max()):.3e}")
        pv = valid / (pms / 1e3) / 1e9
        result["plain_f64"] = {"value": round(pv, 5), "unit": "Gcell-steps/s", "ms_per_step": round(pms, 2),
                               "speedup_of_batched_f32": round(value / world / pv, 2),
                               f"f32_vs_f64_rel_l2_after_{S}_steps": float(f"{math.sqrt(num / den):.3e}"),
                               f"f32_vs_f64_max_rel_per_component_after_{S}_steps": comp,
                               "launches_per_step": launches}
        del s64, keep
        torch.cuda.empty_cache()
    # ---- FP32 batched vs FP64 plain over S steps (reported accuracy) -----------
    if args.accuracy_steps and rank == 0:
        torch.cuda.empty_cache()
        a32 = P.Solver(wl, precision="f32", gauss=False, device=dev, tuning=tuning)
        fill_solver(a32, wl, dev)
        for _ in range(args.accuracy_steps):
            a32.push(sp)
        torch.cuda.synchronize()
        keep = {n: a32.arenas[n].clone() for n in I.EB_NAMES}
        del a32
        torch.cuda.empty_cache()
        a64 = P.Solver(wl, precision="f64", plain=True, gauss=False, device=dev)
        fill_solver(a64, wl, dev)
        for _ in range(args.accuracy_steps):
            a64.push(sp)
        torch.cuda.synchronize()
        num = sum(float(((keep[n].double() - a64.arenas[n]) ** 2).sum()) for n in I.EB_NAMES)
        den = sum(float((a64.arenas[n] ** 2).sum()) for n in I.EB_NAMES)
        result["accuracy"] = {"steps": args.accuracy_steps, "f32_batched_vs_f64_plain_rel_l2": float(f"{math.sqrt(num / den):.3e}")}
        del a64, keep
        torch.cuda.empty_cache()
    # ---- the precision and batching workloads, timed the same way --------------
    if args.extra_workloads and rank == 0:
        sol = None
        torch.cuda.empty_cache()
        result["workloads"] = {w: time_workload(w, args, dev, peak) for w in args.extra_workloads.split(",") if w}
    # ---- CPU oracle baseline (rank 0, N = 1 only) -------------------------------
    if not args.skip_cpu and rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_oracle_sample(wl, args.cpu_budget)
    return result


def time_workload(name, args, dev, peak):
    """One more workload through the same plan and timing as the main line
    (FP32 batched with the Gauss diagnostic, persistent grids, default
    shapes): W warm-up steps, then K steps with CUDA events at the stage
    boundaries.  Returns throughput and, per stage, the algorithmic bytes
    over the mean stage time as a fraction of the HBM peak."""
    import torch
    from paper_1707_08500_gb300 import inputs as I
    from paper_1707_08500_gb300 import psatd as P
    wl = I.workload(name)
    prec = "f32" if wl.precision == "f32" else "f64"
    sol = P.Solver(wl, precision=prec, gauss=True, device=dev)
    fill_solver(sol, wl, dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    for _ in range(args.warmup):
        sol.push(sp)
    K = max(args.steps, 10)
    def mkev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)          # recorded once here, so torch treats it as recorded
        return e
    evs = [[mkev() for _ in range(4)] for _ in range(K)]
    t0, t1 = mkev(), mkev()
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(K):
        P.psatd_push_profiled(sol.plan, sol.fields, sol.gauss_out.data_ptr(), sp, [e.cuda_event for e in evs[k]])
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / K
    stage_ms = {st: sum(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K)) / K for i, st in enumerate("ABC")}
    by, local = stage_bytes(wl, 10, 4 if prec == "f32" else 8)
    engine = P.psatd_plane_engine(sol.plan)
    names = {"A": "k_pass_a_reg" if engine & 1 else "k_pass_a", "B": "k_pass_b_reg" if engine & 2 else "k_pass_b",
             "C": "k_pass_c_reg" if engine & 1 else "k_pass_c"}
    stages = {st: {"kernel": names[st], "ms": round(stage_ms[st], 4),
                   "gbs": round(by[st] / (stage_ms[st] / 1e3) / 1e9, 1),
                   "frac": round(by[st] / (stage_ms[st] / 1e3) / 1e9 / peak, 4)} for st in "ABC"}
    dom = max(stage_ms, key=stage_ms.get)
    del sol
    torch.cuda.empty_cache()
    return {"value": round(wl.valid_cells / (ms / 1e3) / 1e9, 4), "unit": "Gcell-steps/s", "ms_per_step": round(ms, 4),
            "steps": K, "warmup": args.warmup, "dtype": prec, "global_n": list(wl.global_n),
            "subdomains": len(wl.subs), "stages": stages,
            "dominant": {"kernel": names[dom], "frac": stages[dom]["frac"], "peak_gbs": peak}}


YEE_METRIC = "Gcell-steps/s of the Yee FDTD step (Eqs. 2a/2b), FP32; % HBM roof"


def run_yee(args, rank, world, local_rank):
    """The Yee FDTD step (the paper's comparison solver) on the workload's
    global grid: one fused kernel per step, fields ping-ponged between two
    device sets.  Algorithmic bytes per cell: read E, B, J, write E, B."""
    import torch
    from paper_1707_08500_gb300 import build as B
    from paper_1707_08500_gb300 import fdtd as F
    from paper_1707_08500_gb300 import inputs as I
    from paper_1707_08500_gb300 import psatd as P

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = I.workload(args.workload)
    prec = args.precision or "f32"
    esz = 4 if prec == "f32" else 8
    dt = 0.5
    sol = F.YeeSolver(wl.global_n, dt, wl.dx, precision=prec, device=dev)
    glob = I.random_fields(wl.global_n, 1707 + 60, names=F.E_NAMES + F.B_NAMES + F.J_NAMES, device=dev)
    sol.load(glob)
    del glob
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)

    def mkev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e
    for _ in range(args.warmup):
        sol.step(stream.cuda_stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0, t1 = mkev(), mkev()
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(args.steps):
            sol.step(stream.cuda_stream)
        t1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev) / args.steps
    nx, ny, nz = wl.global_n
    cells = nx * ny * nz
    alg = 15 * esz * cells
    peak, peak_kind = _peaks()
    achieved = alg / (ms / 1e3) / 1e9
    result = {
        "metric": YEE_METRIC, "value": round(cells * world / (ms / 1e3) / 1e9, 3), "unit": "Gcell-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": f"yee-{wl.name}-grid", "global_n": list(wl.global_n), "c_dt": dt,
                   "l2": f"fields ({15 * esz * cells / 1e9:.1f} GB per step) larger than L2; no flush",
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
        "roofline": {"bound": "hbm", "kernel": "k_yee", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": _yee_traffic(wl.name), "peak_kind": peak_kind,
                     "alg_bytes_per_cell": 15 * esz},
        "gpu_launches": args.steps * P.psatd_yee_launches(),
        "clocks": clk.summary(),
    }
    if not args.skip_e2e:
        host = {n: torch.empty_like(sol.J[n], device="cpu").pin_memory() for n in F.J_NAMES}
        for n in F.J_NAMES:
            host[n].copy_(sol.J[n])
        probe = torch.empty((ny, nx), dtype=sol.dtype, pin_memory=True)
        k = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        e0, e1 = mkev(), mkev()
        e0.record(stream)
        for _ in range(k):
            for n in F.J_NAMES:
                sol.J[n].copy_(host[n], non_blocking=True)
            sol.step(stream.cuda_stream)
            probe.copy_(sol.sets[sol.cur]["Ez"][nz // 2], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), world, dev) / k
        result["e2e"] = {"value": round(cells * world / (ems / 1e3) / 1e9, 3), "unit": "Gcell-steps/s",
                         "h2d_bytes_per_step": 3 * cells * esz, "d2h_bytes_per_step": nx * ny * esz,
                         "ms_per_step": round(ems, 3),
                         "what": "per step: J copied from pinned host, psatd_yee_step, one Ez plane read back"}
        del host
    if not args.skip_cpu and rank == 0 and world == 1:
        result["cpu_baseline"] = yee_cpu_sample(args.cpu_budget)
    return result


HEAT_METRIC = "Gcell-steps/s of the local-FFT heat-equation step (exact per-mode decay), FP32; % HBM roof"


def run_heat(args, rank, world, local_rank):
    """The local-FFT heat equation (PSATD_HEAT) with a source on the
    workload's decomposition: the same three stages with one field out (two
    in).  D dt = 0.5 cell^2."""
    import torch
    from paper_1707_08500_gb300 import build as B
    from paper_1707_08500_gb300 import inputs as I
    from paper_1707_08500_gb300 import psatd as P

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = I.workload(args.workload)
    prec = args.precision or "f32"
    esz = 4 if prec == "f32" else 8
    d_dt = 0.5
    sol = P.HeatSolver(wl, d_dt, source=True, precision=prec, device=dev)
    g = I.random_fields(wl.global_n, 1707 + 72, names=("Jx", "Jy"), device=dev)
    sol.load_global({"T": g["Jx"], "S": 0.01 * g["Jy"]}, names=("T", "S"), guards=True)
    del g
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def mkev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e
    for _ in range(args.warmup):
        sol.push(sp)
    torch.cuda.synchronize()
    evs = [[mkev() for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    t0, t1 = mkev(), mkev()
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(args.steps):
            P.psatd_push_profiled(sol.plan, sol.fields, None, sp, [e.cuda_event for e in evs[k]])
        t1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev) / args.steps
    stage_ms = {st: sum(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)) / args.steps
                for i, st in enumerate("ABC")}
    by, local = stage_bytes(wl, 2, esz, nout=1)
    peak, peak_kind = _peaks()
    dom = max(stage_ms, key=stage_ms.get)
    reg = P.psatd_plane_engine(sol.plan) & 1
    names = {"A": "k_pass_a_reg" if reg else "k_pass_a", "B": "k_pass_b_heat", "C": "k_pass_c_reg" if reg else "k_pass_c"}
    achieved = by[dom] / (stage_ms[dom] / 1e3) / 1e9
    valid = wl.valid_cells
    result = {
        "metric": HEAT_METRIC, "value": round(replica_value(valid, world, ms), 4), "unit": "Gcell-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": f"heat-{wl.name}", "global_n": list(wl.global_n), "subdomains": len(wl.subs),
                   "local_n": list(wl.subs[0].local), "guards": wl.subs[0].ng, "order": wl.subs[0].p, "d_dt": d_dt,
                   "source": True, "l2": f"inputs ({local * 2 * esz / 1e9:.1f} GB) larger than L2; no flush",
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
        "stages": {st: {"kernel": names[st], "ms": round(stage_ms[st], 3), "alg_bytes": by[st],
                        "gbs": round(by[st] / (stage_ms[st] / 1e3) / 1e9, 1),
                        "frac": round(by[st] / (stage_ms[st] / 1e3) / 1e9 / peak, 4)} for st in "ABC"},
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind},
        "step_roofline": {"three_pass_bytes_per_step": sum(by.values()),
                          "frac_three_pass": round(sum(by.values()) / (ms / 1e3) / 1e9 / peak, 4)},
        "gpu_launches": args.steps * P.psatd_push_launches(sol.plan),
        "clocks": clk.summary(),
    }
    if not args.skip_cpu and rank == 0 and world == 1:
        result["cpu_baseline"] = heat_cpu_sample(wl, args.cpu_budget)
    return result


def heat_cpu_sample(wl, budget_s: float):
    """The FP64 heat oracle on whole subdomain steps until the budget is spent."""
    from oracle import heat_oracle as H
    import numpy as np
    rng = np.random.default_rng(1)
    t_used, cells, nsub = 0.0, 0, 0
    for sd in wl.subs[:: max(1, len(wl.subs) // 64)]:
        lx, ly, lz = sd.local
        T, S = rng.standard_normal((lz, ly, lx)), rng.standard_normal((lz, ly, lx))
        t0 = time.perf_counter()
        H.local_heat_push(T, S, sd.local, wl.dx, sd.p, 0.5)
        t_used += time.perf_counter() - t0
        cells += sd.n[0] * sd.n[1] * sd.n[2]
        nsub += 1
        if t_used > budget_s:
            break
    from oracle import psatd_oracle as O
    return {"value": cells / t_used / 1e9, "unit": "Gcell-steps/s", "cores": O.WORKERS, "kind": "oracle",
            "sample": f"{nsub} of {len(wl.subs)} subdomain steps ({cells} valid cells), {t_used:.1f} s"}


def _yee_traffic(workload: str):
    """DRAM bytes per Yee launch from the committed ncu summary, if it was
    taken on the current kernel source and this workload's grid (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic_yee.json")) as f:
            t = json.load(f)
        with open(os.path.join(ROOT, "paper_1707_08500_gb300", "csrc", "fdtd_yee.cu"), "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
        if t.get("kernel_sha256") != sha or t.get("workload") != workload:
            return None
        return t["bytes_per_launch"].get("k_yee")
    except Exception:
        return None


def yee_cpu_sample(budget_s: float):
    """The FP64 Yee oracle on a 256 x 128 x 128 grid, repeated until the budget is spent."""
    from oracle import yee_oracle as Y
    from paper_1707_08500_gb300 import inputs as I
    n = (256, 128, 128)
    f = {k: v.numpy() for k, v in I.random_fields(n, 1707 + 61, names=Y.E_NAMES + Y.B_NAMES + ("Jx", "Jy", "Jz")).items()}
    steps, t = 0, 0.0
    while t < budget_s:
        t0 = time.perf_counter()
        f = Y.yee_step(f, (1.0, 1.0, 1.0), 0.5)
        t += time.perf_counter() - t0
        steps += 1
    cells = n[0] * n[1] * n[2]
    return {"value": cells * steps / t / 1e9, "unit": "Gcell-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of a {n[0]}x{n[1]}x{n[2]} grid, {t:.1f} s"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, timed as it stands on the host cores."""
    from oracle import psatd_oracle as O
    from paper_1707_08500_gb300 import inputs as I
    if rank != 0:
        return None
    if args.solver == "heat":
        c = heat_cpu_sample(I.workload(args.workload), max(5.0, args.cpu_budget))
        return {"impl": "reference", "metric": HEAT_METRIC, "value": round(c["value"], 6), "unit": c["unit"],
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"heat-{args.workload} (oracle on a bounded sample)"},
                "cpu_baseline": c,
                "e2e": {"value": round(c["value"], 6), "unit": c["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if args.solver == "yee":
        c = yee_cpu_sample(max(5.0, args.cpu_budget))
        return {"impl": "reference", "metric": YEE_METRIC, "value": round(c["value"], 6), "unit": c["unit"],
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"yee-{args.workload}-grid (oracle on a bounded sample)"},
                "cpu_baseline": c,
                "e2e": {"value": round(c["value"], 6), "unit": c["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    wl = I.workload(args.workload)
    per_step = max(1, int(args.ref_subs))
    boxes = [(sd, {k: v.numpy() for k, v in I.box_fields(wl, sd, device="cpu").items()})
             for sd in wl.subs[:per_step]]

    def one():
        for sd, b in boxes:
            O.local_push(b, sd.local, wl.dx, sd.p, wl.c_dt, wl.staggered)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    cells = sum(sd.n[0] * sd.n[1] * sd.n[2] for sd, _ in boxes)
    v = cells / dt / 1e9
    sample = f"each step = {len(boxes)} of {len(wl.subs)} subdomain pushes ({cells} valid cells)"
    return {"impl": "reference", "metric": METRIC,
            "value": round(v, 6), "unit": "Gcell-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "global_n": list(wl.global_n), "subdomains": len(wl.subs)},
            "cpu_baseline": {"value": round(v, 6), "unit": "Gcell-steps/s", "cores": O.WORKERS,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 6), "unit": "Gcell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _free_port() -> int:
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def launch_replicas(args) -> int:
    """--gpus N without a launcher: start N ranks of this script on this node
    (one per GPU, torch.distributed.run on 127.0.0.1) and return their exit
    status.  Each rank runs an independent replica of the workload; the
    ranks share only the barrier and the max over ranks of the timed region."""
    if args.impl == "ours":
        import torch
        have = torch.cuda.device_count()
        if have < args.gpus:
            print(f"bench.py: --gpus {args.gpus} but {have} GPU(s) are visible", file=sys.stderr)
            return 2
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.run(cmd).returncode


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mirror1024")
    ap.add_argument("--no-gauss", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-subs", type=int, default=2)
    ap.add_argument("--chunk-b", type=int, default=0, help="pass-B chunk width (0 = plan default)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (plan default shapes)")
    ap.add_argument("--precision", choices=["f32", "f64"], default=None, help="default: the workload's")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay measurement")
    ap.add_argument("--grid-per-item", action="store_true", help="one CTA per work item instead of persistent grids")
    ap.add_argument("--generic-planes", action="store_true",
                    help="FP32: the generic plane stages instead of the compiled-length ones")
    ap.add_argument("--accuracy-steps", type=int, default=0, help="also report FP32 batched vs FP64 plain after S steps")
    ap.add_argument("--plain-accuracy-steps", type=int, default=100,
                    help="steps of the FP32-vs-FP64 comparison reported with the plain FP64 path")
    ap.add_argument("--extra-workloads", default="broadband256,uneven48",
                    help="comma-separated workloads also timed after the main one (empty: none)")
    ap.add_argument("--solver", choices=["psatd", "yee", "heat"], default="psatd",
                    help="yee: the FDTD comparison solver on the workload's global grid; "
                         "heat: the local-FFT heat equation on the workload's decomposition")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.gpus < 1:
        ap.error("--gpus must be at least 1")
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        sys.exit(launch_replicas(args))
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if world != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but the launcher started {world} rank(s)", file=sys.stderr)
        sys.exit(2)
    print(f"bench.py: rank {rank} of {world} started", file=sys.stderr, flush=True)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    runner = {"yee": run_yee, "heat": run_heat}.get(args.solver, run_ours)
    out = runner(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
