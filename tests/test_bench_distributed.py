"""Host logic of bench.py's multi-GPU mode on CPU: two gloo ranks.

With N GPUs the bench runs N independent replicas of the workload (the path
is replicated, not sharded: no collective on the data path); the only
cross-rank operations are the barrier and the max over ranks of the timed
duration, from which the whole-job throughput is computed."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slowest
        worst = bench.max_over_ranks(ms, world)
        dist.barrier()
        out[rank] = (worst, bench.replica_value(1_000_000, world, worst))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    worst, value = res[0]
    assert worst == 15.0
    assert value == pytest.approx(2 * 1_000_000 / 0.015 / 1e9)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_value(268435456, 1, 100.0) == pytest.approx(2.68435456)


def test_stage_byte_model_matches_the_documented_per_cell_figures():
    """Algorithmic bytes per local cell of the three stages on 96^3 boxes with
    16 guards, FP32, 10 fields in (80.8, 57.2 and 40.3 B per local cell)."""
    import bench
    from paper_1707_08500_gb300 import inputs as I
    wl = I.workload("mirror1024")
    by, local = bench.stage_bytes(wl, 10, 4)
    per = {k: v / local for k, v in by.items()}
    assert abs(per["A"] - 80.83) < 0.01 and abs(per["B"] - 57.17) < 0.01 and abs(per["C"] - 40.33) < 0.01, per
    # heat: two fields in, one out
    by, _ = bench.stage_bytes(wl, 2, 4, nout=1)
    assert abs(by["A"] / local - 2 * (4 + 49 * 8 / 96)) < 1e-6


@pytest.mark.parametrize("solver", ["psatd", "yee", "heat"])
def test_reference_arm_prints_one_json_line(solver):
    """bench.py --impl reference runs the FP64 oracle on the host cores and
    prints one JSON line with the reference fields (no GPU involved)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    args = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3",
            "--ref-subs", "1", "--cpu-budget", "1", "--solver", solver]
    if solver == "heat":
        args += ["--workload", "plain32"]
    r = subprocess.run(args, capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_gpus_flag_starts_that_many_ranks():
    """bench.py --gpus 2 started without a launcher starts two ranks itself
    (torch.distributed.run on 127.0.0.1); on the reference arm rank 0 alone
    prints the JSON line, with n_gpus = 2, and the other rank exits 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3", "--ref-subs", "1", "--workload", "plain32"],
                       capture_output=True, text=True, timeout=600, cwd=root, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    started = sorted(l for l in r.stderr.splitlines() if "started" in l and l.startswith("bench.py: rank"))
    assert started == ["bench.py: rank 0 of 2 started", "bench.py: rank 1 of 2 started"], r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    assert json.loads(lines[0])["n_gpus"] == 2


def test_rank_count_mismatch_fails_loudly():
    """Under a launcher whose world size differs from --gpus the bench refuses
    to run instead of mislabelling its line."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, timeout=300, cwd=root, env=env)
    assert r.returncode == 2 and "--gpus 2" in r.stderr
