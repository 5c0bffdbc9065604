"""The autotuner's selection logic on the host, with a fake timer in place of
GPU launches: the default shapes are a candidate in every coordinate, and a
shape that is slower than the default over the whole step is not returned."""
import pytest

from paper_1707_08500_gb300 import inputs as I
from paper_1707_08500_gb300 import tune as T

DEFAULT = {"chunk_b": 0, "f1": [0, 0, 0]}


def _fake_bench(stage_ms, calls):
    class Fake:
        def __init__(self, wl, flags, device):
            pass

        def time(self, tuning, reps=3):
            calls.append({"chunk_b": tuning["chunk_b"], "f1": list(tuning["f1"])})
            return stage_ms(tuning)

        def agrees_with_default(self, tuning, tol=1e-5, sample=1 << 22):
            return True
    return Fake


def _wl():
    return I.workload("broadband256")


def test_split_that_only_helps_a_and_c_is_rejected_over_the_whole_step(monkeypatch):
    """A non-default x split makes passes A and C 5% faster but pass B 50%
    slower (as when a split tuned on one box takes mixed boxes off the
    compiled-length kernels): the per-axis search prefers it, the whole-step
    check does not."""
    def ms(t):
        x = t["f1"][0] != 0
        return [0.95 if x else 1.0, 1.5 if x else 1.0, 0.95 if x else 1.0]
    calls = []
    monkeypatch.setattr(T, "_Bench", _fake_bench(ms, calls))
    best = T.autotune(_wl(), 0, device="cpu", use_cache=False, reps=1)
    assert best == DEFAULT
    assert any(c["f1"][0] != 0 for c in calls)          # the split was tried


def test_default_is_kept_when_no_candidate_is_faster(monkeypatch):
    calls = []
    monkeypatch.setattr(T, "_Bench", _fake_bench(lambda t: [1.0, 1.0 + 0.01 * t["chunk_b"], 1.0], calls))
    assert T.autotune(_wl(), 0, device="cpu", use_cache=False, reps=1) == DEFAULT


def test_faster_chunk_is_picked(monkeypatch):
    """A chunk width that makes pass B faster without touching A and C wins."""
    calls = []
    monkeypatch.setattr(T, "_Bench", _fake_bench(lambda t: [1.0, 0.8 if t["chunk_b"] == 4 else 1.0, 1.0], calls))
    best = T.autotune(_wl(), 0, device="cpu", use_cache=False, reps=1)
    assert best["chunk_b"] == 4 and best["f1"][:2] == [0, 0]


@pytest.mark.parametrize("agree", [True, False])
def test_disagreeing_shape_falls_back_to_default(monkeypatch, agree):
    calls = []
    Fake = _fake_bench(lambda t: [1.0, 0.8 if t["chunk_b"] == 4 else 1.0, 1.0], calls)
    Fake.agrees_with_default = lambda self, tuning, tol=1e-5, sample=1 << 22: agree
    monkeypatch.setattr(T, "_Bench", Fake)
    best = T.autotune(_wl(), 0, device="cpu", use_cache=False, reps=1)
    assert (best["chunk_b"] == 4) == agree
