"""bench.autotune_refine's choice, on CPU, with a stand-in for the batch.

The autotuner runs the uneven batch with one and with two reduced refinement passes in the
first solve and 2, 3, 4 or 8 passes on the KKT residual.  For each reduced count it keeps the
smallest KKT count that reaches that count's best gate figure; of those pairs that reach the
best figure overall it keeps the one whose captured step replays fastest.  The stand-in
reports a residual and a replay time set per configuration, so the rule can be checked
without a GPU."""
import numpy as np
import pytest

import bench
from paper_2407_05433_gb300 import eclqr

P = 6


def _fake_batch(passes_table, replay_ms, made):
    class FakeBatch:
        def __init__(self, pbs, device=None, refine=2, corr_refine=-1, kkt_refine=8, team_warps=0):
            assert corr_refine == bench.CORR_REFINE
            self.key = (refine, kkt_refine)
            made.append(self.key)
            ok = passes_table[self.key]
            self.resid = _Arr(np.where(np.arange(P) < ok, 1e-12, 1e-6))
            self.status = _Arr(np.zeros(P, np.int32))

        def run(self):
            pass

        def capture(self):
            return 100

        def replay(self):
            pass

        def close(self):
            pass

    return FakeBatch


class _Arr:
    def __init__(self, a):
        self.a = a

    def cpu(self):
        return self

    def numpy(self):
        return self.a


@pytest.fixture
def patched(monkeypatch):
    def install(passes_table, replay_ms):
        made = []
        monkeypatch.setattr(eclqr, "Batch", _fake_batch(passes_table, replay_ms, made))
        monkeypatch.setattr(bench, "_time_runs", lambda b, steps, flush, stream: [10.0 + b.key[1]])
        monkeypatch.setattr(bench, "_time_replays", lambda b, steps, flush, stream: [replay_ms[b.key]] * steps)
        return made
    return install


def _run(pbs=None):
    return bench.autotune_refine(pbs or [None] * P, "cpu", {}, None, None)


def test_fewest_kkt_passes_at_the_best_gate_then_the_faster_replay(patched):
    table = {(1, 2): 5, (1, 3): 6, (1, 4): 6, (1, 8): 6, (2, 2): 6, (2, 3): 6, (2, 4): 6, (2, 8): 6}
    replay = {(1, 3): 90.0, (2, 2): 95.0}
    made = patched(table, replay)
    refine, kr, trials = _run()
    assert (refine, kr) == (1, 3)
    assert [tuple(t) for t in trials["replay"]] == [(1, 3, 90.0), (2, 2, 95.0)]
    assert len(trials["eager"]) == 8 and made[-2:] == [(1, 3), (2, 2)]


def test_a_reduced_count_below_the_best_gate_is_not_replayed(patched):
    table = {(1, 2): 4, (1, 3): 5, (1, 4): 5, (1, 8): 5, (2, 2): 5, (2, 3): 6, (2, 4): 6, (2, 8): 6}
    replay = {(2, 3): 120.0}
    made = patched(table, replay)
    refine, kr, trials = _run()
    assert (refine, kr) == (2, 3)
    assert [tuple(t) for t in trials["replay"]] == [(2, 3, 120.0)]
    assert (1, 2) not in made[8:]


def test_slower_replay_loses_even_with_fewer_passes(patched):
    table = {k: 6 for k in [(r, p) for r in (1, 2) for p in (2, 3, 4, 8)]}
    replay = {(1, 2): 130.0, (2, 2): 110.0}
    patched(table, replay)
    refine, kr, _ = _run()
    assert (refine, kr) == (2, 2)
