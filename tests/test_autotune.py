"""Host logic of the batched planner's autotuner on CPU, with the library's
Batch replaced by a fake that returns scripted timings and statistics: the
candidate shapes it enumerates, that each candidate is planned twice and the
second (warm) plan is the one ranked, the ranking (more solved problems first,
then the shorter batch, then the lower median first-solution time, unsolved
samples last), and that an empty shape list skips its launch form."""
import pytest

from paper_2609_30533_gb300 import autotune as AT
from paper_2609_30533_gb300 import stp


class _Problem:
    def __init__(self, W):
        self.W = W
        self.closed = False

    def close(self):
        self.closed = True


def _stats(solved, first_ms):
    out = []
    for k in range(4):
        ok = k < solved
        out.append({"first_solution_ms": first_ms if ok else 0.0, "first_solution_iter": 3 if ok else -1,
                    "edges_validated": 100, "bridges_validated": 10})
    return out


def _fake_batch(script, log):
    """script[(W, mode, team, nn, vc)] = (batch_ms, solved, first_ms)."""

    class FakeBatch:
        def __init__(self, probs, nn_ctas=0, validate_ctas=0, iters_per_graph=0, launch_mode=0, team_ctas=0):
            self.key = (probs[0].W, launch_mode, team_ctas, nn_ctas, validate_ctas)
            self.calls = 0
            log.append(self.key)

        def plan(self):
            self.calls += 1
            ms, solved, first = script[self.key]
            if self.calls == 1:                     # warm-up: a misleading figure that must not count
                return 0.001, _stats(4, 0.001)
            return ms, _stats(solved, first)

        def close(self):
            pass

    return FakeBatch


def _run(monkeypatch, script, **kw):
    log, made = [], []
    monkeypatch.setattr(stp, "Batch", _fake_batch(script, log))

    def make(W):
        ps = [_Problem(W) for _ in range(4)]
        made.extend(ps)
        return ps

    choice = AT.autotune(make, **kw)
    assert all(p.closed for p in made)
    return choice, log


def _script(workers, teams, nns, vcs, default=(10.0, 2, 5.0)):
    s = {}
    for W in workers:
        for t in teams:
            s[(W, 0, t, 0, 0)] = default
        for nn in nns:
            for vc in vcs:
                s[(W, 1, 0, nn, vc)] = default
    return s


def test_enumerates_every_shape_for_every_width(monkeypatch):
    s = _script((128, 256), (2, 4), (4, 8), (1, 2))
    choice, log = _run(monkeypatch, s, workers=(128, 256), team_ctas=(2, 4), nn_ctas=(4, 8), validate_ctas=(1, 2))
    assert sorted(log) == sorted(s)             # each candidate once, in one batch object
    assert len(choice.trials) == len(s)
    assert {(t.workers, t.launch_mode, t.team_ctas, t.nn_ctas, t.validate_ctas) for t in choice.trials} == set(s)


def test_more_solved_beats_a_faster_batch(monkeypatch):
    s = _script((256,), (4,), (8,), (2,))
    s[(256, 0, 4, 0, 0)] = (5.0, 2, 1.0)        # fastest, fewer solved
    s[(256, 1, 0, 8, 2)] = (50.0, 3, 9.0)       # slow, more solved
    choice, _ = _run(monkeypatch, s, workers=(256,), team_ctas=(4,), nn_ctas=(8,), validate_ctas=(2,))
    assert (choice.launch_mode, choice.nn_ctas, choice.validate_ctas) == (1, 8, 2)


def test_equal_solved_ranks_by_batch_time_then_median_first_solution(monkeypatch):
    s = _script((128, 256), (4, 8), (), ())
    s[(128, 0, 4, 0, 0)] = (20.0, 3, 1.0)
    s[(128, 0, 8, 0, 0)] = (12.0, 3, 7.0)
    s[(256, 0, 4, 0, 0)] = (12.0, 3, 6.0)       # same time as the one above, lower median: wins
    s[(256, 0, 8, 0, 0)] = (30.0, 3, 0.5)
    choice, _ = _run(monkeypatch, s, workers=(128, 256), team_ctas=(4, 8), nn_ctas=(), validate_ctas=())
    assert (choice.workers, choice.launch_mode, choice.team_ctas) == (256, 0, 4)
    t = [x for x in choice.trials if (x.workers, x.team_ctas) == (256, 4)][0]
    assert t.batch_ms == 12.0 and t.solved == 3 and t.p50_first_ms == 6.0
    assert t.edges_per_s == pytest.approx(4 * 110 / 12e-3)


def test_unsolved_sample_ranks_last_on_ties(monkeypatch):
    s = _script((256,), (4, 8), (), ())
    s[(256, 0, 4, 0, 0)] = (10.0, 0, 0.0)       # nothing solved: median is infinite
    s[(256, 0, 8, 0, 0)] = (10.0, 0, 0.0)
    choice, _ = _run(monkeypatch, s, workers=(256,), team_ctas=(4, 8), nn_ctas=(), validate_ctas=())
    assert all(t.p50_first_ms == float("inf") for t in choice.trials)
    assert choice.team_ctas == 4                # full tie: the first candidate stays


@pytest.mark.parametrize("form", ["queue", "steps"])
def test_empty_shape_lists_skip_a_launch_form(monkeypatch, form):
    teams, nns, vcs = ((4,), (), ()) if form == "queue" else ((), (8,), (2,))
    s = _script((256,), teams, nns, vcs)
    choice, log = _run(monkeypatch, s, workers=(256,), team_ctas=teams, nn_ctas=nns, validate_ctas=vcs)
    modes = {k[1] for k in log}
    assert modes == ({0} if form == "queue" else {1})
    assert choice.launch_mode == (0 if form == "queue" else 1)
