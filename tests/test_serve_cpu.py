"""Host-side policy of the serving loop, on the CPU: admission by the HBM
budget, least-recently-used eviction of idle instances, the per-pattern
instance cap, failure of a pattern that cannot fit at all, and the Poisson
arrival generator.  The engine runs unchanged; only the library handle and
the device allocations are replaced by fakes that keep the bookkeeping a
real handle would report (device bytes, completion after a few polls)."""
from dataclasses import dataclass

import numpy as np
import pytest

from paper_2309_11488_gb300 import opm, serve


@dataclass
class _Pat:
    nb: int
    nnzb: int
    rowptr: np.ndarray = None
    colidx: np.ndarray = None
    vals: np.ndarray = None


class _Dev:
    """Stand-in for a device tensor: .cuda() and .clone() return itself."""

    def cuda(self):
        return self

    def clone(self):
        return self


class _FakeTorch:
    class cuda:
        @staticmethod
        def Stream():
            return object()

        @staticmethod
        def synchronize():
            pass

    float64 = "float64"

    @staticmethod
    def from_numpy(a):
        return _Dev()

    @staticmethod
    def empty(*a, **k):
        return _Dev()


class _FakeSolver:
    """Records the handles alive; a launched solve completes after `polls`
    calls of ready()."""
    alive = []
    created = 0
    polls = 3
    bytes_per_row = 1000

    def __init__(self, nb, rp, ci, va, schedule, precision, stream):
        self.nb, self.left, self.closed = nb, 0, False
        _FakeSolver.alive.append(self)
        _FakeSolver.created += 1

    def info(self):
        return type("I", (), {"device_bytes": self.nb * _FakeSolver.bytes_per_row})()

    def launch(self, vals, b, x, rtol, maxit):
        assert self.left == 0 and not self.closed, "launch on a busy or closed handle"
        self.left = _FakeSolver.polls

    def ready(self):
        self.left = max(0, self.left - 1)
        return self.left == 0

    def wait(self):
        return opm.OPM_OK, 5, 1e-3

    def close(self):
        assert self.left == 0, "a busy handle was closed"
        self.closed = True
        _FakeSolver.alive.remove(self)


@pytest.fixture
def fake(monkeypatch):
    _FakeSolver.alive, _FakeSolver.created, _FakeSolver.polls = [], 0, 3
    monkeypatch.setattr(serve.opm, "Solver", _FakeSolver)

    def make(patterns, budget, **kw):
        eng = serve.ServingEngine(patterns, hbm_budget_bytes=budget, **kw)
        eng.torch = _FakeTorch()
        eng._bytes_seen = {p: s.nb * _FakeSolver.bytes_per_row for p, s in enumerate(patterns)}
        return eng
    return make


def _requests(seq, t=0.0):
    return [serve.Request(rid=i, t_arrival=t, pattern=p, vals=None, b=None) for i, p in enumerate(seq)]


def test_budget_is_never_exceeded_and_lru_idle_instances_are_evicted(fake):
    pats = [_Pat(100, 600) for _ in range(3)]
    eng = fake(pats, budget=2 * 100 * 1000)  # room for two instances
    _FakeSolver.polls = 1
    stats = eng.run(_requests([0, 1, 2, 0, 1, 2, 2, 0]))
    assert stats.completed == 8 and stats.failed == 0
    assert stats.hbm_bytes_peak <= eng.budget
    assert sum(s.nb * 1000 for s in _FakeSolver.alive) == eng.hbm_bytes <= eng.budget
    assert stats.evictions >= 1 and len(eng.instances) <= 2


def test_eviction_picks_the_least_recently_used_idle_instance(fake):
    pats = [_Pat(100, 600) for _ in range(3)]
    eng = fake(pats, budget=2 * 100 * 1000)
    a, b = eng.add_instance(0), eng.add_instance(1)
    a.last_used, b.last_used = 5.0, 1.0  # pattern 1 is the older
    c = eng.add_instance(2)
    assert c is not None and eng.evictions == 1
    assert set(eng.by_pattern[0]) == {a.iid} and eng.by_pattern[1] == [] and b.solver.closed


def test_busy_instances_are_never_evicted(fake):
    pats = [_Pat(100, 600) for _ in range(3)]
    eng = fake(pats, budget=2 * 100 * 1000)
    a, b = eng.add_instance(0), eng.add_instance(1)
    a.busy = b.busy = object()
    assert eng.add_instance(2) is None and eng.evictions == 0
    assert not a.solver.closed and not b.solver.closed


def test_the_only_instance_of_the_admitted_pattern_is_kept(fake):
    pats = [_Pat(100, 600)]
    eng = fake(pats, budget=150 * 1000, max_instances_per_pattern=4)
    a = eng.add_instance(0)
    # a second instance of pattern 0 would need evicting the only one: refused
    assert eng.add_instance(0) is None and not a.solver.closed and eng.evictions == 0


def test_instances_per_pattern_are_capped_and_excess_requests_wait(fake):
    pats = [_Pat(10, 60)]
    eng = fake(pats, budget=1 << 30, max_instances_per_pattern=2)
    _FakeSolver.polls = 4
    stats = eng.run(_requests([0] * 7))
    assert stats.completed == 7 and len(eng.by_pattern[0]) == 2 and _FakeSolver.created == 2
    assert stats.max_in_flight == 2 and stats.deferred_admissions > 0


def test_a_pattern_that_cannot_fit_alone_fails_with_oom(fake):
    pats = [_Pat(10, 60), _Pat(10_000, 60_000)]
    eng = fake(pats, budget=1_000_000)
    _FakeSolver.polls = 1
    reqs = _requests([0, 1, 0])
    stats = eng.run(reqs)
    assert stats.completed == 2 and stats.failed == 1 and reqs[1].status == opm.OPM_ERR_OOM
    for r in (reqs[0], reqs[2]):
        assert r.status == opm.OPM_OK and r.t_arrival <= r.t_start <= r.t_done


def test_warm_creates_one_instance_per_pattern_within_the_budget(fake):
    pats = [_Pat(100, 600) for _ in range(4)]
    eng = fake(pats, budget=3 * 100 * 1000)
    eng.warm()
    assert len(eng.instances) == 3 and eng.hbm_bytes == 3 * 100 * 1000
    eng.close()
    assert _FakeSolver.alive == [] and eng.hbm_bytes == 0


def test_poisson_arrivals_are_seeded_sorted_and_at_the_rate():
    t = serve.poisson_arrivals(200.0, 50.0, seed=3)
    assert np.array_equal(t, serve.poisson_arrivals(200.0, 50.0, seed=3))
    assert not np.array_equal(t, serve.poisson_arrivals(200.0, 50.0, seed=4))
    assert np.all(np.diff(t) > 0) and t[-1] < 50.0
    # 10,000 expected arrivals: the count's standard deviation is 100
    assert abs(len(t) - 10_000) < 500
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200) < 0.05 / 200 and abs(gaps.std() / gaps.mean() - 1) < 0.05
