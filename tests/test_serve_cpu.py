"""Host-side policy of the serving loop, on the CPU: admission of lanes by the
HBM budget, least-recently-used eviction of idle lanes, the per-class lane
cap, batched launches of the ready requests of a class, failure of a class
that cannot fit at all, analyses made once per pattern and kept across
evictions, and the Poisson arrival generator.  The engine runs unchanged;
only the library objects (analysis, handle, batch) and the device
allocations are replaced by fakes that keep the bookkeeping the real ones
report (device bytes, completion after a few polls, members sitting out)."""
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


BYTES_PER_ROW = 1000  # device bytes of an instance and its output buffer, per row


class _FakeAnalysis:
    made = []

    def __init__(self, nb, rowptr, colidx, schedule):
        self.nb, self.closed = nb, False
        _FakeAnalysis.made.append(self)

    def close(self):
        self.closed = True


class _FakeSolver:
    alive = []

    @classmethod
    def from_analysis(cls, an, vals, precision, stream):
        assert not an.closed
        self = cls()
        self.nb, self.closed, self.h = an.nb, False, object()
        _FakeSolver.alive.append(self)
        return self

    def info(self):
        return type("I", (), {"device_bytes": self.nb * (BYTES_PER_ROW - 24)})()

    def close(self):
        self.closed = True
        _FakeSolver.alive.remove(self)


class _FakeBatch:
    """A launch completes after `polls` calls of ready(); members with b =
    None sit out and report (OK, 0, 0.0)."""
    polls = 3
    launches = []

    def __init__(self, handles, stream=None):
        self.n, self.left, self.busy, self.closed = len(handles), 0, False, False

    def launch(self, vals, bs, xs, rtol, maxit):
        assert not self.busy and not self.closed, "launch on a busy or closed batch"
        assert len(bs) == len(xs) == self.n
        self.active = [b is not None for b in bs]
        assert all((b is None) == (x is None) for b, x in zip(bs, xs))
        _FakeBatch.launches.append(sum(self.active))
        self.busy, self.left = True, _FakeBatch.polls
        return opm.OPM_OK

    def ready(self):
        self.left = max(0, self.left - 1)
        return self.left == 0

    def wait(self):
        self.busy = False
        st = [opm.OPM_OK] * self.n
        it = [5 if a else 0 for a in self.active]
        rr = [1e-3 if a else 0.0 for a in self.active]
        return opm.OPM_OK, st, it, rr

    def close(self):
        assert not self.busy, "a busy lane was closed"
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    _FakeSolver.alive, _FakeAnalysis.made, _FakeBatch.launches, _FakeBatch.polls = [], [], [], 3
    monkeypatch.setattr(serve.opm, "Solver", _FakeSolver)
    monkeypatch.setattr(serve.opm, "Analysis", _FakeAnalysis)
    monkeypatch.setattr(serve.opm, "Batch", _FakeBatch)

    def make(patterns, budget, **kw):
        eng = serve.ServingEngine(patterns, hbm_budget_bytes=budget, **kw)
        eng.torch = _FakeTorch()
        eng._bytes_seen = {p: s.nb * BYTES_PER_ROW for p, s in enumerate(patterns)}
        return eng
    return make


def _requests(seq, t=0.0):
    return [serve.Request(rid=i, t_arrival=t, pattern=p, vals=_Dev(), b=_Dev()) for i, p in enumerate(seq)]


def test_budget_is_never_exceeded_and_lru_idle_lanes_are_evicted(fake):
    pats = [_Pat(100, 600) for _ in range(3)]
    eng = fake(pats, budget=2 * 100 * BYTES_PER_ROW, class_size=1, lanes_per_class=1)  # room for two lanes
    _FakeBatch.polls = 1
    stats = eng.run(_requests([0, 1, 2, 0, 1, 2, 2, 0]))
    assert stats.completed == 8 and stats.failed == 0
    assert stats.hbm_bytes_peak <= eng.budget
    assert sum(s.nb * BYTES_PER_ROW for s in _FakeSolver.alive) == eng.hbm_bytes <= eng.budget
    assert stats.evictions >= 1 and len(eng.lanes) <= 2
    # each pattern analysed once, however often its lane was evicted and remade
    assert len(_FakeAnalysis.made) == 3 and stats.lanes_created > 2


def test_eviction_picks_the_least_recently_used_idle_lane(fake):
    pats = [_Pat(100, 600) for _ in range(3)]
    eng = fake(pats, budget=2 * 100 * BYTES_PER_ROW, class_size=1, lanes_per_class=1)
    a, b = eng.add_lane(0), eng.add_lane(1)
    a.last_used, b.last_used = 5.0, 1.0  # class 1's lane is the older
    c = eng.add_lane(2)
    assert c is not None and eng.evictions == 1
    assert eng.by_class[0] == [a.lid] and eng.by_class[1] == [] and b.solvers[0].closed and b.batch.closed


def test_lanes_of_classes_with_waiting_requests_are_evicted_last(fake):
    pats = [_Pat(100, 600) for _ in range(3)]
    eng = fake(pats, budget=2 * 100 * BYTES_PER_ROW, class_size=1, lanes_per_class=1)
    a, b = eng.add_lane(0), eng.add_lane(1)
    a.last_used, b.last_used = 1.0, 5.0  # class 0's lane is the older, but class 0 has work waiting
    assert eng.add_lane(2, wanted={0}) is not None
    assert eng.by_class[0] == [a.lid] and eng.by_class[1] == []


def test_busy_lanes_are_never_evicted(fake):
    pats = [_Pat(100, 600) for _ in range(3)]
    eng = fake(pats, budget=2 * 100 * BYTES_PER_ROW, class_size=1, lanes_per_class=1)
    a, b = eng.add_lane(0), eng.add_lane(1)
    a.running = b.running = [object()]
    assert eng.add_lane(2) is None and eng.evictions == 0
    assert not a.solvers[0].closed and not b.solvers[0].closed


def test_ready_requests_of_a_class_share_one_launch(fake):
    """Four requests of four patterns of one class, all waiting: one launch
    takes all four; a fifth request of a pattern already taken waits for the
    next idle lane (the second lane of the class)."""
    pats = [_Pat(50 + k, 300) for k in range(4)]
    eng = fake(pats, budget=1 << 30, class_size=4, lanes_per_class=2)
    eng.warm()
    assert len(eng.lanes) == 2
    stats = eng.run(_requests([0, 1, 2, 3, 2]))
    assert stats.completed == 5
    assert _FakeBatch.launches == [4, 1] and stats.launches == 2 and stats.summary()["mean_batch"] == 2.5


def test_lanes_per_class_are_capped_and_excess_requests_wait(fake):
    pats = [_Pat(10, 60)]
    eng = fake(pats, budget=1 << 30, class_size=1, lanes_per_class=2)
    _FakeBatch.polls = 4
    stats = eng.run(_requests([0] * 7))
    assert stats.completed == 7 and len(eng.by_class[0]) == 2 and stats.lanes_created == 2
    assert stats.max_in_flight == 2 and stats.deferred > 0 and _FakeBatch.launches == [1] * 7


def test_a_class_that_cannot_fit_alone_fails_with_oom(fake):
    pats = [_Pat(10, 60), _Pat(10_000, 60_000)]
    eng = fake(pats, budget=1_000_000, class_size=1)
    _FakeBatch.polls = 1
    reqs = _requests([0, 1, 0])
    stats = eng.run(reqs)
    assert stats.completed == 2 and stats.failed == 1 and reqs[1].status == opm.OPM_ERR_OOM
    for r in (reqs[0], reqs[2]):
        assert r.status == opm.OPM_OK and r.t_arrival <= r.t_start <= r.t_done


def test_warm_gives_every_class_a_lane_before_any_gets_a_second(fake):
    pats = [_Pat(100, 600) for _ in range(4)]
    eng = fake(pats, budget=5 * 100 * BYTES_PER_ROW, class_size=1, lanes_per_class=2)
    eng.warm()
    assert sorted(len(v) for v in eng.by_class.values()) == [1, 1, 1, 2]
    assert eng.hbm_bytes == 5 * 100 * BYTES_PER_ROW and len(_FakeAnalysis.made) == 4
    eng.close()
    assert _FakeSolver.alive == [] and eng.hbm_bytes == 0 and all(a.closed for a in _FakeAnalysis.made)


def test_size_classes_group_patterns_by_cells(fake):
    pats = [_Pat(n, 6 * n) for n in (500, 10, 300, 40, 20, 900)]
    eng = fake(pats, budget=1 << 30, class_size=2)
    assert eng.classes == [[1, 4], [3, 2], [0, 5]]


def test_poisson_arrivals_are_seeded_sorted_and_at_the_rate():
    t = serve.poisson_arrivals(200.0, 50.0, seed=3)
    assert np.array_equal(t, serve.poisson_arrivals(200.0, 50.0, seed=3))
    assert not np.array_equal(t, serve.poisson_arrivals(200.0, 50.0, seed=4))
    assert np.all(np.diff(t) > 0) and t[-1] < 50.0
    # 10,000 expected arrivals: the count's standard deviation is 100
    assert abs(len(t) - 10_000) < 500
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200) < 0.05 / 200 and abs(gaps.std() / gaps.mean() - 1) < 0.05
