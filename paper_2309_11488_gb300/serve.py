"""Continuous-batching serving loop for Newton-step linear solves.

Each request carries new matrix values for one of the resident sparsity
patterns and a right-hand side; it needs an ILU0 refactorisation and a
BiCGStab solve (the per-Newton-step pair of the paper, Sections 4.2 and 4.4:
the pattern, hence its symbolic analysis, never changes, only the values).

Residency.  Every pattern's symbolic analysis is computed once
(``opm.Analysis``) and kept in host memory for the whole run.  Device memory
is organised in *lanes*: a lane holds one instance (a library handle: device
matrix, factors, Krylov vectors) of every pattern of one size class, one
batch over those instances and its own CUDA stream.  Lanes are admitted by
free HBM under a budget.  When a size class needs a lane and the budget is
full, the least recently used idle lane of another class is evicted (its
device memory freed) and the new lane is made from the kept analyses: an
upload and a first factorisation, never a new analysis.

Batching.  Requests wait in a FIFO queue per pattern.  Whenever a lane is
idle, the oldest waiting request of each of its patterns is taken and all of
them go to the GPU in one ``opm_batch_launch`` (refactorisation + solve);
the lane's other instances sit the launch out.  Lanes run at once on their
own streams, so a request that arrives while others are on the GPU is
admitted into the next idle lane of its class and its work overlaps theirs
on the device.  A request's latency runs from its arrival to the host seeing
its completion (queueing included).

The scheduling is host-side bookkeeping only; all numerical work runs in the
library's kernels.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import opm


@dataclass
class Request:
    rid: int
    t_arrival: float          # seconds after the start of the run
    pattern: int
    vals: object              # device tensor (nnzb, 9)
    b: object                 # device tensor (3 nb)
    rtol: float = 1e-2
    t_start: float = -1.0
    t_done: float = -1.0
    status: int = 0
    iters: int = 0
    relres: float = float("nan")
    lane: int = -1
    x: object = None          # copy of the solution (with keep_results)


@dataclass
class Lane:
    lid: int
    cls: int                  # size class
    patterns: list            # member patterns, in member order
    solvers: list             # one opm.Solver per member
    batch: object             # opm.Batch over the members
    stream: object
    xs: list                  # device output buffer per member
    device_bytes: int
    running: list | None = None  # requests of the launch in flight (None: a member sits out)
    last_used: float = 0.0
    launches: int = 0


@dataclass
class ServeStats:
    completed: int = 0
    failed: int = 0
    latencies_ms: list = field(default_factory=list)
    wall_s: float = 0.0
    lanes: int = 0
    hbm_bytes_peak: int = 0
    max_in_flight: int = 0     # requests on the device at once
    deferred: int = 0          # requests that found no idle lane on arrival
    evictions: int = 0
    lanes_created: int = 0     # lanes made during the run (from the kept analyses)
    launches: int = 0
    batched_requests: int = 0  # requests over all launches

    def summary(self):
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.array([np.nan])
        return {"requests": self.completed + self.failed, "completed": self.completed, "failed": self.failed,
                "solves_per_s": self.completed / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(np.mean(lat)), "max_ms": float(np.max(lat)),
                "lanes": self.lanes, "max_in_flight": self.max_in_flight,
                "hbm_bytes_peak": self.hbm_bytes_peak, "deferred": self.deferred,
                "evictions": self.evictions, "lanes_created_in_run": self.lanes_created,
                "launches": self.launches,
                "mean_batch": self.batched_requests / self.launches if self.launches else 0.0}


class ServingEngine:
    """Kept analyses, lanes admitted by free HBM, batched launches per lane."""

    def __init__(self, patterns, precision="fp32", schedule="auto", hbm_budget_bytes=8 << 30, class_size=8,
                 lanes_per_class=2, maxit=200):
        import torch
        self.torch = torch
        self.patterns = patterns
        self.precision = precision
        self.schedule = schedule
        self.budget = int(hbm_budget_bytes)
        self.lanes_per_class = lanes_per_class
        self.maxit = maxit
        # size classes: patterns by cell count, class_size per class
        order = sorted(range(len(patterns)), key=lambda p: (patterns[p].nb, p))
        self.classes = [order[i:i + class_size] for i in range(0, len(order), class_size)]
        self.class_of = {p: c for c, members in enumerate(self.classes) for p in members}
        self.analyses = {}
        self.lanes: dict[int, Lane] = {}
        self.by_class = collections.defaultdict(list)
        self.hbm_bytes = 0
        self._next_lid = 0
        self._bytes_seen = {}
        self.evictions = 0
        self.lanes_created = 0

    # ---------------------------------------------------------------- memory

    def estimate_bytes(self, p):
        """Device bytes of one instance of pattern p and its output buffer
        (measured once an instance was created)."""
        if p in self._bytes_seen:
            return self._bytes_seen[p]
        s = self.patterns[p]
        per_val = 4 if self.precision == "fp32" else 8
        # conservative: values, factors, index and slot arrays, 14 vectors, work lists
        return int(s.nnzb * (72 + 9 * per_val + 48) + s.nb * (24 * 15 + 96) + (1 << 20))

    def lane_bytes(self, c):
        return sum(self.estimate_bytes(p) for p in self.classes[c])

    def fits_alone(self, p):
        return self.lane_bytes(self.class_of[p]) <= self.budget

    def analyse(self):
        """The symbolic analysis of every pattern, once, kept for the run."""
        for p, s in enumerate(self.patterns):
            if p not in self.analyses:
                self.analyses[p] = opm.Analysis(s.nb, s.rowptr, s.colidx, self.schedule)

    def _evict_one(self, keep_class, wanted=()):
        """Free the least recently used idle lane of another class, lanes of
        classes in `wanted` (classes with requests waiting) last; True if one
        was freed."""
        idle = [ln for ln in self.lanes.values() if ln.running is None and ln.cls != keep_class]
        idle.sort(key=lambda ln: (ln.cls in wanted, ln.last_used))
        if not idle:
            return False
        ln = idle[0]
        self._close_lane(ln)
        self.evictions += 1
        return True

    def _close_lane(self, ln):
        ln.batch.close()
        for sv in ln.solvers:
            sv.close()
        self.by_class[ln.cls].remove(ln.lid)
        del self.lanes[ln.lid]
        self.hbm_bytes -= ln.device_bytes

    def add_lane(self, c, evict=True, wanted=(), first_vals=None):
        """A new lane of class c if it fits in the budget (evicting idle
        lanes of other classes when allowed), else None.  Its instances come
        from the kept analyses, factorised once with the values of
        first_vals (pattern -> device values, e.g. a waiting request's) or
        the pattern's base values."""
        if len(self.by_class[c]) >= self.lanes_per_class or self.lane_bytes(c) > self.budget:
            return None
        while self.hbm_bytes + self.lane_bytes(c) > self.budget:
            if not evict or not self._evict_one(c, wanted):
                return None
        self.analyse()
        stream = self.torch.cuda.Stream()
        solvers, xs, nbytes = [], [], 0
        for p in self.classes[c]:
            if first_vals and p in first_vals:
                v = first_vals[p]  # already on the device: no upload
            else:
                v = self.torch.from_numpy(np.ascontiguousarray(self.patterns[p].vals)).cuda()
            sv = opm.Solver.from_analysis(self.analyses[p], v, precision=self.precision, stream=stream)
            del v
            solvers.append(sv)
            xs.append(self.torch.empty(3 * self.patterns[p].nb, dtype=self.torch.float64, device="cuda"))
            b = int(sv.info().device_bytes) + 24 * self.patterns[p].nb
            self._bytes_seen[p] = b
            nbytes += b
        batch = opm.Batch([sv.h for sv in solvers], stream=stream)
        ln = Lane(self._next_lid, c, list(self.classes[c]), solvers, batch, stream, xs, nbytes)
        self._next_lid += 1
        self.lanes[ln.lid] = ln
        self.by_class[c].append(ln.lid)
        self.hbm_bytes += nbytes
        return ln

    def warm(self):
        """The analyses, then lanes class by class (a first lane for every
        class before any second one) while they fit the budget; no eviction."""
        self.analyse()
        for _ in range(self.lanes_per_class):
            for c in range(len(self.classes)):
                if self.hbm_bytes + self.lane_bytes(c) <= self.budget:
                    self.add_lane(c, evict=False)
        self.torch.cuda.synchronize()

    # --------------------------------------------------------------- serving

    def _launch(self, ln, queues, t0):
        """Launch lane ln with the oldest waiting request of each of its
        patterns; False if none waits."""
        picked = [queues[p].popleft() if queues[p] else None for p in ln.patterns]
        k = sum(r is not None for r in picked)
        if k == 0:
            return False
        now = time.perf_counter() - t0
        for r in picked:
            if r is not None:
                r.t_start, r.lane = now, ln.lid
        vals = [r.vals if r is not None else None for r in picked]
        bs = [r.b if r is not None else None for r in picked]
        xs = [x if r is not None else None for x, r in zip(ln.xs, picked)]
        rt = [r.rtol if r is not None else 1e-2 for r in picked]
        st = ln.batch.launch(vals, bs, xs, rtol=rt, maxit=self.maxit)
        if st != opm.OPM_OK:
            raise opm.OpmError(st, "opm_batch_launch")
        ln.running = picked
        ln.launches += 1
        return k

    def run(self, requests, poll_sleep_s=0.0, keep_results=False):
        """Serve requests (sorted by arrival time); returns ServeStats.  A
        request whose pattern's class cannot fit in the budget even alone
        fails with OPM_ERR_OOM."""
        stats = ServeStats()
        queues = collections.defaultdict(collections.deque)
        waiting = collections.Counter()  # requests queued per class
        nxt, done, total = 0, 0, len(requests)
        in_flight = 0
        lanes0 = self.lanes_created
        t0 = time.perf_counter()
        while done < total:
            now = time.perf_counter() - t0
            while nxt < total and requests[nxt].t_arrival <= now:
                r = requests[nxt]
                nxt += 1
                if not self.fits_alone(r.pattern):
                    r.status = opm.OPM_ERR_OOM
                    r.t_done = time.perf_counter() - t0
                    stats.failed += 1
                    done += 1
                    continue
                c = self.class_of[r.pattern]
                if not any(self.lanes[i].running is None for i in self.by_class[c]):
                    stats.deferred += 1
                queues[r.pattern].append(r)
                waiting[c] += 1
            # admit, classes in the order of their oldest waiting request:
            # every idle lane of a class with waiting requests takes the
            # oldest request of each of its patterns; a class without an idle
            # lane gets a new one when the budget allows
            def oldest(c):
                return min((queues[p][0].t_arrival, queues[p][0].rid) for p in self.classes[c] if queues[p])
            for c in sorted((c for c, n in waiting.items() if n > 0), key=oldest):
                for lid in list(self.by_class[c]):
                    ln = self.lanes[lid]
                    if ln.running is None and waiting[c] > 0:
                        k = self._launch(ln, queues, t0)
                        waiting[c] -= k
                        in_flight += k
                        stats.launches += k > 0
                        stats.batched_requests += k
                while waiting[c] > 0 and len(self.by_class[c]) < self.lanes_per_class:
                    first = {p: queues[p][0].vals for p in self.classes[c] if queues[p]}
                    ln = self.add_lane(c, wanted={k for k, n in waiting.items() if n > 0}, first_vals=first)
                    if ln is None:
                        break
                    self.lanes_created += 1
                    k = self._launch(ln, queues, t0)
                    waiting[c] -= k
                    in_flight += k
                    stats.launches += k > 0
                    stats.batched_requests += k
            stats.max_in_flight = max(stats.max_in_flight, in_flight)
            stats.hbm_bytes_peak = max(stats.hbm_bytes_peak, self.hbm_bytes)
            # retire finished launches
            for ln in list(self.lanes.values()):
                if ln.running is None or not ln.batch.ready():
                    continue
                _, st, it, rr = ln.batch.wait()
                t_done = time.perf_counter() - t0
                for m, r in enumerate(ln.running):
                    if r is None:
                        continue
                    r.t_done = t_done
                    r.status, r.iters, r.relres = st[m], it[m], rr[m]
                    if keep_results:
                        r.x = ln.xs[m].clone()
                    done += 1
                    in_flight -= 1
                    if st[m] in (opm.OPM_OK, opm.OPM_NOT_CONVERGED):
                        stats.completed += 1
                        stats.latencies_ms.append(1e3 * (r.t_done - r.t_arrival))
                    else:
                        stats.failed += 1
                ln.running = None
                ln.last_used = t_done
            if poll_sleep_s:
                time.sleep(poll_sleep_s)
        stats.wall_s = time.perf_counter() - t0
        stats.lanes = len(self.lanes)
        stats.evictions = self.evictions
        stats.lanes_created = self.lanes_created - lanes0
        return stats

    def close(self):
        for ln in list(self.lanes.values()):
            self._close_lane(ln)
        for an in self.analyses.values():
            an.close()
        self.analyses.clear()
        self.hbm_bytes = 0


def poisson_arrivals(rate_per_s, duration_s, seed):
    """Arrival times of a Poisson process (exponential gaps), seeded."""
    from .synth import stream_key, uniform
    key = stream_key(seed, 77)
    n_max = int(rate_per_s * duration_s * 2 + 100)
    u = uniform(key, np.arange(n_max, dtype=np.uint64))
    gaps = -np.log1p(-u) / rate_per_s
    t = np.cumsum(gaps)
    return t[t < duration_s]


def request_templates(patterns, per_pattern, precision, seed_base=None):
    """Newton-step value updates of every pattern (Section 5 workloads'
    serving form): per template new block values (each block scaled by one
    U(0.9, 1.1) factor) and b = A' x_true, computed on the GPU with the
    library's own SpMV.  Returns {pattern: [(vals, b), ...]} of device tensors."""
    import torch
    from . import synth
    out = {}
    for p, s in enumerate(patterns):
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        rp, ci = dev(s.rowptr), dev(s.colidx)
        lst = []
        gen = None
        for k in range(per_pattern):
            vals, xt = synth.newton_update(s, 1000 * p + k, seed=seed_base)
            vd = dev(vals)
            if gen is None:
                gen = opm.Solver(s.nb, rp, ci, vd, schedule="auto", precision=precision)
            else:
                gen.factor(vd)
            b = gen.spmv(dev(xt))
            lst.append((vd, b))
        gen.close()
        out[p] = lst
    return out
