"""Continuous-batching serving loop for Newton-step linear solves.

Each request carries new matrix values for one of the resident sparsity
patterns and a right-hand side; it needs an ILU0 refactorisation and a
BiCGStab solve (the per-Newton-step pair of the paper, Sections 4.2 and 4.4:
the pattern, hence the symbolic analysis, never changes, only the values).

The engine keeps, per pattern, one or more *instances*: library handles whose
symbolic analysis, device matrix, factors and Krylov vectors stay resident in
HBM.  Requests that arrive while others are on the GPU are admitted as soon as
an instance of their pattern is idle, or a new instance fits in the HBM
budget; every instance runs on its own CUDA stream, so the work of all
admitted requests overlaps on the device.  A request's latency is measured
from its arrival to the host seeing its completion (queueing included).

The scheduling here is host-side bookkeeping only; all numerical work runs in
the library's kernels through ``opm_solve_launch`` / ``opm_solve_wait``.
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
    instance: int = -1
    x: object = None          # copy of the solution (with keep_results)


@dataclass
class Instance:
    iid: int
    pattern: int
    solver: opm.Solver
    stream: object
    x: object                 # device output buffer
    device_bytes: int
    busy: Request | None = None
    served: int = 0
    last_used: float = 0.0


@dataclass
class ServeStats:
    completed: int = 0
    failed: int = 0
    latencies_ms: list = field(default_factory=list)
    wall_s: float = 0.0
    instances: int = 0
    instances_per_pattern_max: int = 0
    hbm_bytes_peak: int = 0
    max_in_flight: int = 0
    deferred_admissions: int = 0
    evictions: int = 0

    def summary(self):
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.array([np.nan])
        return {"requests": self.completed + self.failed, "completed": self.completed, "failed": self.failed,
                "solves_per_s": self.completed / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(np.mean(lat)), "max_ms": float(np.max(lat)),
                "instances": self.instances, "max_in_flight": self.max_in_flight,
                "hbm_bytes_peak": self.hbm_bytes_peak, "deferred_admissions": self.deferred_admissions,
                "evictions": self.evictions}


class ServingEngine:
    """Admission by free HBM, resident factors per pattern, overlap by streams."""

    def __init__(self, patterns, precision="fp32", schedule="auto", hbm_budget_bytes=8 << 30,
                 max_instances_per_pattern=4, maxit=200):
        import torch
        self.torch = torch
        self.patterns = patterns
        self.precision = precision
        self.schedule = schedule
        self.budget = int(hbm_budget_bytes)
        self.max_per_pattern = max_instances_per_pattern
        self.maxit = maxit
        self.instances: dict[int, Instance] = {}
        self.by_pattern = collections.defaultdict(list)
        self.hbm_bytes = 0
        self._dev = {}
        self._next_iid = 0
        self._bytes_seen = {}
        self.evictions = 0

    def _device_pattern(self, p):
        if p not in self._dev:
            s = self.patterns[p]
            t = self.torch
            self._dev[p] = (t.from_numpy(np.ascontiguousarray(s.rowptr)).cuda(),
                            t.from_numpy(np.ascontiguousarray(s.colidx)).cuda(),
                            t.from_numpy(np.ascontiguousarray(s.vals)).cuda())
        return self._dev[p]

    def estimate_bytes(self, p):
        """Device bytes of one instance of pattern p (measured once created)."""
        if p in self._bytes_seen:
            return self._bytes_seen[p]
        s = self.patterns[p]
        per_val = 4 if self.precision == "fp32" else 8
        # conservative: values, factors, index and slot arrays, 14 vectors, work lists
        return int(s.nnzb * (72 + 9 * per_val + 48) + s.nb * (24 * 14 + 96) + (1 << 20))

    def fits_alone(self, p):
        return self.estimate_bytes(p) <= self.budget

    def _evict_one(self, keep_pattern):
        """Destroy the least recently used idle instance (not the only
        instance of keep_pattern); True if one was freed."""
        idle = [i for i in self.instances.values() if i.busy is None]
        idle.sort(key=lambda i: i.last_used)
        for inst in idle:
            if inst.pattern == keep_pattern and len(self.by_pattern[keep_pattern]) <= 1:
                continue
            inst.solver.close()
            self.by_pattern[inst.pattern].remove(inst.iid)
            del self.instances[inst.iid]
            self.hbm_bytes -= inst.device_bytes
            self.evictions += 1
            return True
        return False

    def add_instance(self, p):
        """Create a resident instance of pattern p if it fits in the budget,
        evicting idle instances of other patterns when needed."""
        if len(self.by_pattern[p]) >= self.max_per_pattern or not self.fits_alone(p):
            return None
        while self.hbm_bytes + self.estimate_bytes(p) > self.budget:
            if not self._evict_one(p):
                return None
        rp, ci, va = self._device_pattern(p)
        stream = self.torch.cuda.Stream()
        sv = opm.Solver(self.patterns[p].nb, rp, ci, va, schedule=self.schedule, precision=self.precision,
                        stream=stream)
        info = sv.info()
        inst = Instance(self._next_iid, p, sv, stream,
                        self.torch.empty(3 * self.patterns[p].nb, dtype=self.torch.float64, device="cuda"),
                        int(info.device_bytes))
        self._next_iid += 1
        self._bytes_seen[p] = inst.device_bytes
        self.instances[inst.iid] = inst
        self.by_pattern[p].append(inst.iid)
        self.hbm_bytes += inst.device_bytes
        return inst

    def warm(self):
        """One resident instance per pattern while the budget allows (the
        symbolic analysis happens here, outside the measured run)."""
        for p in range(len(self.patterns)):
            if not self.by_pattern[p] and self.hbm_bytes + self.estimate_bytes(p) <= self.budget:
                self.add_instance(p)
        self.torch.cuda.synchronize()

    def _idle_instance(self, p):
        for iid in self.by_pattern[p]:
            if self.instances[iid].busy is None:
                return self.instances[iid]
        return self.add_instance(p)

    def run(self, requests, poll_sleep_s=0.0, keep_results=False):
        """Serve requests (sorted by arrival time); returns ServeStats.  A
        request whose pattern cannot fit in the budget even alone fails with
        OPM_ERR_OOM."""
        stats = ServeStats()
        queue = collections.deque()
        in_flight = []
        nxt = 0
        total = len(requests)
        t0 = time.perf_counter()
        done = 0
        while done < total:
            now = time.perf_counter() - t0
            while nxt < total and requests[nxt].t_arrival <= now:
                queue.append(requests[nxt])
                nxt += 1
            # admit every queued request whose pattern has an idle (or new) instance
            waiting = collections.deque()
            while queue:
                r = queue.popleft()
                if not self.fits_alone(r.pattern):
                    r.status = opm.OPM_ERR_OOM
                    r.t_done = time.perf_counter() - t0
                    stats.failed += 1
                    done += 1
                    continue
                inst = self._idle_instance(r.pattern)
                if inst is None:
                    waiting.append(r)
                    stats.deferred_admissions += 1
                    continue
                r.t_start = time.perf_counter() - t0
                r.instance = inst.iid
                inst.busy = r
                inst.solver.launch(r.vals, r.b, inst.x, rtol=r.rtol, maxit=self.maxit)
                in_flight.append(inst)
            queue = waiting
            stats.max_in_flight = max(stats.max_in_flight, len(in_flight))
            stats.hbm_bytes_peak = max(stats.hbm_bytes_peak, self.hbm_bytes)
            # retire finished work
            still = []
            for inst in in_flight:
                if inst.solver.ready():
                    st, it, rr = inst.solver.wait()
                    r = inst.busy
                    r.t_done = time.perf_counter() - t0
                    r.status, r.iters, r.relres = st, it, rr
                    if keep_results:
                        r.x = inst.x.clone()
                    inst.busy = None
                    inst.served += 1
                    inst.last_used = r.t_done
                    done += 1
                    if st in (opm.OPM_OK, opm.OPM_NOT_CONVERGED):
                        stats.completed += 1
                        stats.latencies_ms.append(1e3 * (r.t_done - r.t_arrival))
                    else:
                        stats.failed += 1
                else:
                    still.append(inst)
            in_flight = still
            if poll_sleep_s:
                time.sleep(poll_sleep_s)
        stats.wall_s = time.perf_counter() - t0
        stats.instances = len(self.instances)
        stats.evictions = self.evictions
        stats.instances_per_pattern_max = max(len(v) for v in self.by_pattern.values()) if self.by_pattern else 0
        return stats

    def close(self):
        for inst in self.instances.values():
            inst.solver.close()
        self.instances.clear()
        self.by_pattern.clear()
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
