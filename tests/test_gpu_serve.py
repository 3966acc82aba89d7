"""Serving loop: ready requests of a size class go to the GPU in one batched
launch, lanes overlap on the device, and every served result is bitwise
identical to the same request solved alone; lanes are admitted by the HBM
budget, evicted when idle and remade from the kept analyses."""
import numpy as np
import pytest

from paper_2309_11488_gb300 import opm, serve, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def small_patterns():
    dims = [(12, 10, 6), (20, 15, 8), (9, 9, 9), (30, 12, 5)]
    out = []
    for k, (nx, ny, nz) in enumerate(dims):
        seed = synth.config_seed(5, 900 + k)
        logk = synth._lognormal_field(seed, (nz, ny, nx), 1.0)
        out.append(synth.grid_system(nx, ny, nz, logk, seed=seed))
    return out


def make_requests(templates, npat, nreq, rate, seed):
    t = serve.poisson_arrivals(rate, nreq / rate * 3, seed)[:nreq]
    reqs = []
    for i, ti in enumerate(t):
        p = i % npat
        vals, b = templates[p][i % len(templates[p])]
        reqs.append(serve.Request(i, float(ti), p, vals, b))
    return reqs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_served_results_equal_solo_results(precision):
    pats = small_patterns()
    tmpl = serve.request_templates(pats, 2, precision)
    reqs = make_requests(tmpl, len(pats), 48, rate=20000.0, seed=11)
    eng = serve.ServingEngine(pats, precision=precision, hbm_budget_bytes=4 << 30, class_size=2, lanes_per_class=2)
    eng.warm()
    stats = eng.run(reqs, keep_results=True)
    eng.close()
    assert stats.completed == len(reqs) and stats.failed == 0
    s = stats.summary()
    assert stats.max_in_flight >= 2  # work of several requests was on the device at once
    assert s["mean_batch"] > 1.0  # ready requests shared launches
    assert s["p99_ms"] >= s["p50_ms"] > 0
    # every served result equals the same request solved alone
    for r in reqs:
        pat = pats[r.pattern]
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        with opm.Solver(pat.nb, dev(pat.rowptr), dev(pat.colidx), r.vals, precision=precision) as sv:
            x, st, it, rr = sv.solve(r.b, rtol=r.rtol)
        assert (st, it, rr) == (r.status, r.iters, r.relres)
        np.testing.assert_array_equal(x.cpu().numpy(), r.x.cpu().numpy())


def test_admission_respects_budget_and_evicts_idle_lanes():
    pats = small_patterns()
    tmpl = serve.request_templates(pats, 1, "fp32")
    eng = serve.ServingEngine(pats, precision="fp32", hbm_budget_bytes=1 << 40, class_size=1, lanes_per_class=1)
    eng.warm()  # measured instance sizes
    sizes = [eng.estimate_bytes(p) for p in range(len(pats))]
    eng.close()
    # budget for the two largest lanes only: the others must evict to run
    budget = sorted(sizes)[-1] * 2 + 1
    eng = serve.ServingEngine(pats, precision="fp32", hbm_budget_bytes=budget, class_size=1, lanes_per_class=1)
    eng._bytes_seen = dict(enumerate(sizes))
    reqs = make_requests(tmpl, len(pats), 24, rate=5000.0, seed=12)
    stats = eng.run(reqs, keep_results=True)
    assert len(eng.analyses) == len(pats)  # one analysis per pattern, kept across evictions
    eng.close()
    assert stats.completed == len(reqs)
    assert stats.hbm_bytes_peak <= budget
    assert stats.evictions > 0 and stats.lanes_created > 2
    # results of lanes remade from the kept analyses equal solo solves
    for r in reqs[:8]:
        pat = pats[r.pattern]
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        with opm.Solver(pat.nb, dev(pat.rowptr), dev(pat.colidx), r.vals, precision="fp32") as sv:
            x, st, it, rr = sv.solve(r.b, rtol=r.rtol)
        assert (st, it, rr) == (r.status, r.iters, r.relres)
        np.testing.assert_array_equal(x.cpu().numpy(), r.x.cpu().numpy())
    # a pattern that cannot fit even alone is refused, not waited on forever
    eng = serve.ServingEngine(pats, precision="fp32", hbm_budget_bytes=min(sizes) // 2, class_size=1)
    stats = eng.run(make_requests(tmpl, len(pats), 4, rate=1000.0, seed=13))
    eng.close()
    assert stats.failed == 4 and stats.completed == 0
