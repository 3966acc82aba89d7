"""Autotuner: the chosen configuration is one of the candidates it timed,
the fastest among those that converged, and solves like any other
configuration (every candidate's result still matches the oracle)."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11488_gb300 import opm, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rhs(s):
    return O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true)


def check_report(kw, cands, best):
    assert 0 <= best < len(cands)
    ok = [c for c in cands if c["status"] == opm.OPM_OK]
    assert ok and cands[best]["status"] == opm.OPM_OK
    assert cands[best]["ms"] == min(c["ms"] for c in ok)
    for k in ("schedule", "sweep_launch", "chunk", "small_phase_slices"):
        assert kw[k] == cands[best][k]
    # the coordinate search visits both schedules and, for the winner, the other loop-body lengths
    assert {"level", "colour"} <= {c["schedule"] for c in cands}
    w = [c for c in cands if c["schedule"] == kw["schedule"] and c["sweep_launch"] == kw["sweep_launch"]]
    assert {1, 2, 4} <= {c["chunk"] for c in w}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_single_system(precision):
    s = synth.config1()
    b = dev(rhs(s))
    st, kw, cands, best = opm.autotune(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), b, rtol=1e-6,
                                       maxit=200, repeats=2, precision=precision)
    assert st == opm.OPM_OK
    check_report(kw, cands, best)
    assert "natural" in {c["schedule"] for c in cands}  # 500 rows: the natural order is a candidate
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), precision=precision, **kw) as sv:
        x, st2, it, rr = sv.solve(b, rtol=1e-6)
        assert st2 == opm.OPM_OK and rr <= 1e-6 * (1 + 1e-6)
        perm = sv.permutation()
    x_ref, res, perm_ref, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, rhs(s), 1e-6, 200,
                                             kw["schedule"], f32=(precision == "fp32"))
    np.testing.assert_array_equal(perm, perm_ref)
    x = x.cpu().numpy()
    if it == res.iters:
        assert np.linalg.norm(x - x_ref) <= (1e-8 if precision == "fp64" else 1e-6) * np.linalg.norm(x_ref)
    else:
        assert abs(it - res.iters) == 1


def test_autotune_batch():
    syss = synth.config4(nsys=8)
    bs = [dev(rhs(s)) for s in syss]
    st, kw, cands, best = opm.autotune_batch(
        [(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), b) for s, b in zip(syss, bs)],
        rtol=[1e-2] * len(syss), maxit=200, repeats=2, precision="fp32")
    assert st == opm.OPM_OK
    check_report(kw, cands, best)
    handles = [opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=kw["schedule"],
                          precision="fp32") for s in syss]
    bt = opm.Batch([h.h for h in handles], chunk=kw["chunk"], sweep_launch=kw["sweep_launch"],
                   small_phase_slices=kw["small_phase_slices"])
    xs = [torch.empty_like(b) for b in bs]
    s_all, st_k, it_k, rr_k = bt.solve(bs, xs, rtol=[1e-2] * len(syss))
    assert s_all == opm.OPM_OK
    for k, s in enumerate(syss):
        assert st_k[k] == 0 and rr_k[k] <= 1e-2 * (1 + 1e-6)
        # the tuned batch is bitwise identical to each system alone with the same options
        x1, st1, it1, rr1 = handles[k].solve(bs[k], rtol=1e-2)
        assert (st1, it1, rr1) == (st_k[k], it_k[k], rr_k[k])
        np.testing.assert_array_equal(x1.cpu().numpy(), xs[k].cpu().numpy())
    bt.close()
    for h in handles:
        h.close()
