"""Standard wells kept separate (Section 4.6) through the C ABI against the
oracle: the system operator is A - sum C^T inv(D) B, the preconditioner the
ILU0 of A.  Tolerances as in the plain parity tests (SpMV 1e-12 of
|A'| |x| entrywise, where |A'| includes the wells' terms; FP64 solves 1e-8 on
x).  FP32-factor solves are compared at rtol 1e-10, where both sides are
within the system's conditioning times 1e-10 of its solution, at 1e-7 on x
(at loose rtol two FP32 runs follow different Krylov paths, each only
bounded by its residual)."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11488_gb300 import opm, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def abs_wells(w):
    return synth.Wells(w.ptr, w.cells, np.abs(w.B), np.abs(w.C), np.abs(w.D), -np.abs(w.Dinv))


@pytest.mark.parametrize("maker,nw,layers", [(synth.config1, 3, 4), (synth.config2, 6, 12)])
@pytest.mark.parametrize("schedule", ["colour", "colour_sl", "colour_kempe", "level"])
def test_spmv_with_wells(maker, nw, layers, schedule):
    s = maker()
    w = synth.wells(s, nw, layers)
    x = synth.uniform(synth.stream_key(5, 6), np.arange(3 * s.nb, dtype=np.uint64), -1, 1)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule=schedule) as sv:
        assert sv.set_wells(w) == opm.OPM_OK
        y = sv.spmv(x)
        yd = sv.spmv(dev(x)).cpu().numpy()
    ref = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, x)
    # |A'| |x| bound: |A| |x| plus the wells' terms with absolute values
    bound = O.spmv(s.nb, s.rowptr, s.colidx, np.abs(s.vals), np.abs(x))
    bound = O.apply_wells(abs_wells(w), np.abs(x), bound)
    assert np.all(np.abs(y - ref) <= 1e-12 * bound + 1e-300)
    np.testing.assert_array_equal(y, yd)


def check_solve_wells(s, w, schedule, rtol, precision="fp64", maxit=300):
    b = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, s.x_true)
    x_ref, res, perm, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, rtol, maxit, schedule,
                                         f32=(precision == "fp32"), wells=w)
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=schedule, precision=precision) as sv:
        assert sv.set_wells(w) == opm.OPM_OK
        xd, st, it, relres = sv.solve(dev(b), rtol=rtol, maxit=maxit)
        x = xd.cpu().numpy()
    assert st == res.status == 0
    if precision == "fp32":
        # different FP32 rounding paths: converged to the same solution.  At
        # tight tolerance the count follows the single-precision rounding
        # (a changed reduction order once moved it by 8 of 44), so parity
        # here is the residual and x bound; the count stays within 1/8
        assert abs(it - res.iters) <= max(2, res.iters // 8)
        assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    elif it != res.iters:
        assert abs(it - res.iters) == 1
        h = res.res_hist / res.res_hist[0]
        k = min(it, res.iters)
        assert any(abs(v / rtol - 1) < 1e-6 for v in (h[2 * k - 1], h[2 * k]) if np.isfinite(v))
    else:
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert relres <= rtol * (1 + 1e-6)
    if precision == "fp64":  # same path: the reported true residuals agree
        assert abs(relres - res.relres) <= 1e-6 * max(res.relres, 1e-300) + 1e-14
    return x


@pytest.mark.parametrize("schedule", ["colour", "colour_sl", "colour_kempe", "level"])
def test_solve_with_wells_small(schedule):
    s = synth.config1()
    check_solve_wells(s, synth.wells(s, 3, 4), schedule, 1e-8)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-6), ("fp32", 1e-10)])
def test_solve_with_wells_config2(precision, rtol):
    s = synth.config2()
    check_solve_wells(s, synth.wells(s, 6, 12), "colour_sl", rtol, precision)


def test_solve_with_wells_config3_full_size():
    s = synth.config3()
    check_solve_wells(s, synth.wells(s, 5, 20), "colour_sl", 1e-3)


def test_removing_wells_restores_the_plain_operator():
    s = synth.config2()
    b = dev(O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true))
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl") as a, \
            opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl") as bw:
        assert bw.set_wells(synth.wells(s, 6, 12)) == opm.OPM_OK
        assert bw.set_wells(None) == opm.OPM_OK
        xa, sa, ia, ra = a.solve(b, rtol=1e-6)
        xb, sb, ib, rb = bw.solve(b, rtol=1e-6)
    assert (sa, ia, ra) == (sb, ib, rb)
    np.testing.assert_array_equal(xa.cpu().numpy(), xb.cpu().numpy())


def test_new_well_values_after_a_newton_step():
    """Values re-set (same perforations): the operator follows the new ones."""
    s = synth.config2()
    w0 = synth.wells(s, 6, 12)
    w1 = synth.Wells(w0.ptr, w0.cells, 1.1 * w0.B, 0.9 * w0.C, w0.D, w0.Dinv)
    x = synth.uniform(synth.stream_key(5, 7), np.arange(3 * s.nb, dtype=np.uint64), -1, 1)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="colour_sl") as sv:
        assert sv.set_wells(w0) == opm.OPM_OK
        sv.spmv(x)
        assert sv.set_wells(w1) == opm.OPM_OK
        y = sv.spmv(x)
    ref = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w1, x)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_batch_with_wells_is_bitwise_identical_to_alone():
    syss = synth.config4(nsys=4)
    ws = [synth.wells(s, 2, 5) for s in syss]
    hs = [opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl") for s in syss]
    for h, w in zip(hs, ws):
        assert h.set_wells(w) == opm.OPM_OK
    bs = [dev(O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, s.x_true)) for s, w in zip(syss, ws)]
    alone = [h.solve(b, rtol=1e-8) for h, b in zip(hs, bs)]
    xs = [torch.empty_like(b) for b in bs]
    with opm.Batch([h.h for h in hs]) as bt:
        s_all, st, it, rr = bt.solve(bs, xs, rtol=1e-8)
    assert s_all == opm.OPM_OK
    for k, (xa, sa, ia, ra) in enumerate(alone):
        assert (st[k], it[k], rr[k]) == (sa, ia, ra)
        np.testing.assert_array_equal(xs[k].cpu().numpy(), xa.cpu().numpy())
    for h in hs:
        h.close()


def test_set_wells_rejects_bad_input():
    s = synth.config1()
    w = synth.wells(s, 3, 4)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals) as sv:
        bad = synth.Wells(w.ptr, w.cells.copy(), w.B, w.C, w.D, w.Dinv)
        bad.cells[0] = s.nb
        assert sv.set_wells(bad) == opm.OPM_ERR_ARG
        bad2 = synth.Wells(w.ptr[::-1].copy(), w.cells, w.B, w.C, w.D, w.Dinv)
        assert sv.set_wells(bad2) == opm.OPM_ERR_ARG
        assert sv.set_wells(w) == opm.OPM_OK
