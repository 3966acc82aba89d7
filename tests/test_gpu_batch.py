"""Batched and asynchronous solves: every system's result inside a batch (or
through the asynchronous launch) must be bitwise identical to the same
system solved alone, and must still match the FP64 oracle."""
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


def systems():
    out = [synth.config1(), synth.random_pattern_system(777, 3, 5), synth.chain_system(45),
           synth.block_diagonal_system(70, 2),
           synth.one_way_system(synth.random_pattern_system(300, 4, 48), 0.5, 49)]  # non-symmetric pattern
    out += synth.config4(nsys=6)  # uneven grid sizes of the batched workload
    return out


def make(s, precision, schedule="colour"):
    return opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=schedule, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("sweep", ["per_phase", "cooperative"])
def test_batch_is_bitwise_identical_to_alone(precision, sweep):
    syss = systems()
    bs = [dev(rhs(s)) for s in syss]
    rtols = [1e-8 if k % 2 == 0 else 1e-3 for k in range(len(syss))]
    alone = []
    for s, b, rt in zip(syss, bs, rtols):
        with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour", precision=precision,
                        sweep_launch=sweep) as sv:
            x, st, it, rr = sv.solve(b, rtol=rt)
            alone.append((x.cpu().numpy(), st, it, rr))
    handles = [opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour",
                          precision=precision, sweep_launch=sweep) for s in syss]
    xs = [torch.empty_like(b) for b in bs]
    with opm.Batch([h.h for h in handles], sweep_launch=sweep) as bt:
        s_all, st, it, rr = bt.solve(bs, xs, rtol=rtols)
        assert s_all == opm.OPM_OK
        for k in range(len(syss)):
            xa, sta, ita, rra = alone[k]
            assert st[k] == sta == 0 and it[k] == ita and rr[k] == rra
            np.testing.assert_array_equal(xs[k].cpu().numpy(), xa)
        # refactor inside the batch with new values: still identical to alone
        new_vals = [synth.newton_update(s, 3)[0] for s in syss]
        f, fst = bt.factor([dev(v) for v in new_vals])
        assert f == opm.OPM_OK and all(v == 0 for v in fst)
        s2, st2, it2, rr2 = bt.solve(bs, xs, rtol=1e-2)
    for h in handles:
        h.close()
    for k, (s, v) in enumerate(zip(syss, new_vals)):
        with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(v), schedule="colour", precision=precision,
                        sweep_launch=sweep) as sv:
            x, st, it, rr = sv.solve(bs[k], rtol=1e-2)
            assert st == st2[k] and it == it2[k] and rr == rr2[k]
            np.testing.assert_array_equal(x.cpu().numpy(), xs[k].cpu().numpy())


def test_batch_matches_oracle_and_masks_converged_systems():
    syss = systems()
    bs = [rhs(s) for s in syss]
    handles = [make(s, "fp64") for s in syss]
    xs = [np.empty(3 * s.nb) for s in syss]  # host buffers on purpose
    rtols = [10.0 ** -(2 + (k % 6)) for k in range(len(syss))]  # uneven iteration counts
    with opm.Batch([h.h for h in handles]) as bt:
        s_all, st, it, rr = bt.solve(bs, xs, rtol=rtols)
    for h in handles:
        h.close()
    assert s_all == 0 and len(set(it)) > 1
    for k, s in enumerate(syss):
        x_ref, res, _, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, bs[k], rtols[k], 200, "colour")
        assert st[k] == 0 and it[k] == res.iters
        assert np.linalg.norm(xs[k] - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_batch_reports_a_singular_pivot_per_system():
    syss = [synth.config1(), synth.config1(seed=synth.config_seed(1, 5)), synth.chain_system(60)]
    handles = [make(s, "fp64") for s in syss]
    bad = syss[1].vals.copy()
    rows = np.repeat(np.arange(syss[1].nb), np.diff(syss[1].rowptr))
    d = np.flatnonzero(rows == syss[1].colidx)
    bad[d[0]] = 0.0  # row 0 is in colour 0: its pivot is the zeroed block
    with opm.Batch([h.h for h in handles]) as bt:
        f, fst = bt.factor([dev(syss[0].vals), dev(bad), dev(syss[2].vals)])
        assert f == opm.OPM_ERR_ZERO_PIVOT and fst == [0, opm.OPM_ERR_ZERO_PIVOT, 0]
    assert opm.opm_last_error_row(handles[1].h) == 0
    for h in handles:
        h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_async_launch_matches_synchronous(precision):
    s = synth.config2()
    b = dev(rhs(s))
    vals2 = dev(synth.newton_update(s, 7)[0])
    with make(s, precision) as sv:
        sv.factor(vals2)
        x_sync, st_s, it_s, rr_s = sv.solve(b, rtol=1e-2)
    stream = torch.cuda.Stream()
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour", precision=precision,
                    stream=stream) as sv:
        x = torch.empty_like(b)
        sv.launch(vals2, b, x, rtol=1e-2)
        st, it, rr = sv.wait()
        assert (st, it, rr) == (st_s, it_s, rr_s)
        np.testing.assert_array_equal(x.cpu().numpy(), x_sync.cpu().numpy())
        assert sv.ready()


@pytest.mark.parametrize("pinned", [True, False])
def test_async_launch_with_host_buffers(pinned):
    """Host values, b and x (page-locked or pageable) are copied on the
    handle's stream; results equal the device-buffer launch bit for bit."""
    s = synth.config2()
    b = rhs(s)
    vals2 = synth.newton_update(s, 7)[0]
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="colour") as sv:
        xd = torch.empty(3 * s.nb, dtype=torch.float64, device="cuda")
        sv.launch(dev(vals2), dev(b), xd, rtol=1e-2)
        ref = sv.wait()
        vh, bh = torch.from_numpy(vals2.copy()), torch.from_numpy(b.copy())
        xh = torch.zeros(3 * s.nb, dtype=torch.float64)
        if pinned:
            vh, bh, xh = vh.pin_memory(), bh.pin_memory(), xh.pin_memory()
        sv.launch(vh, bh, xh, rtol=1e-2)
        got = sv.wait()
    assert got == ref
    np.testing.assert_array_equal(xh.numpy(), xd.cpu().numpy())


def test_batch_async_launch():
    syss = synth.config4(nsys=5)
    bs = [dev(rhs(s)) for s in syss]
    handles = [make(s, "fp32") for s in syss]
    xs = [torch.empty_like(b) for b in bs]
    xs2 = [torch.empty_like(b) for b in bs]
    with opm.Batch([h.h for h in handles]) as bt:
        s1, st1, it1, rr1 = bt.solve(bs, xs, rtol=1e-2)
        assert bt.launch([dev(s.vals) for s in syss], bs, xs2, rtol=1e-2) == 0
        s2, st2, it2, rr2 = bt.wait()
    for h in handles:
        h.close()
    assert (s1, st1, it1, rr1) == (s2, st2, it2, rr2)
    for a, c in zip(xs, xs2):
        np.testing.assert_array_equal(a.cpu().numpy(), c.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("part", [False, True])
def test_handle_from_kept_analysis_equals_a_created_one(precision, part):
    """A handle made from a kept analysis (opm_bsr_create_from_analysis) has
    the created handle's order, factors and solves, bitwise, also after the
    analysis object is gone and after a refactorisation with new values."""
    s = synth.config2() if not part else synth.config1()
    pt = synth.partition_grid(s, 6) if part else None
    b = dev(rhs(s))
    an = opm.Analysis(s.nb, dev(s.rowptr), dev(s.colidx), "colour_kempe", part=pt)
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_kempe", precision=precision,
                    part=pt) as ref:
        h = opm.Solver.from_analysis(an, dev(s.vals), precision=precision)
        an.close()
        with h:
            assert h.status == ref.status == opm.OPM_OK
            np.testing.assert_array_equal(h.permutation(), ref.permutation())
            assert h.info().nupdates == ref.info().nupdates > 0
            for k in range(2):
                if k == 1:
                    v = dev(synth.newton_update(s, 5)[0])
                    assert h.factor(v) == ref.factor(v) == opm.OPM_OK
                la, da = h.factors()
                lb, db = ref.factors()
                np.testing.assert_array_equal(la, lb)
                np.testing.assert_array_equal(da, db)
                # the Newton-updated values need more than 200 iterations at 1e-6
                xa, sta, ita, rra = h.solve(b, rtol=1e-6)
                xb, stb, itb, rrb = ref.solve(b, rtol=1e-6)
                assert (sta, ita, rra) == (stb, itb, rrb) and sta in (opm.OPM_OK, opm.OPM_NOT_CONVERGED)
                np.testing.assert_array_equal(xa.cpu().numpy(), xb.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_members_can_sit_a_launch_out(precision):
    """opm_batch_launch with b[i] = x[i] = NULL: the member's x, values,
    factors and state are untouched (its later solve alone equals a fresh
    handle's), the others' results are bitwise those of their solves alone,
    with and without a refactorisation in the launch."""
    syss = systems()[:6]
    bs = [dev(rhs(s)) for s in syss]
    new_vals = [dev(synth.newton_update(s, 9)[0]) for s in syss]
    handles = [make(s, precision) for s in syss]
    active = [k % 2 == 0 for k in range(len(syss))]
    xs = [torch.full_like(b, np.nan) for b in bs]
    with opm.Batch([h.h for h in handles]) as bt:
        for refactor in (False, True):
            vals = [v if a else None for v, a in zip(new_vals, active)] if refactor else None
            assert bt.launch(vals, [b if a else None for b, a in zip(bs, active)],
                             [x if a else None for x, a in zip(xs, active)], rtol=1e-8) == opm.OPM_OK
            s_all, st, it, rr = bt.wait()
            assert s_all == opm.OPM_OK
            for k, s in enumerate(syss):
                if not active[k]:
                    assert (st[k], it[k], rr[k]) == (opm.OPM_OK, 0, 0.0)
                    assert torch.isnan(xs[k]).all()
                    continue
                vk = new_vals[k] if refactor else dev(s.vals)
                with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), vk, schedule="colour", precision=precision) as sv:
                    xa, sta, ita, rra = sv.solve(bs[k], rtol=1e-8)
                assert (st[k], it[k], rr[k]) == (sta, ita, rra)
                np.testing.assert_array_equal(xs[k].cpu().numpy(), xa.cpu().numpy())
    # the members that sat out still hold their original factors
    for k, s in enumerate(syss):
        if active[k]:
            continue
        xa, sta, ita, rra = handles[k].solve(bs[k], rtol=1e-8)
        with make(s, precision) as fresh:
            xb, stb, itb, rrb = fresh.solve(bs[k], rtol=1e-8)
        assert (sta, ita, rra) == (stb, itb, rrb)
        np.testing.assert_array_equal(xa.cpu().numpy(), xb.cpu().numpy())
    for h in handles:
        h.close()


def test_handles_made_and_freed_while_another_solves():
    """Device memory comes from a stream-ordered pool: handles made and
    destroyed on other streams while a solve runs (the serving loop's
    eviction) leave that solve's result bitwise unchanged, and a handle made
    in memory another one freed solves like a fresh one."""
    s = synth.config2()
    b = dev(rhs(s))
    with make(s, "fp64") as ref:
        x_ref, st, it, rr = ref.solve(b, rtol=1e-6)
        x_ref = x_ref.cpu().numpy()
    main_stream = torch.cuda.Stream()
    side = torch.cuda.Stream()
    small = synth.config1()
    an = opm.Analysis(small.nb, small.rowptr, small.colidx, "auto")
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour", stream=main_stream) as sv:
        x = torch.empty_like(b)
        vals = dev(s.vals)
        for rep in range(3):
            sv.launch(vals, b, x, rtol=1e-6, maxit=200)
            for _ in range(4):  # churn on another stream while the solve runs
                h = opm.Solver.from_analysis(an, dev(small.vals), precision="fp32", stream=side)
                h.close()
            st2, it2, rr2 = sv.wait()
            assert (st2, it2) == (st, it)
            np.testing.assert_array_equal(x.cpu().numpy(), x_ref)
    bs = dev(O.spmv(small.nb, small.rowptr, small.colidx, small.vals, small.x_true))
    with opm.Solver.from_analysis(an, dev(small.vals), precision="fp64", stream=side) as h, \
            make(small, "fp64", schedule="colour_kempe") as fresh:
        xa, sta, ita, rra = h.solve(bs, rtol=1e-8)
        xb, stb, itb, rrb = fresh.solve(bs, rtol=1e-8)
        assert (sta, ita, rra) == (stb, itb, rrb)
        np.testing.assert_array_equal(xa.cpu().numpy(), xb.cpu().numpy())
    an.close()
