"""Block-Jacobi ILU0 (Section 4.5) through the C ABI against the oracle: the
preconditioner keeps only the partition-internal blocks; schedule,
permutation and factors follow that pattern, the SpMV the whole matrix.
Tolerances as in the plain parity tests (factors 1e-12, FP64 solves 1e-8 on
x).  FP32-factor solves are compared at rtol 1e-10 at 1e-7 on x: both sides
factorise and sweep in FP32 but round in different orders (FMA, sums), so
at loose rtol their Krylov paths part; at a tight rtol both are pinned to
the system's solution."""
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


def ref_jacobi(s, part, schedule, f32=False):
    jrp, jci, jv, _ = O.jacobi_pattern(s.nb, s.rowptr, s.colidx, s.vals, part)
    perm, nsets = O.schedule_perm(s.nb, jrp, jci, schedule)
    prow, pcol, _ = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    mprow, mpcol, mpval = O.permute(s.nb, jrp, jci, jv, perm)
    fac = O.ilu0(s.nb, mprow, mpcol, mpval, f32=f32)
    return perm, nsets, prow, pcol, mprow, mpcol, fac


CASES = {
    "c1_4parts": (synth.config1, lambda s: synth.partition_grid(s, 4)),
    "ragged_mod3": (lambda: synth.random_pattern_system(70, 4, 45), lambda s: (np.arange(s.nb) % 3).astype(np.int32)),
    "chain_cut": (lambda: synth.chain_system(100), lambda s: (np.arange(s.nb) >= 37).astype(np.int32)),
    "c1_rowwise": (synth.config1, lambda s: np.arange(s.nb, dtype=np.int32)),
}


def case(name):
    make, split = CASES[name]
    s = make()
    return s, split(s)


@pytest.mark.parametrize("sweep", ["per_phase", "cooperative"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("schedule", ["level", "colour", "colour_sl", "colour_kempe"])
def test_jacobi_permutation_and_factors(name, schedule, sweep):
    s, part = case(name)
    perm, nsets, prow, pcol, mprow, mpcol, fac = ref_jacobi(s, part, schedule)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule=schedule, sweep_launch=sweep, part=part) as sv:
        np.testing.assert_array_equal(sv.permutation(), perm)
        info = sv.info()
        assert info.nsets == nsets and info.nphases == nsets
        assert info.nnzb == s.nnzb and info.nnzb_lower + info.nnzb_upper + s.nb == mprow[-1]
        lu, dinv = sv.factors()
    # the kept blocks, in the full permuted pattern's order, are the Jacobi pattern's blocks
    rows = np.repeat(np.arange(s.nb), np.diff(prow))
    kept = part[perm[rows]] == part[perm[pcol]]
    assert np.array_equal(pcol[kept], mpcol)
    assert np.all(lu[~kept] == 0.0)
    mrows = np.repeat(np.arange(s.nb), np.diff(mprow))
    off = mrows != mpcol
    ref = fac.lu
    err = np.abs(lu[kept] - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-300)
    assert err[off].max(initial=0.0) <= 1e-12
    derr = np.abs(dinv - fac.dinv).max(axis=1) / np.maximum(np.abs(fac.dinv).max(axis=1), 1e-300)
    assert derr.max() <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("schedule", ["level", "colour_sl"])
def test_jacobi_ilu_apply(name, schedule):
    s, part = case(name)
    perm, nsets, prow, pcol, mprow, mpcol, fac = ref_jacobi(s, part, schedule)
    r = synth.uniform(synth.stream_key(9, 9), np.arange(3 * s.nb, dtype=np.uint64), -1, 1)
    zp = O.ilu_apply(s.nb, mprow, mpcol, fac, r.reshape(-1, 3)[perm].ravel())
    z_ref = np.empty_like(zp)
    z_ref.reshape(-1, 3)[perm] = zp.reshape(-1, 3)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule=schedule, part=part) as sv:
        z = sv.ilu_apply(r)
    np.testing.assert_allclose(z, z_ref, rtol=1e-11, atol=1e-12 * np.abs(z_ref).max())


def check_jacobi_solve(s, part, schedule, rtol, precision="fp64", maxit=200):
    b = rhs(s)
    x_ref, res, perm, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, rtol, maxit, schedule,
                                         f32=(precision == "fp32"), part=part)
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=schedule, precision=precision,
                    part=dev(part)) as sv:
        np.testing.assert_array_equal(sv.permutation(), perm)
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
    return it, res.iters


@pytest.mark.parametrize("name", ["c1_4parts", "ragged_mod3", "chain_cut"])
@pytest.mark.parametrize("schedule", ["level", "colour", "colour_sl", "colour_kempe"])
def test_jacobi_solve_small(name, schedule):
    s, part = case(name)
    check_jacobi_solve(s, part, schedule, 1e-8)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-6), ("fp32", 1e-10)])
def test_jacobi_solve_config2(precision, rtol):
    s = synth.config2()
    check_jacobi_solve(s, synth.partition_grid(s, 16), "level", rtol, precision)


@pytest.mark.parametrize("schedule", ["level", "colour_sl"])
def test_jacobi_solve_config3_full_size(schedule):
    s = synth.config3()
    check_jacobi_solve(s, synth.partition_grid(s, 150), schedule, 1e-3)


def test_one_partition_is_the_plain_preconditioner():
    s = synth.config2()
    b = dev(rhs(s))
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl") as a, \
            opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl",
                       part=np.zeros(s.nb, dtype=np.int32)) as j:
        np.testing.assert_array_equal(a.permutation(), j.permutation())
        xa, sa, ia, ra = a.solve(b, rtol=1e-6)
        xj, sj, ij, rj = j.solve(b, rtol=1e-6)
    assert (sa, ia, ra) == (sj, ij, rj)
    np.testing.assert_array_equal(xa.cpu().numpy(), xj.cpu().numpy())


def test_jacobi_batch_is_bitwise_identical_to_alone():
    syss = synth.config4(nsys=5)
    parts = [synth.partition_grid(s, 4) for s in syss]
    hs = [opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl", precision="fp32",
                     part=p) for s, p in zip(syss, parts)]
    bs = [dev(rhs(s)) for s in syss]
    alone = [h.solve(b, rtol=1e-6) for h, b in zip(hs, bs)]
    xs = [torch.empty_like(b) for b in bs]
    with opm.Batch([h.h for h in hs]) as bt:
        s_all, st, it, rr = bt.solve(bs, xs, rtol=1e-6)
    assert s_all == opm.OPM_OK
    for k, (xa, sa, ia, ra) in enumerate(alone):
        assert (st[k], it[k], rr[k]) == (sa, ia, ra)
        np.testing.assert_array_equal(xs[k].cpu().numpy(), xa.cpu().numpy())
    for h in hs:
        h.close()
