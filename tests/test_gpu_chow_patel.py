"""GPU parity of the iterative ILU0 (Chow & Patel sweeps, option cp_sweeps)
and of the Jacobi triangular solves (option tri_sweeps) against the oracle.

Both sides use the same schedule order (the oracle's own permutation) and the
same number of sweeps.  Tolerances as for the exact path: FP64 factors 1e-12
relative to the block row's largest entry, applications 1e-11, solves equal
iteration counts (one apart only at a threshold tie) and x within 1e-8.
A converged iteration must give the exact factorisation bit for bit, since
every target sees the exact path's FMA chain in the same order.
"""
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


def permuted(s, schedule):
    perm, nsets = O.schedule_perm(s.nb, s.rowptr, s.colidx, schedule)
    prow, pcol, pval = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    return perm, nsets, prow, pcol, pval


def check_factors(nb, prow, pcol, fac, lu, dinv, tol):
    rows = np.repeat(np.arange(nb), np.diff(prow))
    off = rows != pcol
    ref = fac.lu
    err = np.abs(lu - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-300)
    assert err[off].max(initial=0.0) <= tol
    derr = np.abs(dinv - fac.dinv).max(axis=1) / np.maximum(np.abs(fac.dinv).max(axis=1), 1e-300)
    assert derr.max() <= tol


SMALL = {
    "c1": synth.config1,
    "one_row": lambda: synth.block_diagonal_system(1, 3),
    "ragged33": lambda: synth.random_pattern_system(33, 3, 41),
    "long_rows": lambda: synth.random_pattern_system(70, 20, 42),
    "chain": lambda: synth.chain_system(100),
    "one_way200": lambda: synth.one_way_system(synth.random_pattern_system(200, 4, 45), 0.5, 46),
}


@pytest.fixture(scope="module")
def c3():
    return synth.config3()


@pytest.mark.parametrize("sweeps", [1, 2, 5])
@pytest.mark.parametrize("schedule", ["natural", "level", "colour"])
@pytest.mark.parametrize("name", list(SMALL))
def test_cp_factors_match_oracle(name, schedule, sweeps):
    s = SMALL[name]()
    perm, nsets, prow, pcol, pval = permuted(s, schedule)
    fac = O.ilu0(s.nb, prow, pcol, pval, cp_sweeps=sweeps)
    assert fac.status == 0
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule=schedule, cp_sweeps=sweeps) as sv:
        np.testing.assert_array_equal(sv.permutation(), perm)
        lu, dinv = sv.factors()
    check_factors(s.nb, prow, pcol, fac, lu, dinv, 1e-12)


@pytest.mark.parametrize("schedule", ["natural", "colour"])
def test_cp_converged_is_the_exact_factorisation_bitwise(schedule):
    """The longest dependency chain of a 40-row pattern is below 41 sweeps."""
    s = synth.random_pattern_system(40, 3, 43)
    _, _, prow, pcol, _ = permuted(s, schedule)
    off = np.repeat(np.arange(s.nb), np.diff(prow)) != pcol
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule=schedule) as sv:
        lu0, d0 = sv.factors()
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule=schedule, cp_sweeps=41) as sv:
        lu1, d1 = sv.factors()
    np.testing.assert_array_equal(lu1[off], lu0[off])
    np.testing.assert_array_equal(d1, d0)


def test_cp_one_sweep_is_exact_under_two_colours():
    """Two colours: every dependency chain has length one (the initial guess
    is already exact for the first colour's rows and for L)."""
    s = synth.config1()
    _, nsets, *_ = permuted(s, "colour")
    assert nsets == 2
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="colour") as sv:
        lu0, d0 = sv.factors()
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="colour", cp_sweeps=1) as sv:
        lu1, d1 = sv.factors()
    _, _, prow, pcol, _ = permuted(s, "colour")
    off = np.repeat(np.arange(s.nb), np.diff(prow)) != pcol
    np.testing.assert_array_equal(lu1[off], lu0[off])
    np.testing.assert_array_equal(d1, d0)


@pytest.mark.parametrize("schedule", ["level", "colour"])
def test_cp_factors_config3_full_size(c3, schedule):
    perm, nsets, prow, pcol, pval = permuted(c3, schedule)
    fac = O.ilu0(c3.nb, prow, pcol, pval, cp_sweeps=2)
    with opm.Solver(c3.nb, dev(c3.rowptr), dev(c3.colidx), dev(c3.vals), schedule=schedule, cp_sweeps=2) as sv:
        lu, dinv = sv.factors()
    check_factors(c3.nb, prow, pcol, fac, lu, dinv, 1e-12)


def test_cp_refactor_with_new_values():
    """opm_ilu0_factor with new values runs the sweeps on them (the initial
    guess copies the caller's values)."""
    s = synth.config1()
    vals2 = s.vals * 1.5
    vals2[::7] *= 0.9
    perm, nsets, prow, pcol, _ = permuted(s, "level")
    _, _, pval2 = O.permute(s.nb, s.rowptr, s.colidx, vals2, perm)
    fac = O.ilu0(s.nb, prow, pcol, pval2, cp_sweeps=3)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="level", cp_sweeps=3) as sv:
        assert sv.factor(vals2) == 0
        lu, dinv = sv.factors()
        assert sv.factor() == 0  # refactor the values the handle now holds
        lu2, dinv2 = sv.factors()
    check_factors(s.nb, prow, pcol, fac, lu, dinv, 1e-12)
    np.testing.assert_array_equal(lu2, lu)
    np.testing.assert_array_equal(dinv2, dinv)


def test_cp_flags_a_singular_pivot():
    s = synth.block_diagonal_system(4, 9)
    vals = s.vals.copy()
    vals[2] = np.array([1.0, 2, 3, 2, 4, 6, 0, 0, 1])
    st, h = opm.opm_bsr_create(s.nb, s.rowptr, s.colidx, vals,
                               opm.opm_options_default(schedule="natural", cp_sweeps=2), check=False)
    try:
        assert st == opm.OPM_ERR_ZERO_PIVOT
        assert opm.opm_last_error_row(h) == 2
    finally:
        opm.opm_destroy(h)


@pytest.mark.parametrize("sweeps", [1, 3, 8])
@pytest.mark.parametrize("schedule", ["natural", "level", "colour"])
@pytest.mark.parametrize("name", list(SMALL))
def test_jacobi_apply_matches_oracle(name, schedule, sweeps):
    s = SMALL[name]()
    perm, nsets, prow, pcol, pval = permuted(s, schedule)
    fac = O.ilu0(s.nb, prow, pcol, pval)
    r = synth.uniform(synth.stream_key(9, 9), np.arange(3 * s.nb, dtype=np.uint64), -1, 1)
    zp = O.ilu_apply(s.nb, prow, pcol, fac, r.reshape(-1, 3)[perm].ravel(), tri_sweeps=sweeps)
    z_ref = np.empty_like(zp)
    z_ref.reshape(-1, 3)[perm] = zp.reshape(-1, 3)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule=schedule, tri_sweeps=sweeps) as sv:
        z = sv.ilu_apply(r)
    np.testing.assert_allclose(z, z_ref, rtol=1e-11, atol=1e-12 * np.abs(z_ref).max())


def test_jacobi_apply_config3_full_size(c3):
    perm, nsets, prow, pcol, pval = permuted(c3, "level")
    fac = O.ilu0(c3.nb, prow, pcol, pval, cp_sweeps=2)
    r = synth.uniform(synth.stream_key(9, 10), np.arange(3 * c3.nb, dtype=np.uint64), -1, 1)
    zp = O.ilu_apply(c3.nb, prow, pcol, fac, r.reshape(-1, 3)[perm].ravel(), tri_sweeps=3)
    z_ref = np.empty_like(zp)
    z_ref.reshape(-1, 3)[perm] = zp.reshape(-1, 3)
    with opm.Solver(c3.nb, dev(c3.rowptr), dev(c3.colidx), dev(c3.vals), schedule="level", cp_sweeps=2,
                    tri_sweeps=3) as sv:
        z = sv.ilu_apply(dev(r)).cpu().numpy()
    np.testing.assert_allclose(z, z_ref, rtol=1e-11, atol=1e-12 * np.abs(z_ref).max())


def check_solve(s, schedule, rtol, cp, tri, maxit=400, xtol=1e-8):
    b = rhs(s)
    x_ref, res, perm, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, rtol, maxit, schedule,
                                         cp_sweeps=cp, tri_sweeps=tri)
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=schedule, cp_sweeps=cp,
                    tri_sweeps=tri) as sv:
        xd, st, it, relres = sv.solve(dev(b), rtol=rtol, maxit=maxit)
        x = xd.cpu().numpy()
    assert st == res.status == 0
    if it != res.iters:
        assert abs(it - res.iters) == 1
        h = res.res_hist / res.res_hist[0]
        k = min(it, res.iters)
        near = [h[2 * k - 1], h[2 * k]]
        assert any(abs(v / rtol - 1) < 1e-6 for v in near if np.isfinite(v))
    else:
        assert np.linalg.norm(x - x_ref) <= xtol * np.linalg.norm(x_ref)
    assert relres <= rtol * (1 + 1e-6)
    assert abs(relres - res.relres) <= 1e-6 * max(res.relres, 1e-300) + 1e-14
    return it


@pytest.mark.parametrize("cp,tri", [(0, 2), (2, 0), (3, 3), (1, 6)])
@pytest.mark.parametrize("schedule", ["natural", "level", "colour"])
def test_solve_matches_oracle(schedule, cp, tri):
    check_solve(synth.config1(), schedule, 1e-8, cp, tri)


def test_solve_config2():
    check_solve(synth.config2(), "level", 1e-6, 3, 3)


def test_solve_config3_full_size(c3):
    check_solve(c3, "level", 1e-3, 3, 3)


def test_gmres_with_iterative_preconditioner_converges():
    s = synth.config1()
    b = rhs(s)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="level", cp_sweeps=3, tri_sweeps=3) as sv:
        x, st, it, relres = sv.gmres(b, rtol=1e-8, maxit=300, restart=30)
    assert st == 0 and relres <= 1e-8 * (1 + 1e-6)
    assert np.linalg.norm(x - s.x_true) <= 1e-6 * np.linalg.norm(s.x_true)


def test_batch_is_bitwise_the_handles_alone():
    systems = [synth.config1(seed=100 + q) for q in range(3)]
    alone = []
    for s in systems:
        with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="level", cp_sweeps=2, tri_sweeps=3) as sv:
            x, st, it, rr = sv.solve(rhs(s), rtol=1e-8, maxit=300)
            alone.append((x, st, it, rr))
    sv = [opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="level") for s in systems]
    try:
        with opm.Batch([v.h for v in sv], cp_sweeps=2, tri_sweeps=3) as bt:
            s0, sts = bt.factor([s.vals for s in systems])
            assert s0 == 0
            xs = [np.empty(3 * s.nb) for s in systems]
            s1, sts, its, rrs = bt.solve([rhs(s) for s in systems], xs, rtol=1e-8, maxit=300)
        for q in range(3):
            assert sts[q] == alone[q][1] == 0 and its[q] == alone[q][2]
            np.testing.assert_array_equal(xs[q], alone[q][0])
    finally:
        for v in sv:
            v.close()


def test_fp32_factors_with_iterative_sweeps_reach_the_tight_tolerance():
    s = synth.config2()
    b = rhs(s)
    x_ref, res, _, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-10, 400, "level", cp_sweeps=3,
                                      tri_sweeps=3)
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="level", precision="fp32", cp_sweeps=3,
                    tri_sweeps=3) as sv:
        x, st, it, relres = sv.solve(b, rtol=1e-10, maxit=400)
    assert st == 0 and relres <= 1e-10 * (1 + 1e-6)
    # single-precision sweeps give a slightly different preconditioner, which
    # BiCGStab at 1e-10 turns into a few iterations either way
    assert abs(it - res.iters) <= max(2, res.iters // 8)
    assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
