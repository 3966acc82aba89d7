"""Oracle pins for BiCGStab breakdown (Section 4.2 method; van der Vorst 1992):
on the small systems of tests/golden/bicgstab_breakdown.txt one of the four
divisors -- (r^, r), (r^, v), (t, t) or (t, s) -- is exactly zero, as the
fixture's exact rational derivation shows.  The oracle's building blocks
reproduce the fixture's vectors exactly (every value is a small dyadic
rational, so floating point is exact here), and its BiCGStab returns the
breakdown status -5 in the stated iteration, in natural and level order and,
for the block-Jacobi case, with the partition-internal preconditioner
(Section 4.5).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from breakdown_fixture import load

CASES = load()


def fdot(u, v):
    return sum((a * b for a, b in zip(u, v)), Fraction(0))


def _m_pattern(c):
    if c.part is None:
        return c.rowptr, c.colidx, c.vals
    mrp, mci, mv, _ = O.jacobi_pattern(c.nb, c.rowptr, c.colidx, c.vals, c.part)
    return mrp, mci, mv


def test_fixture_lists_every_breakdown_kind():
    assert {c.event for c in CASES.values()} == {"rho", "rhv", "tt", "omega"}
    assert {c.k for c in CASES.values()} == {1, 2}


@pytest.mark.parametrize("name", list(CASES))
def test_fixture_quantities_are_consistent(name):
    """The listed vectors satisfy the recurrence's scalar relations exactly,
    and the listed zero is the one the case names (block dots are three
    times the scalar ones, which leaves zeros and ratios unchanged)."""
    c = CASES[name]
    q = c.q
    b = [Fraction(v) for v in c.b[::3]]
    assert q["rho1"] == [fdot(b, b)]
    for k in (1, 2):
        if f"rhv{k}" in q:
            assert q[f"rhv{k}"] == [fdot(b, q[f"v{k}"])]
        if f"alpha{k}" in q:
            alpha = q[f"rho{k}"][0] / q[f"rhv{k}"][0]
            assert q[f"alpha{k}"] == [alpha]
            r_prev = b if k == 1 else q[f"r{k - 1}"]
            assert q[f"s{k}"] == [r - alpha * v for r, v in zip(r_prev, q[f"v{k}"])]
        if f"tt{k}" in q:
            assert q[f"tt{k}"] == [fdot(q[f"t{k}"], q[f"t{k}"])]
        if f"omega{k}" in q:
            assert q[f"omega{k}"] == [fdot(q[f"t{k}"], q[f"s{k}"]) / q[f"tt{k}"][0]]
        if f"r{k}" in q:
            om = q[f"omega{k}"][0]
            assert q[f"r{k}"] == [s - om * t for s, t in zip(q[f"s{k}"], q[f"t{k}"])]
            assert q[f"rho{k + 1}"] == [fdot(b, q[f"r{k}"])]
    assert q[f"{c.event}{c.k}"] == [0]


@pytest.mark.parametrize("name", list(CASES))
def test_oracle_building_blocks_reproduce_the_fixture_exactly(name):
    c = CASES[name]
    mrp, mci, mv = _m_pattern(c)
    fac = O.ilu0(c.nb, mrp, mci, mv)
    assert fac.status == 0
    q = c.q
    np.testing.assert_array_equal(O.ilu_apply(c.nb, mrp, mci, fac, c.b), c.vec("ph1"))  # p1 = r0 = b
    for k in (1, 2):
        if f"v{k}" in q:
            np.testing.assert_array_equal(O.spmv(c.nb, c.rowptr, c.colidx, c.vals, c.vec(f"ph{k}")), c.vec(f"v{k}"))
        if f"sh{k}" in q:
            np.testing.assert_array_equal(O.ilu_apply(c.nb, mrp, mci, fac, c.vec(f"s{k}")), c.vec(f"sh{k}"))
            np.testing.assert_array_equal(O.spmv(c.nb, c.rowptr, c.colidx, c.vals, c.vec(f"sh{k}")),
                                          c.vec(f"t{k}"))
    if "ph2" in q:
        # p2 = r1 + beta2 (p1 - omega1 v1), beta2 = (rho2 / rho1)(alpha1 / omega1), p1 = b
        beta = (q["rho2"][0] / q["rho1"][0]) * (q["alpha1"][0] / q["omega1"][0])
        p2 = [r + beta * (p - q["omega1"][0] * v) for r, p, v in zip(q["r1"], [Fraction(v) for v in c.b[::3]],
                                                                     q["v1"])]
        np.testing.assert_array_equal(O.ilu_apply(c.nb, mrp, mci, fac, np.repeat([float(v) for v in p2], 3)),
                                      c.vec("ph2"))
    if "x1" in q:
        # one iteration: the oracle's iterate is the fixture's x1, its residual norm ||r1||
        res = O.bicgstab(c.nb, c.rowptr, c.colidx, c.vals, fac, c.b, rtol=1e-14, maxit=1,
                         mpattern=(mrp, mci))
        assert res.status == 1 and res.iters == 1
        np.testing.assert_array_equal(res.x, c.vec("x1"))
        np.testing.assert_allclose(res.res_hist[2], np.sqrt(3 * float(fdot(q["r1"], q["r1"]))), rtol=1e-15)


@pytest.mark.parametrize("name", list(CASES))
def test_oracle_bicgstab_reports_breakdown_in_the_stated_iteration(name):
    c = CASES[name]
    mrp, mci, mv = _m_pattern(c)
    fac = O.ilu0(c.nb, mrp, mci, mv)
    res = O.bicgstab(c.nb, c.rowptr, c.colidx, c.vals, fac, c.b, rtol=1e-14, maxit=50, mpattern=(mrp, mci))
    assert res.status == -5
    assert res.iters == c.k
    # whole-path form with the oracle's own schedule permutation (identity for
    # these patterns in natural and level order)
    for schedule in ("natural", "level"):
        x, r2, perm, _ = O.solve_system(c.nb, c.rowptr, c.colidx, c.vals, c.b, 1e-14, 50, schedule, part=c.part)
        np.testing.assert_array_equal(perm, np.arange(c.nb))
        assert (r2.status, r2.iters) == (-5, c.k)


def test_scaling_b_keeps_the_breakdown():
    """Every divisor scales with b (rho and (r^, v) by c^2, (t, t) by c^2,
    (t, s) by c^2): scaling b by a power of two keeps the exact zero."""
    for c in CASES.values():
        mrp, mci, mv = _m_pattern(c)
        fac = O.ilu0(c.nb, mrp, mci, mv)
        res = O.bicgstab(c.nb, c.rowptr, c.colidx, c.vals, fac, 4.0 * c.b, rtol=1e-14, maxit=50,
                         mpattern=(mrp, mci))
        assert (res.status, res.iters) == (-5, c.k)
