"""BiCGStab breakdown on the GPU (Section 4.2 method, van der Vorst 1992):
the small systems of tests/golden/bicgstab_breakdown.txt meet an exact zero
in one of the four divisors -- (r^, r), (r^, v), (t, t), (t, s) -- in a
stated iteration.  Their values are small dyadic rationals, so every
floating-point order reaches the same exact zero; the oracle pins
(tests/test_oracle_breakdown.py) show the oracle returning status -5 there.

The library must return OPM_ERR_BREAKDOWN with the same iteration count and
x zero-filled (the opm_bicgstab_solve contract for a negative status), alone,
with FP32 factors, and inside a batch whose other members are unaffected
(bitwise equal to their solves alone).
"""
import numpy as np
import pytest

import oracle as O
from breakdown_fixture import load
from paper_2309_11488_gb300 import opm, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solver(c, schedule, precision="fp64"):
    return opm.Solver(c.nb, dev(c.rowptr), dev(c.colidx), dev(c.vals), schedule=schedule, precision=precision,
                      part=c.part)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("schedule", ["natural", "level"])
@pytest.mark.parametrize("name", list(CASES))
def test_breakdown_status_iteration_and_zero_fill(name, schedule, precision):
    c = CASES[name]
    _, ref, perm, _ = O.solve_system(c.nb, c.rowptr, c.colidx, c.vals, c.b, 1e-14, 50, schedule,
                                     f32=precision == "fp32", part=c.part)
    assert (ref.status, ref.iters) == (-5, c.k)
    with solver(c, schedule, precision) as sv:
        assert sv.status == opm.OPM_OK
        np.testing.assert_array_equal(sv.permutation(), perm)
        for on_device in (True, False):
            b = dev(c.b) if on_device else c.b.copy()
            x = torch.full_like(b, np.nan) if on_device else np.full(3 * c.nb, np.nan)
            x, st, it, rr = sv.solve(b, x, rtol=1e-14, maxit=50)
            assert st == opm.OPM_ERR_BREAKDOWN
            assert it == c.k
            xh = x.cpu().numpy() if on_device else x
            np.testing.assert_array_equal(xh, np.zeros(3 * c.nb))
        # the handle stays usable: a solve with a right-hand side that does
        # not break down converges (b = A e, e the all-ones vector)
        b_ok = O.spmv(c.nb, c.rowptr, c.colidx, c.vals, np.ones(3 * c.nb))
        _, ref_ok, _, _ = O.solve_system(c.nb, c.rowptr, c.colidx, c.vals, b_ok, 1e-10, 50, schedule,
                                         f32=precision == "fp32", part=c.part)
        if ref_ok.status == 0:
            x, st, it, rr = sv.solve(dev(b_ok), rtol=1e-10, maxit=50)
            assert st == opm.OPM_OK and np.isfinite(x.cpu().numpy()).all()


def test_breakdown_in_a_scaled_right_hand_side():
    """Scaling b by a power of two scales every divisor by its square: the
    exact zero, the status and the iteration stay."""
    for c in CASES.values():
        with solver(c, "natural") as sv:
            x, st, it, rr = sv.solve(dev(8.0 * c.b), rtol=1e-14, maxit=50)
            assert (st, it) == (opm.OPM_ERR_BREAKDOWN, c.k)
            assert not x.cpu().numpy().any()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_breakdown_inside_a_batch_leaves_the_others_alone(precision):
    """Breakdown members report OPM_ERR_BREAKDOWN in their own iteration with
    x zero-filled; the ordinary members converge exactly as when solved
    alone (bitwise), and the batch's combined status is the breakdown."""
    normal = [synth.config1(), synth.random_pattern_system(300, 3, 61), synth.chain_system(40)]
    members = []  # (system, partition, b, its breakdown case or None)
    for k, s in enumerate(normal):
        members.append((s, None, O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true), None))
        c = list(CASES.values())[k % len(CASES)]
        members.append((c, c.part, c.b, c))
    c_last = CASES["jacobi_rho2"]
    members.append((c_last, c_last.part, c_last.b, c_last))
    rtol = 1e-10
    alone = []
    for s, part, b, c in members:
        sched = "natural" if c is not None else "colour"
        with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=sched, precision=precision,
                        part=part) as sv:
            x, st, it, rr = sv.solve(dev(b), rtol=rtol, maxit=50)
            alone.append((x.cpu().numpy(), st, it, rr))
    handles = []
    for s, part, b, c in members:
        sched = "natural" if c is not None else "colour"
        handles.append(opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=sched,
                                  precision=precision, part=part))
    bs = [dev(b) for _, _, b, _ in members]
    xs = [torch.full_like(b, np.nan) for b in bs]
    with opm.Batch([h.h for h in handles]) as bt:
        s_all, st, it, rr = bt.solve(bs, xs, rtol=rtol, maxit=50)
    for h in handles:
        h.close()
    assert s_all == opm.OPM_ERR_BREAKDOWN
    for k, (s, part, b, c) in enumerate(members):
        xa, sta, ita, rra = alone[k]
        xk = xs[k].cpu().numpy()
        if c is not None:
            assert (st[k], it[k]) == (opm.OPM_ERR_BREAKDOWN, c.k) == (sta, ita)
            np.testing.assert_array_equal(xk, np.zeros(3 * s.nb))
        else:
            assert st[k] == sta == opm.OPM_OK and it[k] == ita and rr[k] == rra
            np.testing.assert_array_equal(xk, xa)
