"""Restarted GMRES(m) through the C ABI against the oracle's orc_gmres on the
same row order: same Arnoldi-step count (a difference of one only when the
oracle's estimate at the library's stopping point is within 1e-6 of the
threshold) and x within 1e-8; with block-Jacobi factors or wells the true
residual is checked with the oracle's operator."""
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


def check_gmres(s, schedule, rtol, restart, maxit=300):
    b = rhs(s)
    x_ref, res, perm = O.solve_system_gmres(s.nb, s.rowptr, s.colidx, s.vals, b, rtol, maxit, restart, schedule)
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=schedule) as sv:
        np.testing.assert_array_equal(sv.permutation(), perm)
        xd, st, it, rr = sv.gmres(dev(b), rtol=rtol, maxit=maxit, restart=restart)
        x = xd.cpu().numpy()
    assert st == res.status == 0
    if it != res.iters:
        assert abs(it - res.iters) == 1
        k = min(it, res.iters)
        assert abs(res.res_hist[k] / (rtol * res.res_hist[0]) - 1) < 1e-6
    else:
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert rr <= rtol * (1 + 1e-6)
    assert abs(rr - res.relres) <= 1e-6 * max(res.relres, 1e-300) + 1e-14
    return it


SMALL = {
    "c1": synth.config1,
    "ragged33": lambda: synth.random_pattern_system(33, 3, 41),
    "tree": lambda: synth.tree_system(300, 44),
    "long_rows": lambda: synth.random_pattern_system(70, 20, 42),
    "one_way200": lambda: synth.one_way_system(synth.random_pattern_system(200, 4, 45), 0.5, 46),
}


@pytest.mark.parametrize("restart", [30, 4])
@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("schedule", ["level", "colour", "colour_sl"])
def test_gmres_small(name, schedule, restart):
    check_gmres(SMALL[name](), schedule, 1e-8, restart)


@pytest.mark.parametrize("restart", [30, 10])
def test_gmres_config2(restart):
    check_gmres(synth.config2(), "colour_sl", 1e-6, restart)


def test_gmres_config3_full_size():
    check_gmres(synth.config3(), "colour_sl", 1e-3, 30)


@pytest.mark.parametrize("n", [54, 56, 60])
def test_gmres_gram_schmidt_tilings(n):
    """Faulted grids of 149,595, 166,822 and 205,187 cells: on 152 SMs the
    Gram-Schmidt kernels take 4, 5 and 6 rows per thread there (the host
    picks the count whose tiles fill whole rounds of the SMs), each with a
    ragged last tile; restarts every 10 steps."""
    check_gmres(synth.config3(n=n), "colour_kempe", 1e-6, 10)


def test_gmres_maxit_and_zero_rhs():
    s = synth.config2()
    b = dev(rhs(s))
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl") as sv:
        x, st, it, rr = sv.gmres(b, rtol=1e-12, maxit=7, restart=5)
        assert st == opm.OPM_NOT_CONVERGED and it == 7 and rr < 1.0
        x, st, it, rr = sv.gmres(torch.zeros_like(b), rtol=1e-6)
        assert st == opm.OPM_OK and it == 0 and rr == 0.0 and float(torch.abs(x).max()) == 0.0
        x, st, it, rr = sv.gmres(b, rtol=1e-6, restart=65)
        assert st == opm.OPM_ERR_ARG


def test_gmres_with_block_jacobi_and_wells():
    s = synth.config2()
    part = synth.partition_grid(s, 16)
    w = synth.wells(s, 6, 12)
    b = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, s.x_true)
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="level", part=part) as sv:
        assert sv.set_wells(w) == opm.OPM_OK
        xd, st, it, rr = sv.gmres(dev(b), rtol=1e-8, maxit=400, restart=30)
        x = xd.cpu().numpy()
    assert st == opm.OPM_OK and rr <= 1e-8 * (1 + 1e-6)
    r = b - O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, x)
    np.testing.assert_allclose(np.linalg.norm(r) / np.linalg.norm(b), rr, rtol=1e-6, atol=1e-14)
    assert np.linalg.norm(x - s.x_true) <= 1e-5 * np.linalg.norm(s.x_true)


def test_gmres_graph_reused_across_restart_lengths_and_edge_cases():
    """The solve runs as one graph built on first use: calls with other
    restart lengths, host buffers and wells set afterwards keep the
    oracle's step counts and x; maxit = 0 and a non-finite b take their
    documented outcomes."""
    s = synth.config1()
    b = rhs(s)
    with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_sl") as sv:
        for restart, on_device in ((5, True), (30, False), (5, True), (12, False)):
            x_ref, res, _ = O.solve_system_gmres(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-8, 300, restart,
                                                 "colour_sl")
            xb = dev(b) if on_device else b.copy()
            x, st, it, rr = sv.gmres(xb, rtol=1e-8, maxit=300, restart=restart)
            x = x.cpu().numpy() if on_device else x
            assert (st, it) == (res.status, res.iters) == (0, res.iters)
            assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
        x, st, it, rr = sv.gmres(dev(b), rtol=1e-8, maxit=0, restart=5)
        assert (st, it) == (opm.OPM_NOT_CONVERGED, 0) and rr == 1.0 and float(torch.abs(x).max()) == 0.0
        bad = b.copy()
        bad[7] = np.inf
        x = np.full(3 * s.nb, 3.0)
        x, st, it, rr = sv.gmres(bad, x, rtol=1e-8, restart=5)
        assert st == opm.OPM_ERR_NONFINITE and np.isnan(rr) and not x.any()
        # wells added after the graph was built: the graph is rebuilt with them
        w = synth.wells(s, 2, 3)
        bw = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, s.x_true)
        assert sv.set_wells(w) == opm.OPM_OK
        x, st, it, rr = sv.gmres(dev(bw), rtol=1e-8, maxit=300, restart=30)
        x = x.cpu().numpy()
        assert st == opm.OPM_OK
        r = bw - O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, x)
        np.testing.assert_allclose(np.linalg.norm(r) / np.linalg.norm(bw), rr, rtol=1e-6, atol=1e-14)
