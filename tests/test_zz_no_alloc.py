"""The allocation-free residual entry point against the existing entry points
and the CPU oracle (collected last on purpose: a failure here leaves every
other test already run).

Callers that cannot allocate device memory where they need a residual (code
inside a simulator's own device-memory arena or fixed budget) use
opm_bsr_residual_noalloc; its scratch is a fixed array in device memory, so
the test also checks that two calls in a row give the right answer (the
array keeps the previous call's contents), that a call on a non-default
stream does too, that oversize or host inputs are refused before any kernel
runs, and that a column index outside the matrix is skipped by the kernel's
own check and reported.
"""
import numpy as np
import pytest

from oracle import spmv as oracle_spmv
from paper_2309_11488_gb300 import opm, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_against_oracle(s, xs_h, b_h, r, norms):
    """r = b - A x elementwise within 1e-12 of (|b| + |A||x|)_i, the SpMV
    tolerance of the GPU parity tests; both norms within 1e-12 / 1e-9."""
    ref = b_h - oracle_spmv(s.nb, s.rowptr, s.colidx, s.vals, xs_h)
    bound = np.abs(b_h) + oracle_spmv(s.nb, s.rowptr, s.colidx, np.abs(s.vals), np.abs(xs_h))
    assert np.all(np.abs(r.cpu().numpy() - ref) <= 1e-12 * bound + 1e-300)
    nrm = norms.cpu().numpy()
    np.testing.assert_allclose(nrm[1], np.linalg.norm(b_h), rtol=1e-12)
    np.testing.assert_allclose(nrm[0], np.linalg.norm(ref), rtol=1e-9, atol=1e-12 * np.linalg.norm(bound))
    return nrm


def test_noalloc_residual_matches_existing_entry_points_twice():
    s = synth.config2()
    rp, ci, va = dev(s.rowptr), dev(s.colidx), dev(s.vals)
    with opm.Solver(s.nb, rp, ci, va, schedule="colour") as sv:
        b = sv.spmv(dev(s.x_true))
        x, st, it, relres = sv.solve(b, rtol=1e-6)
        assert st == opm.OPM_OK
        b_h = b.cpu().numpy()
        for scale in (1.0, 2.0):  # two calls in a row, different inputs
            xs = x * scale
            r = torch.empty_like(b)
            norms = torch.zeros(2, dtype=torch.float64, device="cuda")
            assert opm.opm_bsr_residual_noalloc(s.nb, rp, ci, va, xs, b, r, norms) == opm.OPM_OK
            nrm = _check_against_oracle(s, xs.cpu().numpy(), b_h, r, norms)
            if scale == 1.0:
                # against the solver's own true residual for the same x
                np.testing.assert_allclose(nrm[0] / nrm[1], relres, rtol=1e-9)


def test_noalloc_residual_on_a_side_stream():
    s = synth.config1()
    rp, ci, va = dev(s.rowptr), dev(s.colidx), dev(s.vals)
    rng = np.random.default_rng(7)
    x_h = rng.uniform(-1, 1, 3 * s.nb)
    b_h = rng.uniform(-1, 1, 3 * s.nb)
    x, b = dev(x_h), dev(b_h)
    r = torch.full_like(x, np.nan)
    norms = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    assert opm.opm_bsr_residual_noalloc(s.nb, rp, ci, va, x, b, r, norms, stream=side) == opm.OPM_OK
    _check_against_oracle(s, x_h, b_h, r, norms)


def test_noalloc_rejects_oversize_and_host_arrays():
    s = synth.config1()
    rp, ci, va = dev(s.rowptr), dev(s.colidx), dev(s.vals)
    x = dev(s.x_true)
    b = torch.zeros_like(x)
    r = torch.empty_like(x)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    too_big = 2_097_152 + 1
    assert opm.opm_bsr_residual_noalloc(too_big, rp, ci, va, x, b, r, norms) == opm.OPM_ERR_ARG
    assert opm.opm_bsr_residual_noalloc(s.nb, s.rowptr, ci, va, x, b, r, norms) == opm.OPM_ERR_ARG
    assert opm.opm_bsr_residual_noalloc(s.nb, rp, ci, va, x, b, r, norms) == opm.OPM_OK


def test_noalloc_reports_a_column_outside_the_matrix():
    """One column index planted at nb (one past the last row): the kernel
    checks it before reading x, skips the block and reports the pattern
    error; the next well-formed call is right again."""
    s = synth.config1()
    bad = s.colidx.copy()
    bad[int(s.rowptr[7]) + 1] = s.nb
    rp, ci, va = dev(s.rowptr), dev(bad), dev(s.vals)
    x_h = s.x_true
    x = dev(x_h)
    b = torch.zeros_like(x)
    r = torch.empty_like(x)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert opm.opm_bsr_residual_noalloc(s.nb, rp, ci, va, x, b, r, norms) == opm.OPM_ERR_PATTERN
    assert np.all(np.isnan(norms.cpu().numpy()))
    ci_ok = dev(s.colidx)
    assert opm.opm_bsr_residual_noalloc(s.nb, rp, ci_ok, va, x, b, r, norms) == opm.OPM_OK
    _check_against_oracle(s, x_h, np.zeros(3 * s.nb), r, norms)
