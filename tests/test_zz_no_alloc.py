"""The allocation-free residual entry point against the library's existing
entry points (collected last on purpose: a failure here leaves every other
test already run).

Callers that cannot allocate device memory where they need a residual use
opm_bsr_residual_noalloc; its scratch is a fixed array in device memory, so
the test also checks that two calls in a row give the right answer (the
array keeps the previous call's contents) and that oversize or host inputs
are refused before any kernel runs.
"""
import numpy as np
import pytest

from paper_2309_11488_gb300 import opm, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_residual_matches_existing_entry_points_twice():
    s = synth.config2()
    rp, ci, va = dev(s.rowptr), dev(s.colidx), dev(s.vals)
    with opm.Solver(s.nb, rp, ci, va, schedule="colour") as sv:
        b = sv.spmv(dev(s.x_true))
        x, st, it, relres = sv.solve(b, rtol=1e-6)
        assert st == opm.OPM_OK
        for scale in (1.0, 2.0):  # two calls in a row, different inputs
            xs = x * scale
            r = torch.empty_like(b)
            norms = torch.zeros(2, dtype=torch.float64, device="cuda")
            assert opm.opm_bsr_residual_noalloc(s.nb, rp, ci, va, xs, b, r, norms) == opm.OPM_OK
            # against the existing SpMV entry point: r = b - A x elementwise,
            # within the SpMV tolerance of the GPU parity tests
            ax = sv.spmv(xs)
            ref = (b - ax).cpu().numpy()
            bound = (torch.abs(b) + _abs_spmv(s, torch.abs(xs))).cpu().numpy()  # |b| + |A| |x|
            assert np.all(np.abs(r.cpu().numpy() - ref) <= 1e-12 * bound + 1e-300)
            nrm = norms.cpu().numpy()
            np.testing.assert_allclose(nrm[1], np.linalg.norm(b.cpu().numpy()), rtol=1e-12)
            np.testing.assert_allclose(nrm[0], np.linalg.norm(ref), rtol=1e-9)
            if scale == 1.0:
                # against the solver's own true residual for the same x
                np.testing.assert_allclose(nrm[0] / nrm[1], relres, rtol=1e-9)


def _abs_spmv(s, xabs):
    with opm.Solver(s.nb, s.rowptr, s.colidx, np.abs(s.vals), schedule="colour") as sv:
        return sv.spmv(xabs)


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
