"""GPU parity of the BiCGStab products after a preconditioner application
(opm_options.product_reuse, on by default for FP64 factors): with it, the
products take (A p^)_i = p_i on rows with no block left of the diagonal and
the backward sweep's upper sum on rows whose upper blocks no elimination
product changed.  Every case solves with the reuse on and off through the C
ABI and compares both with the FP64 CPU oracle (same seeded inputs, same row
order) at the tolerances of the parity tests: x within 1e-8 of the oracle's,
equal iteration counts (one apart only at the stopping threshold), relres
within 1e-6 relative of the oracle's true residual.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_11488_gb300 import opm, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _close_to_oracle(res, it, x, relres, x_ref, rtol):
    if it != res.iters:
        assert abs(it - res.iters) == 1
        h = res.res_hist / res.res_hist[0]
        k = min(it, res.iters)
        assert any(abs(v / rtol - 1) < 1e-6 for v in (h[2 * k - 1], h[2 * k]) if np.isfinite(v))
    else:
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert relres <= rtol * (1 + 1e-6)
    assert abs(relres - res.relres) <= 1e-6 * max(res.relres, 1e-300) + 1e-14


def _solve_both(s, schedule, rtol, maxit=200, wells=None, **kw):
    if wells is None:
        b = O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true)
    else:
        b = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, wells, s.x_true)
    x_ref, res, perm, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, rtol, maxit, schedule,
                                         part=kw.get("part"), wells=wells)
    out = {}
    for reuse in (0, -1):
        with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule=schedule,
                        product_reuse=reuse, **kw) as sv:
            np.testing.assert_array_equal(sv.permutation(), perm)
            if wells is not None:
                assert sv.set_wells(wells) == opm.OPM_OK
            info = sv.info()
            xd, st, it, relres = sv.solve(dev(b), rtol=rtol, maxit=maxit)
            x = xd.cpu().numpy()
        assert st == res.status == 0
        _close_to_oracle(res, it, x, relres, x_ref, rtol)
        out[reuse] = (it, x, info)
    return out


SMALL = {
    "c1": synth.config1,
    "ragged33": lambda: synth.random_pattern_system(33, 3, 41),
    "long_rows": lambda: synth.random_pattern_system(70, 20, 42),
    "dense40": lambda: synth.random_pattern_system(40, 0, 43, dense=True),
    "tree": lambda: synth.tree_system(300, 44),
    "one_way200": lambda: synth.one_way_system(synth.random_pattern_system(200, 4, 45), 0.5, 46),
    "faulted12": lambda: synth.config3(n=12),
}


@pytest.mark.parametrize("sweep", ["per_phase", "cooperative"])
@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("schedule", ["natural", "level", "colour_kempe"])
def test_small_systems_with_and_without_reuse(name, schedule, sweep):
    s = SMALL[name]()
    out = _solve_both(s, schedule, 1e-8, sweep_launch=sweep)
    assert out[0][2].nnzb_product <= out[-1][2].nnzb_product == s.rowptr[-1]
    st, _, an = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, schedule)
    assert out[0][2].nnzb_product == an.nnzb_product and out[0][2].rows_reuse == an.rows_reuse


@pytest.mark.parametrize("rtol", [1e-2, 1e-6])
def test_config2_with_and_without_reuse(rtol):
    _solve_both(synth.config2(), "colour_kempe", rtol)


def test_config3_full_size_with_and_without_reuse():
    out = _solve_both(synth.config3(), "colour_kempe", 1e-6)
    info = out[0][2]
    assert info.nnzb_product < 0.55 * info.nnzb and info.rows_identity > 0.45 * info.nb


def test_block_jacobi_with_and_without_reuse():
    s = synth.config1()
    part = synth.partition_grid(s, 6).astype(np.int32)
    _solve_both(s, "colour_kempe", 1e-8, part=part)


def test_chow_patel_factors_with_and_without_reuse():
    """Chow-Patel factors keep A's values on the rows the reuse relies on
    (no listed product touches them), so after enough sweeps to reach the
    exact factors the solve matches the oracle either way."""
    s = synth.config1()
    b = O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true)
    x_ref, res, perm, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-8, 200, "colour_kempe")
    for reuse in (0, -1):
        with opm.Solver(s.nb, dev(s.rowptr), dev(s.colidx), dev(s.vals), schedule="colour_kempe",
                        cp_sweeps=8, product_reuse=reuse) as sv:
            xd, st, it, relres = sv.solve(dev(b), rtol=1e-8)
            x = xd.cpu().numpy()
        assert st == 0
        _close_to_oracle(res, it, x, relres, x_ref, 1e-8)


def test_fp32_factors_never_reuse():
    s = synth.config1()
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="colour_kempe", precision="fp32") as sv:
        info = sv.info()
    assert info.nnzb_product == info.nnzb and info.rows_reuse == 0


def test_jacobi_triangular_sweeps_never_reuse():
    s = synth.config1()
    with opm.Solver(s.nb, s.rowptr, s.colidx, s.vals, schedule="colour_kempe", tri_sweeps=4) as sv:
        info = sv.info()
    assert info.nnzb_product == info.nnzb


@pytest.mark.parametrize("schedule", ["level", "colour_kempe"])
def test_wells_with_and_without_reuse(schedule):
    """The wells' term starts the product's sum as in the plain product."""
    s = synth.config1()
    _solve_both(s, schedule, 1e-8, wells=synth.wells(s, 3, 4))
