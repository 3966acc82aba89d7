"""The products after a preconditioner application (opm_options.product_reuse),
on the CPU: the ILU0 property they rest on, checked with the oracle, and the
library's host analysis of which rows use it, checked against a brute-force
count over the permuted pattern.

ILU0 (Algorithm 2) leaves (LU)_ij = A_ij on the pattern.  Two consequences
for v = A p^ with p^ = inv(LU) p:
  * a row with no block left of its diagonal has an empty L row, so its U row
    is A's (no elimination touches it) and (A p^)_i = (U p^)_i = p_i;
  * a row on whose upper blocks no elimination product lands keeps
    U_ij = A_ij for j > i, so sum_{j>i} A_ij p^_j is the backward sweep's
    sum_{j>i} U_ij p^_j.
Block-Jacobi drops blocks from the preconditioner: rows with a dropped block
(the first case) or a dropped upper block (the second) walk A in full.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_11488_gb300 import opm, synth


def _classify(nb, rowptr, colidx, perm, part=None):
    """Brute force over the permuted pattern.  Returns (identity rows,
    reusing rows, blocks the products walk) in the permuted numbering."""
    iperm = np.empty(nb, dtype=np.int64)
    iperm[perm] = np.arange(nb)
    rows = []
    for ni in range(nb):
        oi = perm[ni]
        cols = {}
        for m in range(rowptr[oi], rowptr[oi + 1]):
            j = int(colidx[m])
            cols[int(iperm[j])] = part is None or part[oi] == part[j]
        rows.append(cols)
    ident, reuse, walked = set(), set(), 0
    for i in range(nb):
        cols = rows[i]
        lower = sum(1 for j in cols if j < i)
        upper = [j for j in cols if j > i]
        if lower == 0 and all(cols.values()):
            ident.add(i)
            continue
        hit = False
        for k, kept in cols.items():
            if k >= i or not kept:
                continue
            for j, kj_kept in rows[k].items():
                if j > k and kj_kept and j > i and cols.get(j, False):
                    hit = True
        if upper and all(cols[j] for j in upper) and not hit:
            reuse.add(i)
            walked += 1 + lower
        else:
            walked += len(cols)
    return ident, reuse, walked


def _patterns():
    yield "grid 10x10x5", synth.config1(), None
    yield "faulted grid 9^3", synth.config3(n=9), None
    yield "random pattern", synth.random_pattern_system(300, 3, seed=11), None
    s = synth.config1()
    yield "grid, 6 Jacobi partitions", s, synth.partition_grid(s, 6).astype(np.int32)


@pytest.mark.parametrize("schedule", ["colour_kempe", "level", "natural"])
def test_analysis_classifies_rows_like_brute_force(schedule):
    for name, s, part in _patterns():
        st, perm, info = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, schedule, part=part)
        assert st == opm.OPM_OK
        ident, reuse, walked = _classify(s.nb, s.rowptr, s.colidx, perm, part)
        assert info.rows_identity == len(ident), name
        assert info.rows_reuse == len(reuse), name
        assert info.nnzb_product == walked, name
        assert walked < len(s.colidx), name   # every pattern here saves blocks


def test_ilu0_keeps_a_on_clean_rows_and_products_equal():
    """The oracle's ILU0 of P A P^T: U's row is A's, bit for bit, on identity
    rows and on reusing rows' upper blocks; and the products formed the
    reusing way equal A p^ to rounding."""
    for name, s, part in _patterns():
        if part is not None:
            continue
        for schedule in ("colour_kempe", "natural"):
            perm, _ = O.schedule_perm(s.nb, s.rowptr, s.colidx, schedule)
            rp, ci, va = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
            ident, reuse, _ = _classify(s.nb, s.rowptr, s.colidx, perm)
            fac = O.ilu0(s.nb, rp, ci, va)
            assert fac.status == 0
            A = va.reshape(-1, 9)
            for i in ident | reuse:
                for m in range(rp[i], rp[i + 1]):
                    if ci[m] > i or (ci[m] == i and i in ident):
                        assert np.array_equal(fac.lu[m], A[m]), (name, schedule, i)
            rng = np.random.default_rng(5)
            p = rng.uniform(-1, 1, 3 * s.nb)
            ph = O.ilu_apply(s.nb, rp, ci, fac, p)
            v = O.spmv(s.nb, rp, ci, va, ph)
            bound = O.spmv(s.nb, rp, ci, np.abs(va), np.abs(ph)) + np.abs(p)
            for i in ident:
                sl = slice(3 * i, 3 * i + 3)
                assert np.all(np.abs(v[sl] - p[sl]) <= 1e-12 * bound[sl]), (name, schedule, i)
            for i in reuse:
                sl = slice(3 * i, 3 * i + 3)
                w = np.zeros(3)
                rest = np.zeros(3)
                for m in range(rp[i], rp[i + 1]):
                    blk = fac.lu[m].reshape(3, 3) if ci[m] > i else A[m].reshape(3, 3)
                    if ci[m] > i:
                        w += blk @ ph[3 * ci[m]:3 * ci[m] + 3]
                    else:
                        rest += blk @ ph[3 * ci[m]:3 * ci[m] + 3]
                assert np.all(np.abs(rest + w - v[sl]) <= 1e-13 * bound[sl]), (name, schedule, i)


def test_product_reuse_option_is_checked():
    o = opm.opm_options_default(product_reuse=1)
    s = synth.config1()
    st, h = opm.opm_bsr_create(s.nb, s.rowptr, s.colidx, s.vals, o, check=False)
    assert st == opm.OPM_ERR_ARG and h is None
