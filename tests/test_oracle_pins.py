"""Pins of the FP64 CPU oracle to facts outside itself (CPU only).

Each test checks the oracle against mathematics or the paper, never against a
retyping of its own formula: dense brute force, exact LU on no-fill patterns,
the ILU0 defining identity (LU)_ij = A_ij on the pattern, closed forms of the
block Thomas recurrence and of grid schedules, and the generator's sizes
printed in the paper's benchmark table.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2309_11488_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_facts():
    out = {}
    with open(os.path.join(GOLDEN, "paper_facts.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


def dense_factors(sysm, fac):
    """Dense unit-lower L and upper U from the oracle's packed factors."""
    nb = sysm.nb
    L = np.eye(3 * nb)
    U = np.zeros((3 * nb, 3 * nb))
    lu = fac.lu.reshape(-1, 3, 3).astype(np.float64)
    for i in range(nb):
        for m in range(sysm.rowptr[i], sysm.rowptr[i + 1]):
            j = sysm.colidx[m]
            if j < i:
                L[3 * i:3 * i + 3, 3 * j:3 * j + 3] = lu[m]
            else:
                U[3 * i:3 * i + 3, 3 * j:3 * j + 3] = lu[m]
    return L, U


def rhs(s):
    return O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true)


# ---------------------------------------------------------------- blocks

def test_inv3_matches_numpy():
    key = synth.stream_key(7, 1)
    a = synth.uniform(key, np.arange(9 * 50, dtype=np.uint64), -1, 1).reshape(50, 3, 3)
    a += 3 * np.eye(3)
    for m in range(50):
        inv, st = O.inv3(a[m])
        assert st == 0
        np.testing.assert_allclose(inv, np.linalg.inv(a[m]), rtol=1e-13, atol=1e-14)


def test_inv3_needs_pivoting_and_flags_singular():
    a = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 2.0]])  # zero leading entry
    inv, st = O.inv3(a)
    assert st == 0
    np.testing.assert_allclose(inv @ a, np.eye(3), atol=1e-15)
    _, st = O.inv3(np.array([[1.0, 2, 3], [2, 4, 6], [0, 0, 1]]))
    assert st == -1


# ---------------------------------------------------------------- SpMV

@pytest.mark.parametrize("maker", [synth.config1, lambda: synth.random_pattern_system(40, 3, 11),
                                   lambda: synth.tree_system(30, 5)])
def test_spmv_brute_force(maker):
    s = maker()
    A = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    y = O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true)
    np.testing.assert_allclose(y, A @ s.x_true, rtol=1e-13, atol=1e-13)


def test_spmv_block_is_row_major():
    # one block row, one block: y = B x with B[r][c] = vals[3r + c]
    vals = np.arange(1.0, 10.0).reshape(1, 9)
    y = O.spmv(1, np.array([0, 1]), np.array([0]), vals, np.array([1.0, 0.0, 0.0]))
    np.testing.assert_array_equal(y, [1.0, 4.0, 7.0])  # first column of row-major [[1,2,3],[4,5,6],[7,8,9]]


# ---------------------------------------------------------------- ILU0

def test_block_thomas_closed_form():
    rows = []
    with open(os.path.join(GOLDEN, "block_thomas.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    nb = len(rows)
    rowptr = [0]
    colidx, vals = [], []
    for i in range(nb):
        for j in (i - 1, i, i + 1):
            if 0 <= j < nb:
                colidx.append(j)
                vals.append((2.0 if i == j else -1.0) * np.eye(3).ravel())
        rowptr.append(len(colidx))
    rowptr, colidx, vals = np.array(rowptr), np.array(colidx), np.array(vals)
    fac = O.ilu0(nb, rowptr, colidx, vals)
    assert fac.status == 0
    for k, (_, d, l) in enumerate(rows):
        d = float(Fraction(d))
        np.testing.assert_allclose(fac.dinv[k].reshape(3, 3), np.eye(3) / d, rtol=1e-15)
        md = rowptr[k] + (1 if k > 0 else 0)
        np.testing.assert_allclose(fac.lu[md].reshape(3, 3), d * np.eye(3), rtol=1e-15)
        if l != "none":
            ml = rowptr[k + 1]  # block (k+1, k) is first in row k+1
            np.testing.assert_allclose(fac.lu[ml].reshape(3, 3), float(Fraction(l)) * np.eye(3),
                                       rtol=1e-15)


@pytest.mark.parametrize("nb", [1, 2, 5])
def test_ilu0_dense_pattern_is_exact_lu(nb):
    s = synth.random_pattern_system(nb, 0, seed=100 + nb, dense=True)
    assert s.nnzb == nb * nb
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    assert fac.status == 0
    L, U = dense_factors(s, fac)
    A = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    np.testing.assert_allclose(L @ U, A, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    # dinv is the inverse of U's diagonal blocks
    for i in range(nb):
        np.testing.assert_allclose(fac.dinv[i].reshape(3, 3) @ U[3 * i:3 * i + 3, 3 * i:3 * i + 3],
                                   np.eye(3), atol=1e-12)


@pytest.mark.parametrize("maker", [lambda: synth.chain_system(40), lambda: synth.tree_system(60, 3),
                                   lambda: synth.block_diagonal_system(25, 4)])
def test_no_fill_patterns_exact_and_one_iteration(maker):
    s = maker()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    assert fac.status == 0
    L, U = dense_factors(s, fac)
    A = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    np.testing.assert_allclose(L @ U, A, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    b = rhs(s)
    z = O.ilu_apply(s.nb, s.rowptr, s.colidx, fac, b)
    xd, st = O.dense_solve(A, b)
    assert st == 0
    np.testing.assert_allclose(z, xd, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(xd, s.x_true, rtol=1e-10, atol=1e-11)
    res = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-10, maxit=50)
    assert res.status == 0 and res.iters == 1
    assert res.relres < 1e-13
    np.testing.assert_allclose(res.x, s.x_true, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("maker", [synth.config1, lambda: synth.random_pattern_system(60, 4, 21, dense=False),
                                   lambda: synth.one_way_system(synth.random_pattern_system(60, 6, 22), 0.5, 23)])
def test_ilu0_defining_identity_on_pattern(maker):
    s = maker()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    assert fac.status == 0
    L, U = dense_factors(s, fac)
    A = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    LU = L @ U
    scale = np.abs(A).max()
    mask = np.zeros((s.nb, s.nb), dtype=bool)
    for i in range(s.nb):
        mask[i, s.colidx[s.rowptr[i]:s.rowptr[i + 1]]] = True
    big = np.kron(mask, np.ones((3, 3), dtype=bool))
    err_on = np.abs(LU - A)[big].max() / scale
    assert err_on < 1e-13
    # and it is an *incomplete* factorisation: fill outside the pattern is dropped
    assert np.abs(LU - A)[~big].max() / scale > 1e-6


def test_ilu_apply_solves_lu_system():
    s = synth.config1()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    L, U = dense_factors(s, fac)
    r = synth.uniform(synth.stream_key(3, 3), np.arange(3 * s.nb, dtype=np.uint64), -1, 1)
    z = O.ilu_apply(s.nb, s.rowptr, s.colidx, fac, r)
    assert np.linalg.norm(L @ (U @ z) - r) / np.linalg.norm(r) < 1e-13


def test_ilu0_flags_singular_pivot_row():
    s = synth.block_diagonal_system(4, 9)
    vals = s.vals.copy()
    vals[2] = np.array([1.0, 2, 3, 2, 4, 6, 0, 0, 1])  # rank-2 diagonal block at row 2
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, vals)
    assert fac.status == -(1 + 2)


def test_ilu0_f32_close_to_f64():
    s = synth.config1()
    f64 = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    f32 = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals, f32=True)
    assert f32.status == 0 and f32.lu.dtype == np.float32
    rel = np.abs(f32.lu - f64.lu).max() / np.abs(f64.lu).max()
    assert 0 < rel < 1e-5


# ---------------------------------------------------------------- BiCGStab

def test_bicgstab_converges_to_x_true_at_tight_tolerance():
    s = synth.config1()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = rhs(s)
    res = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-12, maxit=200)
    assert res.status == 0
    assert res.relres <= 1e-12 * (1 + 1e-6) * 10  # true residual near the recurrence bound
    A = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(res.x - s.x_true) / np.linalg.norm(s.x_true)
    assert err <= kappa * 1e-11


@pytest.mark.parametrize("rtol", [1e-2, 1e-4, 1e-8])
def test_bicgstab_stopping_rule(rtol):
    s = synth.config1()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = rhs(s)
    res = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=rtol, maxit=200)
    assert res.status == 0
    h = res.res_hist / res.res_hist[0]
    k = res.iters
    last = h[2 * k - 1] if np.isnan(h[2 * k]) else h[2 * k]
    assert last <= rtol
    # no earlier half or full step met the rule
    assert np.all(h[1:2 * k - 1][~np.isnan(h[1:2 * k - 1])] > rtol)
    assert res.relres <= rtol * (1 + 1e-6)


@pytest.mark.parametrize("maker", [synth.config1, lambda: synth.random_pattern_system(300, 6, 12)])
def test_bicgstab_stops_at_the_first_step_that_meets_the_rule(maker):
    """BiCGStab's path does not depend on rtol, only where it stops does.
    One run to 1e-13 gives the residual after every half and full step; for
    each step whose residual is below all earlier ones, an rtol just above it
    must stop exactly there (a half-step or a full-step exit), and both kinds
    of exit must occur among the cases."""
    s = maker()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = rhs(s)
    full = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-13, maxit=400)
    assert full.status == 0
    h = full.res_hist / full.res_hist[0]
    kinds, running = set(), np.inf
    for q in range(1, len(h)):
        if np.isnan(h[q]):
            break
        tau = h[q] * (1 + 1e-9)
        if tau < running:  # every earlier step is above tau: q is the first to meet it
            r = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=tau, maxit=400)
            k = r.iters
            stop = 2 * k - 1 if np.isnan(r.res_hist[2 * k]) else 2 * k
            assert r.status == 0 and stop == q, (q, stop)
            kinds.add(q % 2)
        running = min(running, h[q])
    assert kinds == {0, 1}


def test_bicgstab_scaling_and_zero_rhs():
    s = synth.config1()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = rhs(s)
    r1 = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-6)
    r2 = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, 4.0 * b, rtol=1e-6)
    assert r1.iters == r2.iters
    np.testing.assert_allclose(r2.x, 4.0 * r1.x, rtol=1e-12, atol=1e-14)
    r0 = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, np.zeros_like(b))
    assert r0.status == 0 and r0.iters == 0 and r0.relres == 0.0
    assert np.all(r0.x == 0.0)


def test_bicgstab_maxit_and_nonfinite():
    s = synth.config1()
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = rhs(s)
    r = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-14, maxit=1)
    assert r.status == 1 and r.iters == 1
    b2 = b.copy()
    b2[5] = np.nan
    r = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b2)
    assert r.status == -6


def test_bicgstab_matches_dense_solution_on_config2_subset():
    s = synth.random_pattern_system(80, 3, 77)
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = rhs(s)
    res = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-13, maxit=200)
    xd, _ = O.dense_solve(O.to_dense(s.nb, s.rowptr, s.colidx, s.vals), b)
    np.testing.assert_allclose(res.x, xd, rtol=1e-9, atol=1e-10)


def test_f32_preconditioner_reaches_the_same_residual():
    s = synth.config1()
    b = rhs(s)
    f32 = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals, f32=True)
    f64 = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    r32 = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, f32, b, rtol=1e-10)
    r64 = O.bicgstab(s.nb, s.rowptr, s.colidx, s.vals, f64, b, rtol=1e-10)
    assert r32.status == 0 and r32.relres <= 1e-10 * (1 + 1e-6)
    np.testing.assert_allclose(r32.x, r64.x, rtol=1e-8, atol=1e-9)


# ---------------------------------------------------------------- schedules

def grid_pattern(nx, ny, nz):
    s = synth.grid_system(nx, ny, nz, np.zeros((nz, ny, nx)))
    return s


def test_levels_closed_form_on_full_grid():
    nx, ny, nz = 6, 5, 4
    s = grid_pattern(nx, ny, nz)
    lev, n = O.levels(s.nb, s.rowptr, s.colidx)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    np.testing.assert_array_equal(lev, (i + j + k).ravel())
    assert n == nx + ny + nz - 2


def test_colours_closed_form_on_full_grid():
    nx, ny, nz = 7, 4, 3
    s = grid_pattern(nx, ny, nz)
    col, n = O.colours(s.nb, s.rowptr, s.colidx)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    np.testing.assert_array_equal(col, ((i + j + k) % 2).ravel())
    assert n == 2


def _edges(s):
    rows = np.repeat(np.arange(s.nb), np.diff(s.rowptr))
    off = rows != s.colidx
    return rows[off], s.colidx[off]


@pytest.mark.parametrize("maker", [synth.config2, lambda: synth.random_pattern_system(300, 3, 5),
                                   lambda: synth.one_way_system(synth.random_pattern_system(300, 4, 6), 0.5, 7)])
def test_schedule_sets_are_independent_and_minimal(maker):
    s = maker()
    a, b = _edges(s)
    lev, nl = O.levels(s.nb, s.rowptr, s.colidx)
    col, nc = O.colours(s.nb, s.rowptr, s.colidx)
    assert np.all(lev[a] != lev[b]) and np.all(col[a] != col[b])
    # brute-force definitions on the symmetrised graph
    nbrs = [set() for _ in range(s.nb)]
    for x, y in zip(a.tolist(), b.tolist()):
        nbrs[x].add(y)
        nbrs[y].add(x)
    for i in range(s.nb):
        earlier = [j for j in nbrs[i] if j < i]
        assert lev[i] == (1 + max(lev[j] for j in earlier) if earlier else 0)
        used = {int(col[j]) for j in earlier}
        c = 0
        while c in used:
            c += 1
        assert col[i] == c
    assert nl == lev.max() + 1 and nc == col.max() + 1


@pytest.mark.parametrize("maker", [lambda: synth.random_pattern_system(120, 4, 9),
                                   lambda: synth.random_pattern_system(200, 2, 3), synth.config1])
def test_smallest_last_colouring_brute_force(maker):
    """Smallest-last greedy colouring (Matula & Beck 1983) by its definition,
    quadratic and plain: remove a least-degree row (ties to the lowest row)
    until none is left, colour first-fit in reverse removal order; the
    colour count is at most one more than the largest degree met at a
    removal (the degeneracy bound)."""
    s = maker()
    a, b = _edges(s)
    nbrs = [set() for _ in range(s.nb)]
    for x, y in zip(a.tolist(), b.tolist()):
        nbrs[x].add(y)
        nbrs[y].add(x)
    left = set(range(s.nb))
    order, worst = [], 0
    while left:
        v = min(left, key=lambda i: (len(nbrs[i] & left), i))
        worst = max(worst, len(nbrs[v] & left))
        order.append(v)
        left.remove(v)
    expect = np.full(s.nb, -1)
    for v in reversed(order):
        used = {int(expect[u]) for u in nbrs[v] if expect[u] >= 0}
        c = 0
        while c in used:
            c += 1
        expect[v] = c
    col, n = O.colours_sl(s.nb, s.rowptr, s.colidx)
    np.testing.assert_array_equal(col, expect)
    assert n == expect.max() + 1 <= worst + 1
    assert np.all(col[a] != col[b])


def test_smallest_last_colours_a_grid_with_two_colours_and_faults_with_few():
    s = grid_pattern(6, 5, 4)
    col, n = O.colours_sl(s.nb, s.rowptr, s.colidx)
    a, b = _edges(s)
    assert n == 2 and np.all(col[a] != col[b])
    c2 = synth.config2()
    _, n_nat = O.colours(c2.nb, c2.rowptr, c2.colidx)
    _, n_sl = O.colours_sl(c2.nb, c2.rowptr, c2.colidx)
    assert n_sl <= n_nat


def _pattern_from_edges(n, edges):
    """Symmetric BSR pattern (diagonal plus both directions of each edge)."""
    rows = [{i} for i in range(n)]
    for a, b in edges:
        rows[a].add(b)
        rows[b].add(a)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colidx = np.array([c for r in rows for c in sorted(r)], dtype=np.int32)
    return rowptr, colidx


def _chromatic_number(n, edges):
    """Smallest k admitting a proper colouring, by exhaustive search."""
    for k in range(1, n + 1):
        for cols in np.ndindex(*([k] * n)):
            if all(cols[a] != cols[b] for a, b in edges):
                return k
    return n


def _is_bipartite(s):
    a, b = _edges(s)
    adj = [[] for _ in range(s.nb)]
    for x, y in zip(a, b):
        adj[x].append(y)
        adj[y].append(x)
    side = -np.ones(s.nb, dtype=np.int64)
    for r in range(s.nb):
        if side[r] >= 0:
            continue
        side[r] = 0
        stack = [r]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if side[y] < 0:
                    side[y] = 1 - side[x]
                    stack.append(y)
                elif side[y] == side[x]:
                    return False
    return True


@pytest.mark.parametrize("maker", [synth.config1, synth.config2, lambda: synth.random_pattern_system(300, 3, 5),
                                   lambda: synth.random_pattern_system(120, 4, 9), lambda: synth.tree_system(200, 3),
                                   lambda: synth.chain_system(50)])
def test_kempe_reduction_keeps_a_proper_colouring_with_no_more_colours(maker):
    s = maker()
    col, n = O.colours_kempe(s.nb, s.rowptr, s.colidx)
    _, n_sl = O.colours_sl(s.nb, s.rowptr, s.colidx)
    a, b = _edges(s)
    assert np.all(col[a] != col[b])
    assert n <= n_sl
    assert set(np.unique(col)) == set(range(n))  # classes 0..n-1, none empty
    if _is_bipartite(s) and len(a):
        # forests and unfaulted grids are bipartite; the reduction reaches 2 there
        assert n == 2


def test_kempe_reduction_reaches_two_colours_on_the_bipartite_config2_pattern():
    """C2's pattern happens to be bipartite (checked by BFS parity): greedy
    smallest-last needs 4 colours there, the Kempe exchanges reach the
    minimum, 2; C3's faults leave odd cycles and 3 colours."""
    c2 = synth.config2()
    assert _is_bipartite(c2)
    assert O.colours_sl(c2.nb, c2.rowptr, c2.colidx)[1] == 4
    assert O.colours_kempe(c2.nb, c2.rowptr, c2.colidx)[1] == 2


@pytest.mark.parametrize("seed", range(12))
def test_kempe_reduction_never_beats_the_chromatic_number(seed):
    """Brute force on tiny random graphs: the count is at least the
    chromatic number, and an odd cycle keeps 3 colours."""
    rng = np.random.default_rng(seed)
    n = 7
    edges = sorted({tuple(sorted(e)) for e in rng.integers(0, n, size=(9, 2)) if e[0] != e[1]})
    rowptr, colidx = _pattern_from_edges(n, edges)
    col, k = O.colours_kempe(n, rowptr, colidx)
    assert all(col[a] != col[b] for a, b in edges)
    assert k >= _chromatic_number(n, edges)
    cyc = [(i, (i + 1) % 5) for i in range(5)]
    rowptr, colidx = _pattern_from_edges(5, cyc)
    assert O.colours_kempe(5, rowptr, colidx)[1] == 3


def test_order_by_key_is_stable_and_complete():
    key = np.array([2, 0, 1, 0, 2, 1, 0])
    perm = O.order_by_key(key, 3)
    np.testing.assert_array_equal(perm, [1, 3, 6, 2, 5, 0, 4])


@pytest.mark.parametrize("maker", [lambda: synth.random_pattern_system(60, 90, seed=11),
                                   lambda: synth.random_pattern_system(300, 2, 13)])
@pytest.mark.parametrize("schedule", ["level", "colour", "colour_sl", "colour_kempe"])
def test_schedule_order_is_set_major_with_closed_rows_first(schedule, maker):
    """Brute force on the sets the oracle returns: each set is contiguous in
    set order; inside it the rows without a neighbour in a later set come
    first; inside each of those groups the rows with more blocks than the
    most common count come last; natural order inside each part.  The dense
    pattern mixes long and short rows in a set; the sparse one also mixes
    closed and open rows, which the check asserts, so that both rules act."""
    s = maker()
    key, n = {"level": O.levels, "colour": O.colours, "colour_sl": O.colours_sl,
              "colour_kempe": O.colours_kempe}[schedule](s.nb, s.rowptr, s.colidx)
    perm, nsets = O.schedule_perm(s.nb, s.rowptr, s.colidx, schedule)
    assert nsets == n and sorted(perm.tolist()) == list(range(s.nb))
    nbrs = [set() for _ in range(s.nb)]
    for i in range(s.nb):
        for m in range(s.rowptr[i], s.rowptr[i + 1]):
            j = int(s.colidx[m])
            if j != i:
                nbrs[i].add(j)
                nbrs[j].add(i)
    expect = []
    lens = [int(s.rowptr[i + 1] - s.rowptr[i]) for i in range(s.nb)]
    counts = {}
    for v in lens:
        counts[v] = counts.get(v, 0) + 1
    common = min(v for v in counts if counts[v] == max(counts.values()))
    mixed = 0
    for c in range(n):
        rows = [i for i in range(s.nb) if key[i] == c]
        closed = [i for i in rows if all(key[j] <= c for j in nbrs[i])]
        opened = [i for i in rows if any(key[j] > c for j in nbrs[i])]
        mixed += bool(closed) and bool(opened)
        for grp in (closed, opened):
            expect += [i for i in grp if lens[i] <= common] + [i for i in grp if lens[i] > common]
    assert perm.tolist() == expect
    assert mixed > 0 or s.nb == 60
    # a closed row has no U block in the permuted matrix
    prow, pcol, _ = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    for ip in range(s.nb):
        i = int(perm[ip])
        if all(key[j] <= key[i] for j in nbrs[i]):
            assert (pcol[prow[ip]:prow[ip + 1]] <= ip).all()


def test_order_inside_a_colour_does_not_change_the_factors():
    """Rows of one colour share no edge: the colour-major order with and
    without the closed-first rule gives the same ILU0 factors row by row
    (only the order of each row's sums may differ)."""
    s = synth.config2()
    key, n = O.colours(s.nb, s.rowptr, s.colidx)
    p1 = O.order_by_key(key, n)
    p2, _ = O.schedule_perm(s.nb, s.rowptr, s.colidx, "colour")
    assert not np.array_equal(p1, p2)
    f = []
    for perm in (p1, p2):
        prow, pcol, pval = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
        fac = O.ilu0(s.nb, prow, pcol, pval)
        assert fac.status == 0
        f.append((perm, prow, pcol, fac))
    (pa, ra, ca, fa), (pb, rb, cb, fb) = f
    ia = np.empty_like(pa)
    ia[pa] = np.arange(s.nb)
    ib = np.empty_like(pb)
    ib[pb] = np.arange(s.nb)
    np.testing.assert_allclose(fb.dinv, fa.dinv[ia[pb]], rtol=1e-12, atol=1e-14)
    for ipb in range(0, s.nb, 53):
        i = pb[ipb]
        ipa = ia[i]
        # same natural column set, mapped through each order
        cols_b = {int(pb[c]): m for m, c in zip(range(rb[ipb], rb[ipb + 1]), cb[rb[ipb]:rb[ipb + 1]])}
        for m in range(ra[ipa], ra[ipa + 1]):
            j = int(pa[ca[m]])
            mb = cols_b[j]
            np.testing.assert_allclose(fb.lu[mb], fa.lu[m], rtol=1e-12, atol=1e-13 * np.abs(fa.lu[m]).max())


def test_level_order_gives_the_natural_factors():
    s = synth.config2()
    nat = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    perm, _ = O.schedule_perm(s.nb, s.rowptr, s.colidx, "level")
    prow, pcol, pval = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    lev = O.ilu0(s.nb, prow, pcol, pval)
    assert nat.status == 0 and lev.status == 0
    # block (i', j') of the permuted factors is block (perm[i'], perm[j']) of the natural ones
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(s.nb)
    for ip in range(0, s.nb, 97):
        i = perm[ip]
        for m in range(prow[ip], prow[ip + 1]):
            j = perm[pcol[m]]
            mn = s.rowptr[i] + np.searchsorted(s.colidx[s.rowptr[i]:s.rowptr[i + 1]], j)
            np.testing.assert_allclose(lev.lu[m], nat.lu[mn], rtol=1e-12,
                                       atol=1e-13 * np.abs(nat.lu[mn]).max())
    np.testing.assert_allclose(lev.dinv, nat.dinv[perm], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("rtol", [1e-2, 1e-8])
def test_level_order_solves_along_the_natural_path(rtol):
    """Level order relabels the natural factorisation, so BiCGStab in level
    order takes the natural-order path: the same residual after every half
    and full step (to rounding of the reordered sums), the same iteration
    count, and the same x mapped back."""
    s = synth.config1()
    b = rhs(s)
    x_nat, r_nat, _, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, rtol, 200, "natural")
    x_lev, r_lev, perm, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, rtol, 200, "level")
    assert not np.array_equal(perm, np.arange(s.nb))  # the order did change
    assert r_nat.status == r_lev.status == 0 and r_nat.iters == r_lev.iters
    hn, hl = r_nat.res_hist, r_lev.res_hist
    ok = ~np.isnan(hn)
    np.testing.assert_array_equal(ok, ~np.isnan(hl))
    np.testing.assert_allclose(hl[ok], hn[ok], rtol=1e-10)
    np.testing.assert_allclose(x_lev, x_nat, rtol=1e-10, atol=1e-12)


def test_colour_order_changes_the_preconditioner_but_still_solves():
    s = synth.config2()
    b = rhs(s)
    x_nat, r_nat, _, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-6, 200, "natural")
    x_gc, r_gc, perm, nc = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-6, 200, "colour")
    assert r_nat.status == 0 and r_gc.status == 0
    assert r_gc.relres <= 1e-6 * (1 + 1e-6) and r_nat.relres <= 1e-6 * (1 + 1e-6)
    assert nc >= 2
    # the paper reports more iterations for colouring than for level scheduling
    facts = paper_facts()
    assert facts["gc_linear_iterations"] > facts["ls_linear_iterations"]
    assert r_gc.iters >= r_nat.iters


def test_permute_round_trip():
    s = synth.random_pattern_system(50, 3, 8)
    perm, _ = O.schedule_perm(s.nb, s.rowptr, s.colidx, "colour")
    prow, pcol, pval = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    A = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    PA = O.to_dense(s.nb, prow, pcol, pval)
    P = np.kron(np.eye(s.nb)[perm], np.eye(3))
    np.testing.assert_array_equal(PA, P @ A @ P.T)
    assert all(np.all(np.diff(pcol[prow[i]:prow[i + 1]]) > 0) for i in range(s.nb))


# ---------------------------------------------------------------- generator

def test_generator_matches_paper_sizes_and_is_deterministic():
    facts = paper_facts()
    s2 = synth.config2()
    assert s2.nb == int(facts["norne_active_cells"])
    s1a, s1b = synth.config1(), synth.config1()
    assert s1a.nb == 500 and s1a.nnzb == 3100
    np.testing.assert_array_equal(s1a.vals, s1b.vals)
    np.testing.assert_array_equal(s1a.x_true, s1b.x_true)
    assert np.all(np.diff(s1a.rowptr) >= 1)


def test_generator_rows_are_diagonally_dominant_up_to_noise():
    s = synth.config1()
    v = s.vals.reshape(-1, 3, 3)
    rows = np.repeat(np.arange(s.nb), np.diff(s.rowptr))
    diag = rows == s.colidx
    off_sum = np.zeros((s.nb, 3))
    for r in range(3):
        off_sum[:, r] = np.bincount(rows[~diag], weights=np.abs(v[~diag, r, :]).sum(axis=1), minlength=s.nb)
    d = v[diag]
    for r in range(3):
        assert np.all(d[:, r, r] >= off_sum[:, r] + 0.1 - 0.05)


def test_one_way_generator_drops_blocks_one_way_and_keeps_the_rest():
    """The non-symmetric stand-in: every kept block has A's value, the
    diagonal stays, some blocks lose their mirror, and a fraction near the
    requested one goes."""
    base = synth.random_pattern_system(400, 5, 31)
    s = synth.one_way_system(base, 0.4, 32)
    key = lambda sy: np.repeat(np.arange(sy.nb), np.diff(sy.rowptr)).astype(np.int64) * sy.nb + sy.colidx
    kb, ks = key(base), key(s)
    pos = np.searchsorted(kb, ks)
    np.testing.assert_array_equal(kb[pos], ks)                  # a subset of base's blocks, in row order
    np.testing.assert_array_equal(s.vals, base.vals[pos])       # with base's values
    rows = np.repeat(np.arange(s.nb), np.diff(s.rowptr))
    assert np.count_nonzero(rows == s.colidx) == s.nb           # every diagonal kept
    nb_off = base.nnzb - base.nb
    assert abs((base.nnzb - s.nnzb) / nb_off - 0.4) < 0.03
    mirrored = np.isin(s.colidx.astype(np.int64) * s.nb + rows, ks)
    assert np.count_nonzero(~mirrored) > 0.2 * (s.nnzb - s.nb)  # one-way blocks present
    np.testing.assert_array_equal(synth.one_way_system(base, 0.4, 32).colidx, s.colidx)


def test_batched_and_serving_workload_recipes():
    """The batched workload: 256 grids, every axis 5..40, 500..20,000 cells.
    The serving patterns: cells log-uniform in 5,000..250,000 (up to the
    rounding of the axes), nz no larger than nx or ny."""
    d4 = synth.config4_dims(256)
    cells = [x * y * z for x, y, z in d4]
    assert len(d4) == 256 and all(5 <= v <= 40 for d in d4 for v in d)
    assert all(500 <= c <= 20000 for c in cells) and len(set(d4)) > 200
    d5 = synth.config5_dims(32)
    c5 = np.array([x * y * z for x, y, z in d5], dtype=float)
    assert len(d5) == 32 and all(z <= x and z <= y for x, y, z in d5)
    assert 0.8 * 5000 <= c5.min() and c5.max() <= 1.25 * 250000
    # the mean of 32 uniform logs on [ln 5e3, ln 2.5e5] has a standard deviation near 0.2
    assert abs(np.log(c5).mean() - (np.log(5000) + np.log(250000)) / 2) < 0.6


def test_one_million_cell_recipe():
    """The 100^3 workload from first principles: about 5% of the cells
    inactive, every face between two active cells a connection, and
    round(1% of the active cells) extra fault connections, each joining two
    active cells that are not face neighbours, at most 3 cells apart on
    every axis.  Every connection gives two blocks, every cell one."""
    s = synth.config3()
    kji = s.geom["kji"]
    act = np.zeros(s.geom["shape"], dtype=bool)
    act[kji[:, 0], kji[:, 1], kji[:, 2]] = True
    assert abs(s.nb - 950000) < 2000  # binomial standard deviation ~218
    faces = int((act[1:] & act[:-1]).sum() + (act[:, 1:] & act[:, :-1]).sum() + (act[:, :, 1:] & act[:, :, :-1]).sum())
    nfault = int(round(0.01 * s.nb))
    assert s.nnzb == s.nb + 2 * faces + 2 * nfault
    rows = np.repeat(np.arange(s.nb), np.diff(s.rowptr))
    off = rows != s.colidx
    d = np.abs(kji[rows[off]] - kji[s.colidx[off]])
    far = d.sum(axis=1) > 1
    assert int(far.sum()) == 2 * nfault and d[far].max() <= 3
    # a stand-in for the paper's BigModel: its size and its blocks per row
    facts = paper_facts()
    assert 0.8 < s.nb / facts["bigmodel_active_cells"] < 1.2
    assert abs(s.nnzb / s.nb / facts["bigmodel_nnz_per_row"] - 1) < 0.1


def test_defaults_are_the_papers_stopping_rule():
    """The oracle's default rtol and maxit are the stopping rule the paper
    states (relative reduction 0.01, at most 200 iterations); the blocks
    are 3x3."""
    import inspect
    facts = paper_facts()
    for fn in (O.bicgstab, O.solve_system):
        sig = inspect.signature(fn).parameters
        assert sig["rtol"].default == facts["default_rtol"] and sig["maxit"].default == facts["default_maxit"], fn
    s = synth.config1()
    assert s.vals.shape[1] == facts["block_size"] ** 2 and s.x_true.size == facts["block_size"] * s.nb


# ------------------------------------------------------- block-Jacobi ILU0

def test_jacobi_pattern_keeps_exactly_the_partition_internal_blocks():
    """Brute force on the copy-index gather (Section 4.5): kept blocks are
    those with part[i] == part[j], in row order, values gathered by index."""
    s = synth.random_pattern_system(90, 4, 21)
    part = np.arange(s.nb) % 7
    jrp, jci, jv, idx = O.jacobi_pattern(s.nb, s.rowptr, s.colidx, s.vals, part)
    k = 0
    for i in range(s.nb):
        for m in range(s.rowptr[i], s.rowptr[i + 1]):
            j = s.colidx[m]
            if part[i] == part[j]:
                assert idx[k] == m and jci[k] == j
                np.testing.assert_array_equal(jv[k], s.vals[m])
                k += 1
        assert jrp[i + 1] == k
    assert k == len(idx)


def test_jacobi_with_one_partition_is_plain_ilu0():
    s = synth.config1()
    b = rhs(s)
    x0, r0, p0, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-8, 200, "colour")
    x1, r1, p1, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-8, 200, "colour",
                                   part=np.zeros(s.nb, dtype=np.int32))
    np.testing.assert_array_equal(p0, p1)
    assert r0.iters == r1.iters
    np.testing.assert_array_equal(x0, x1)


def test_jacobi_with_one_row_per_partition_is_block_diagonal_jacobi():
    """Every row its own partition: the preconditioner is block-diagonal and
    applies z_i = inv(A_ii) r_i (closed form)."""
    s = synth.config1()
    part = np.arange(s.nb, dtype=np.int32)
    jrp, jci, jv, _ = O.jacobi_pattern(s.nb, s.rowptr, s.colidx, s.vals, part)
    assert np.all(np.diff(jrp) == 1) and np.all(jci == np.arange(s.nb))
    fac = O.ilu0(s.nb, jrp, jci, jv)
    r = np.random.default_rng(3).standard_normal(3 * s.nb)
    z = O.ilu_apply(s.nb, jrp, jci, fac, r)
    for i in range(0, s.nb, 7):
        blk = jv[i].reshape(3, 3)
        np.testing.assert_allclose(z[3 * i:3 * i + 3], np.linalg.solve(blk, r[3 * i:3 * i + 3]), rtol=1e-12,
                                   atol=1e-13)


def test_jacobi_on_a_cut_chain_is_the_exact_block_inverse():
    """A chain (block-tridiagonal, no fill) cut into two partitions: each
    part's ILU0 is its exact LU, so the preconditioner is the exact inverse of
    blockdiag(A_11, A_22), compared with dense solves of the two parts."""
    s = synth.chain_system(40)
    h = 17
    part = (np.arange(s.nb) >= h).astype(np.int32)
    jrp, jci, jv, _ = O.jacobi_pattern(s.nb, s.rowptr, s.colidx, s.vals, part)
    fac = O.ilu0(s.nb, jrp, jci, jv)
    assert fac.status == 0
    r = np.random.default_rng(5).standard_normal(3 * s.nb)
    z = O.ilu_apply(s.nb, jrp, jci, fac, r)
    a = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    for lo, hi in ((0, h), (h, s.nb)):
        sl = slice(3 * lo, 3 * hi)
        np.testing.assert_allclose(z[sl], np.linalg.solve(a[sl, sl], r[sl]), rtol=1e-10, atol=1e-12)
    # and the block coupling the parts is indeed absent from the preconditioner
    assert not np.any((jci < h) & (np.repeat(np.arange(s.nb), np.diff(jrp)) >= h))


def test_partition_grid_gives_balanced_boxes():
    s = synth.config2()
    part = synth.partition_grid(s, 16)
    counts = np.bincount(part)
    assert len(counts) == 16 and counts.min() > 0
    assert counts.max() <= 2.5 * counts.min()
    kji = s.geom["kji"]
    for p in range(16):
        c = kji[part == p]
        lo, hi = c.min(axis=0), c.max(axis=0)
        # every active cell inside the part's bounding box belongs to the part
        inside = np.all((kji >= lo) & (kji <= hi), axis=1)
        assert np.all(part[inside] == p)


def test_jacobi_solve_converges_on_the_44k_cell_system():
    s = synth.config2()
    b = rhs(s)
    part = synth.partition_grid(s, 16)
    x, res, perm, nsets = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-6, 200, "level", part=part)
    assert res.status == 0 and res.relres <= 1e-6 * (1 + 1e-6)
    _, nlev_full = O.levels(s.nb, s.rowptr, s.colidx)
    assert nsets < nlev_full  # the partition cuts the dependency chains (Section 4.5)


# -------------------------------------------------- standard wells, separate

def test_separate_wells_equal_the_dense_schur_operator():
    """y = A x - sum C^T inv(D) B x against the dense matrix
    A - sum_w C_w^T inv(D_w) B_w, assembled from the blocks."""
    s = synth.config1()
    w = synth.wells(s, 3, 4)
    a = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    for k in range(w.nwells):
        Bw = np.zeros((4, 3 * s.nb))
        Cw = np.zeros((4, 3 * s.nb))
        for p in range(w.ptr[k], w.ptr[k + 1]):
            c = w.cells[p]
            Bw[:, 3 * c:3 * c + 3] += w.B[p].reshape(4, 3)
            Cw[:, 3 * c:3 * c + 3] += w.C[p].reshape(4, 3)
        a -= Cw.T @ np.linalg.inv(w.D[k].reshape(4, 4)) @ Bw
    x = np.random.default_rng(7).standard_normal(3 * s.nb)
    y = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, x)
    np.testing.assert_allclose(y, a @ x, rtol=1e-12, atol=1e-12 * np.abs(a @ x).max())


def test_separate_wells_equal_the_coupled_matrix():
    """The paper's two forms agree: adding C^T inv(D) B into A's blocks (on a
    pattern widened by every pair of a well's perforated cells) gives the
    same product as applying the wells separately."""
    s = synth.config1()
    w = synth.wells(s, 3, 4)
    blocks = {}
    for i in range(s.nb):
        for m in range(s.rowptr[i], s.rowptr[i + 1]):
            blocks[(i, int(s.colidx[m]))] = s.vals[m].reshape(3, 3).copy()
    for k in range(w.nwells):
        dinv = w.Dinv[k].reshape(4, 4)
        for p in range(w.ptr[k], w.ptr[k + 1]):
            for q in range(w.ptr[k], w.ptr[k + 1]):
                key = (int(w.cells[p]), int(w.cells[q]))
                blk = blocks.setdefault(key, np.zeros((3, 3)))
                blk -= w.C[p].reshape(4, 3).T @ dinv @ w.B[q].reshape(4, 3)
    keys = sorted(blocks)
    rowptr = np.zeros(s.nb + 1, dtype=np.int32)
    for (i, _) in keys:
        rowptr[i + 1] += 1
    rowptr = np.cumsum(rowptr).astype(np.int32)
    colidx = np.array([j for (_, j) in keys], dtype=np.int32)
    vals = np.array([blocks[k].ravel() for k in keys])
    x = np.random.default_rng(8).standard_normal(3 * s.nb)
    y_coupled = O.spmv(s.nb, rowptr, colidx, vals, x)
    y_sep = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, x)
    np.testing.assert_allclose(y_sep, y_coupled, rtol=1e-12, atol=1e-12 * np.abs(y_coupled).max())


def test_solve_with_wells_recovers_x_true():
    """b = (A - sum C^T inv(D) B) x_true; BiCGStab on that operator with the
    ILU0 of A converges, and the true residual it reports is the operator's."""
    s = synth.config2()
    w = synth.wells(s, 4, 10)
    b = O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, s.x_true)
    x, res, perm, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-10, 300, "colour", wells=w)
    assert res.status == 0 and res.relres <= 1e-10 * (1 + 1e-6)
    r = b - O.spmv_wells(s.nb, s.rowptr, s.colidx, s.vals, w, x)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - res.relres) <= 1e-3 * res.relres
    assert np.linalg.norm(x - s.x_true) <= 1e-6 * np.linalg.norm(s.x_true)


# ------------------------------------------------------------ restarted GMRES

def test_gmres_minimises_the_residual_over_the_krylov_space():
    """After j steps (no restart) GMRES's estimate equals
    min over c of ||b - A inv(M) K_j c||, computed by brute force from the
    explicit Krylov basis K_j = [b, (A inv(M)) b, ...] and a dense
    least-squares solve."""
    s = synth.random_pattern_system(20, 3, 31)
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = np.random.default_rng(4).standard_normal(3 * s.nb)
    a = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    minv = np.column_stack([O.ilu_apply(s.nb, s.rowptr, s.colidx, fac, e) for e in np.eye(3 * s.nb)])
    op = a @ minv
    for j in (1, 3, 6):
        res = O.gmres(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-300, maxit=j, restart=50)
        assert res.status == 1 and res.iters == j
        K = np.column_stack([np.linalg.matrix_power(op, q) @ b for q in range(j)])
        c, *_ = np.linalg.lstsq(op @ K, b, rcond=None)
        best = np.linalg.norm(b - op @ K @ c)
        np.testing.assert_allclose(res.res_hist[j], best, rtol=1e-8)
        # and the returned x attains it: x = inv(M) K c (the true residual of x)
        np.testing.assert_allclose(res.relres * np.linalg.norm(b), best, rtol=1e-8)


def test_gmres_with_an_exact_preconditioner_takes_one_step():
    """No-fill pattern: ILU0 is the exact LU, A inv(M) = I, one step."""
    s = synth.chain_system(60)
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    b = rhs(s)
    res = O.gmres(s.nb, s.rowptr, s.colidx, s.vals, fac, b, rtol=1e-10, maxit=50, restart=30)
    assert res.status == 0 and res.iters == 1
    np.testing.assert_allclose(res.x, s.x_true, rtol=0, atol=1e-12 * np.abs(s.x_true).max())


def test_gmres_restart_longer_than_the_solve_changes_nothing():
    s = synth.config1()
    b = rhs(s)
    x1, r1, _ = O.solve_system_gmres(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-8, 200, 60, "colour")
    x2, r2, _ = O.solve_system_gmres(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-8, 200, 100, "colour")
    assert r1.iters == r2.iters < 60
    np.testing.assert_array_equal(x1, x2)
    # a short restart still converges, the estimate tracking the true residual at the end
    x3, r3, _ = O.solve_system_gmres(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-8, 300, 5, "colour")
    assert r3.status == 0 and r3.relres <= 1e-8 * (1 + 1e-6) and r3.iters > r1.iters
    assert np.linalg.norm(x3 - s.x_true) <= 1e-6 * np.linalg.norm(s.x_true)


# ---------------------------------------------------------------- iterative ILU0, Jacobi triangular solves

def _pattern_mask(s):
    mask = np.zeros((s.nb, s.nb), dtype=bool)
    for i in range(s.nb):
        mask[i, s.colidx[s.rowptr[i]:s.rowptr[i + 1]]] = True
    return mask


def _cp_depth(s):
    """Sweeps after which the synchronous fixed-point sweeps are exact, by
    brute force over the dependency graph of the ILU0 equations: an entry
    depends on L_ik and U_kj for every k < min(i,j) in the pattern, and
    L_ij also on the pivot U_jj.  The initial guess is already exact for an
    entry with an empty sum whose pivot (for L) is exact from the start;
    every other entry is exact one sweep after its last dependency."""
    mask = _pattern_mask(s)
    depth = {}
    for i in range(s.nb):          # rows in order: every dependency is in an earlier row
        for j in np.nonzero(mask[i])[0]:
            deps = [(i, k) for k in range(min(i, j)) if mask[i, k] and mask[k, j]]
            deps += [(k, j) for k in range(min(i, j)) if mask[i, k] and mask[k, j]]
            empty_sum = len(deps) == 0
            if j < i:
                deps.append((j, j))
            worst = max((depth[d] for d in deps), default=0)
            depth[(i, j)] = 0 if empty_sum and worst == 0 else 1 + worst
    return max(depth.values())


def test_chow_patel_zero_sweeps_is_the_initial_guess():
    """No sweep leaves the initial guess L_ij = A_ij inv(A_jj), U_ij = A_ij."""
    s = synth.random_pattern_system(30, 3, 41)
    lu = np.empty((int(s.rowptr[-1]), 9))
    dinv = np.empty((s.nb, 9))
    st = O.lib().orc_ilu0_cp(s.nb, O._p(O._i32(s.rowptr), O._i32p), O._p(O._i32(s.colidx), O._i32p),
                            O._p(O._f64(s.vals), O._f64p), 0, O._p(lu, O._f64p), O._p(dinv, O._f64p))
    assert st == 0
    a = s.vals.reshape(-1, 3, 3)
    diag = [s.rowptr[i] + int(np.nonzero(s.colidx[s.rowptr[i]:s.rowptr[i + 1]] == i)[0][0]) for i in range(s.nb)]
    for i in range(s.nb):
        for m in range(s.rowptr[i], s.rowptr[i + 1]):
            j = s.colidx[m]
            want = a[m] @ np.linalg.inv(a[diag[j]]) if j < i else a[m]
            np.testing.assert_allclose(lu[m].reshape(3, 3), want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
        np.testing.assert_allclose(dinv[i].reshape(3, 3), np.linalg.inv(a[diag[i]]), rtol=1e-12)


@pytest.mark.parametrize("maker", [lambda: synth.grid_system(4, 4, 3, synth.uniform(
    synth.stream_key(5, 5), np.arange(48, dtype=np.uint64), -1, 1)),
    lambda: synth.random_pattern_system(40, 3, 43),
    lambda: synth.one_way_system(synth.random_pattern_system(40, 4, 44), 0.5, 45)])
def test_chow_patel_reaches_the_ilu0_identity_after_the_dependency_depth(maker):
    """After exactly as many sweeps as the longest dependency chain (brute
    force) the iterates satisfy (LU)_ij = A_ij on the pattern (checked with
    dense products) and equal, bit for bit, the ILU0 of Algorithm 2, which
    takes the same operations in the same order; one sweep earlier they
    do not yet."""
    s = maker()
    d = _cp_depth(s)
    assert 1 < d < s.nb
    A = O.to_dense(s.nb, s.rowptr, s.colidx, s.vals)
    big = np.kron(_pattern_mask(s), np.ones((3, 3), dtype=bool))
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals, cp_sweeps=d)
    assert fac.status == 0
    L, U = dense_factors(s, fac)
    assert np.abs(L @ U - A)[big].max() / np.abs(A).max() < 1e-14
    for i in range(s.nb):          # the kept inverse pivots are the inverses of U's diagonal blocks
        np.testing.assert_allclose(fac.dinv[i].reshape(3, 3) @ U[3 * i:3 * i + 3, 3 * i:3 * i + 3],
                                   np.eye(3), atol=1e-12)
    exact = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    np.testing.assert_array_equal(fac.lu, exact.lu)
    np.testing.assert_array_equal(fac.dinv, exact.dinv)
    early = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals, cp_sweeps=d - 1)
    assert not np.array_equal(early.lu, exact.lu)
    late = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals, cp_sweeps=d + 3)
    np.testing.assert_array_equal(late.lu, exact.lu)


def test_chow_patel_converges_geometrically_on_a_dominant_grid():
    """On the diagonally dominant reservoir-like system a few sweeps already
    bring the factors close (Chow & Patel report a handful of sweeps): the
    distance to the exact ILU0 falls geometrically, by a factor of three or
    more every two sweeps (an L entry takes its pivot from the previous
    sweep, so a correction travels L -> U -> L in two)."""
    s = synth.config1()
    exact = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    dist = []
    for t in (1, 3, 5, 7):
        fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals, cp_sweeps=t)
        assert fac.status == 0
        dist.append(np.abs(fac.lu - exact.lu).max() / np.abs(exact.lu).max())
    assert dist[0] < 0.1
    assert all(b < a / 3 for a, b in zip(dist, dist[1:])), dist


def test_chow_patel_flags_a_singular_pivot():
    s = synth.block_diagonal_system(4, 9)
    vals = s.vals.copy()
    vals[2] = np.array([1.0, 2, 3, 2, 4, 6, 0, 0, 1])
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, vals, cp_sweeps=2)
    assert fac.status == -(1 + 2)


def test_jacobi_triangular_sweeps_follow_the_error_recurrence():
    """Jacobi for L y = r (unit L) from y = r: y_t - y* = (-N)^t (r - y*) with
    N the strictly lower part; for U z = y_T from z = inv(D) y_T:
    z_t - z* = (-inv(D) S)^t (z_0 - z*) with S the strictly upper part."""
    s = synth.random_pattern_system(25, 3, 45)
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    L, U = dense_factors(s, fac)
    n = 3 * s.nb
    N = L - np.eye(n)
    D = np.zeros_like(U)
    for i in range(s.nb):
        D[3 * i:3 * i + 3, 3 * i:3 * i + 3] = U[3 * i:3 * i + 3, 3 * i:3 * i + 3]
    Dinv = np.linalg.inv(D)
    S = U - D
    r = np.random.default_rng(9).standard_normal(n)
    ystar = np.linalg.solve(L, r)
    for t in (1, 2, 5):
        yt = ystar + np.linalg.matrix_power(-N, t) @ (r - ystar)
        zstar = np.linalg.solve(U, yt)
        zt = zstar + np.linalg.matrix_power(-Dinv @ S, t) @ (Dinv @ yt - zstar)
        z = O.ilu_apply(s.nb, s.rowptr, s.colidx, fac, r, tri_sweeps=t)
        np.testing.assert_allclose(z, zt, rtol=0, atol=1e-11 * np.abs(zt).max())


def test_jacobi_triangular_sweeps_are_exact_after_the_chain_length():
    """Strictly triangular parts are nilpotent: after as many sweeps as the
    longest chain of the factor's graph the Jacobi solve is the exact one."""
    s = synth.grid_system(5, 4, 3, synth.uniform(synth.stream_key(5, 6), np.arange(60, dtype=np.uint64), -1, 1))
    fac = O.ilu0(s.nb, s.rowptr, s.colidx, s.vals)
    lev, nlev = O.levels(s.nb, s.rowptr, s.colidx)
    r = np.random.default_rng(10).standard_normal(3 * s.nb)
    exact = O.ilu_apply(s.nb, s.rowptr, s.colidx, fac, r)
    z = O.ilu_apply(s.nb, s.rowptr, s.colidx, fac, r, tri_sweeps=nlev - 1)
    np.testing.assert_allclose(z, exact, rtol=0, atol=1e-13 * np.abs(exact).max())
    z = O.ilu_apply(s.nb, s.rowptr, s.colidx, fac, r, tri_sweeps=nlev - 2)
    assert np.abs(z - exact).max() > 1e-10 * np.abs(exact).max()


def test_iterative_ilu0_with_jacobi_solves_still_solves():
    """BiCGStab with three Chow-Patel sweeps and three Jacobi sweeps per
    triangle reaches x_true, at some cost in iterations over exact ILU0
    (natural order).  Under a two-colour order every dependency chain has
    length one, so a single sweep of each is already exact."""
    s = synth.config1()
    b = rhs(s)
    x0, r0, *_ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-10, 400, "natural")
    x1, r1, *_ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-10, 400, "natural", cp_sweeps=3,
                               tri_sweeps=3)
    assert r0.status == 0 and r1.status == 0
    assert r0.iters < r1.iters <= 4 * r0.iters
    assert np.linalg.norm(x1 - s.x_true) <= 1e-7 * np.linalg.norm(s.x_true)
    x2, r2, _, nsets = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-10, 400, "colour")
    x3, r3, _, _ = O.solve_system(s.nb, s.rowptr, s.colidx, s.vals, b, 1e-10, 400, "colour", cp_sweeps=1,
                                  tri_sweeps=1)
    assert nsets == 2 and r2.iters == r3.iters
    np.testing.assert_allclose(x3, x2, rtol=0, atol=1e-12 * np.abs(x2).max())
