"""Seeded synthetic black-oil Jacobians in 3x3 block-CSR (BSR) form.

This module only *generates inputs*: a sparsity pattern, block values and a
reference solution ``x_true``.  It holds none of the solver's arithmetic (no
products with the matrix, no factorisation, no Krylov step); the right-hand
side ``b = A @ x_true`` is formed by whoever consumes the system.  It is the one
module that both the CPU oracle's tests and the GPU path import.

Why synthetic: the paper's benchmark decks (Section 5.1, Table "Selected
Benchmarks": NORNE with 44,431 active cells, NORNE refined with 355,407 and a
proprietary 1.09M-cell model) are not available, so only their sizes and
densities are mimicked.  The matrices follow the structure the paper describes
for OPM Flow (Section 2.1): one block row per active cell, 3 unknowns per cell
(bs = 3), a two-point-flux (7-point) stencil on a corner grid, blocks stored
contiguously and row-major inside each block (Section 4.1; Section 4.7,
figure "Memory layout of blocks in OPM").

Randomness comes from a counter-based generator (SplitMix64 of Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value
number ``c`` of stream ``s`` is ``mix(s + (c + 1) * 0x9E3779B97F4A7C15)``, so a
draw depends only on (seed, stream, counter) and every machine gets
bit-identical integers.  Uniforms take the top 53 bits.  Normals use the
Box-Muller transform.

Recipe (shared by every configuration):

* cells (i, j, k) on an nx x ny x nz grid, active cells numbered in natural
  order (i fastest, then j, then k);
* permeability k_x = exp(log k) per cell, k_y = k_x, k_z = 0.1 k_x;
* face transmissibility = harmonic mean 2 k_a k_b / (k_a + k_b) of the two
  cells' directional permeabilities (unit geometric factors);
* off-diagonal block A_ab = -T_ab * M_ab with M entries U(0.5, 1.5), drawn
  independently for (a, b) and (b, a), so A is non-symmetric;
* diagonal block: entry (r, r) = acc_a + S_{a,r} + 0.05 U(-1, 1) with
  acc_a ~ U(0.1, 1) and S_{a,r} = sum over the off-diagonal blocks of row a of
  the absolute entries of their row r; entries (r, c != r) = 0.05 U(-1, 1);
* x_true entries U(-1, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 2309114880

# stream identifiers (any distinct constants)
_S_PERM, _S_LAYER, _S_MASK, _S_FAULT, _S_M, _S_ACC, _S_DNOISE, _S_X, _S_DIMS, _S_SCALE, _S_WELL, _S_DROP = range(1, 13)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of one named random stream of a seed."""
    with np.errstate(over="ignore"):
        k = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        return _mix(k)[0]


def rand_u64(key: np.uint64, counters) -> np.ndarray:
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (c + np.uint64(1)) * _GOLDEN)


def uniform(key, counters, lo=0.0, hi=1.0) -> np.ndarray:
    u = (rand_u64(key, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(key, counters) -> np.ndarray:
    c = np.asarray(counters, dtype=np.uint64)
    u1 = uniform(key, c * np.uint64(2))
    u2 = uniform(key, c * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class BsrSystem:
    """A 3x3 block-CSR system.  ``vals`` has shape (nnzb, 9), row-major blocks."""

    nb: int
    rowptr: np.ndarray  # int32 [nb+1]
    colidx: np.ndarray  # int32 [nnzb]
    vals: np.ndarray    # float64 [nnzb, 9]
    x_true: np.ndarray  # float64 [nb*3]
    meta: dict = field(default_factory=dict)
    # grid systems: cell coordinates (k, j, i) of the active cells [nb, 3] and
    # the face transmissibilities per axis (0 where a face joins an inactive
    # cell); used only to partition the grid
    geom: dict | None = None

    @property
    def nnzb(self) -> int:
        return int(self.colidx.shape[0])


def _assemble(nb, conn_a, conn_b, conn_t, key_m, key_acc, key_dn, key_x):
    """Build the BSR arrays from a connection list (a < b not required)."""
    nc = conn_a.shape[0]
    # two off-diagonal blocks per connection: (a,b) uses counters 18c+0..8,
    # (b,a) uses 18c+9..17
    cidx = np.arange(nc, dtype=np.uint64)
    ctr = cidx[:, None] * np.uint64(18) + np.arange(18, dtype=np.uint64)[None, :]
    m = uniform(key_m, ctr, 0.5, 1.5)
    off_ab = -conn_t[:, None] * m[:, :9]
    off_ba = -conn_t[:, None] * m[:, 9:]
    rows_off = np.concatenate([conn_a, conn_b])
    cols_off = np.concatenate([conn_b, conn_a])
    vals_off = np.concatenate([off_ab, off_ba])

    # S_{a,r}: absolute row sums of the off-diagonal blocks, per block row
    s = np.zeros((nb, 3))
    absv = np.abs(vals_off).reshape(-1, 3, 3).sum(axis=2)
    for r in range(3):
        s[:, r] = np.bincount(rows_off, weights=absv[:, r], minlength=nb)
    acc = uniform(key_acc, np.arange(nb, dtype=np.uint64), 0.1, 1.0)
    dn = 0.05 * uniform(key_dn, np.arange(nb * 9, dtype=np.uint64), -1.0, 1.0).reshape(nb, 3, 3)
    diag = dn.copy()
    for r in range(3):
        diag[:, r, r] += acc + s[:, r]
    rows = np.concatenate([np.arange(nb, dtype=np.int64), rows_off.astype(np.int64)])
    cols = np.concatenate([np.arange(nb, dtype=np.int64), cols_off.astype(np.int64)])
    vals = np.concatenate([diag.reshape(nb, 9), vals_off])
    order = np.argsort(rows * nb + cols, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(nb + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(rows, minlength=nb))
    x_true = uniform(key_x, np.arange(nb * 3, dtype=np.uint64), -1.0, 1.0)
    return (rowptr.astype(np.int32), cols.astype(np.int32), np.ascontiguousarray(vals), x_true)


def grid_system(nx, ny, nz, logk, active=None, faults=None, seed=SEED_BASE, meta=None) -> BsrSystem:
    """Jacobian-shaped BSR system on a grid.

    ``logk``: natural log of k_x per grid cell (shape nz, ny, nx).
    ``active``: boolean mask (nz, ny, nx) or None for all active.
    ``faults``: optional (a, b, t) arrays of extra connections between active
    cell numbers with their transmissibilities.
    """
    shape = (nz, ny, nx)
    if active is None:
        active = np.ones(shape, dtype=bool)
    active = np.asarray(active, dtype=bool)
    flat_active = active.ravel()
    idx = np.full(flat_active.shape[0], -1, dtype=np.int64)
    nb = int(flat_active.sum())
    idx[flat_active] = np.arange(nb)
    idx3 = idx.reshape(shape)
    kx = np.exp(np.asarray(logk, dtype=np.float64)).reshape(shape)
    kz = 0.1 * kx
    conn_a, conn_b, conn_t = [], [], []
    tface = {}
    for axis, kk in ((2, kx), (1, kx), (0, kz)):
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[axis] = slice(0, shape[axis] - 1)
        sl_hi[axis] = slice(1, shape[axis])
        a = idx3[tuple(sl_lo)].ravel()
        b = idx3[tuple(sl_hi)].ravel()
        ka = kk[tuple(sl_lo)].ravel()
        kb = kk[tuple(sl_hi)].ravel()
        ok = (a >= 0) & (b >= 0)
        conn_a.append(a[ok])
        conn_b.append(b[ok])
        conn_t.append(2.0 * ka[ok] * kb[ok] / (ka[ok] + kb[ok]))
        tf = np.where(ok, 2.0 * ka * kb / (ka + kb), 0.0)
        fshape = list(shape)
        fshape[axis] -= 1
        tface[axis] = tf.reshape(fshape)
    if faults is not None:
        fa, fb, ft = faults
        conn_a.append(np.asarray(fa, dtype=np.int64))
        conn_b.append(np.asarray(fb, dtype=np.int64))
        conn_t.append(np.asarray(ft, dtype=np.float64))
    ca = np.concatenate(conn_a)
    cb = np.concatenate(conn_b)
    ct = np.concatenate(conn_t)
    rowptr, colidx, vals, x_true = _assemble(
        nb, ca, cb, ct, stream_key(seed, _S_M), stream_key(seed, _S_ACC),
        stream_key(seed, _S_DNOISE), stream_key(seed, _S_X))
    md = {"grid": [nx, ny, nz], "seed": seed, "n_connections": int(ca.shape[0])}
    if meta:
        md.update(meta)
    kk, jj, ii = np.nonzero(active)
    geom = {"shape": shape, "kji": np.stack([kk, jj, ii], axis=1).astype(np.int32), "tface": tface}
    return BsrSystem(nb, rowptr, colidx, vals, x_true, md, geom)


def _lognormal_field(seed, shape, sigma):
    n = int(np.prod(shape))
    return sigma * normal(stream_key(seed, _S_PERM), np.arange(n, dtype=np.uint64)).reshape(shape)


def config_seed(config_id: int, system_index: int = 0) -> int:
    return SEED_BASE + config_id * 1000 + system_index


# ---------------------------------------------------------------------------
# The five workload configurations
# ---------------------------------------------------------------------------

def config1(seed=None) -> BsrSystem:
    """10 x 10 x 5 grid, all 500 cells active, sigma = 1, natural ordering."""
    seed = config_seed(1) if seed is None else seed
    shape = (5, 10, 10)
    return grid_system(10, 10, 5, _lognormal_field(seed, shape, 1.0), seed=seed,
                       meta={"config": "C1 10x10x5"})


def _grow_region(shape, target, key):
    """Seeded connected region growth: start at a random cell, then repeatedly
    activate a uniformly chosen frontier cell until ``target`` cells are active."""
    nz, ny, nx = shape
    ncell = nx * ny * nz
    draws = uniform(key, np.arange(target + 1, dtype=np.uint64))
    active = np.zeros(ncell, dtype=bool)
    in_front = np.zeros(ncell, dtype=bool)
    start = min(int(draws[0] * ncell), ncell - 1)
    frontier = [start]
    in_front[start] = True
    count = 0
    t = 1
    while count < target:
        pick = min(int(draws[t] * len(frontier)), len(frontier) - 1)
        t += 1
        g = frontier[pick]
        frontier[pick] = frontier[-1]
        frontier.pop()
        active[g] = True
        count += 1
        i = g % nx
        j = (g // nx) % ny
        k = g // (nx * ny)
        for di, dj, dk in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
            ii, jj, kk = i + di, j + dj, k + dk
            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                h = ii + nx * (jj + ny * kk)
                if not active[h] and not in_front[h]:
                    in_front[h] = True
                    frontier.append(h)
    return active.reshape(shape)


NORNE_ACTIVE_CELLS = 44431


def config2(seed=None) -> BsrSystem:
    """46 x 112 x 22 grid with a connected active region of exactly 44,431 cells
    (the NORNE active-cell count), layered lognormal permeability."""
    seed = config_seed(2) if seed is None else seed
    nx, ny, nz = 46, 112, 22
    shape = (nz, ny, nx)
    active = _grow_region(shape, NORNE_ACTIVE_CELLS, stream_key(seed, _S_MASK))
    layer = 1.5 * normal(stream_key(seed, _S_LAYER), np.arange(nz, dtype=np.uint64))
    noise = 0.25 * normal(stream_key(seed, _S_PERM), np.arange(nx * ny * nz, dtype=np.uint64))
    logk = layer[:, None, None] + noise.reshape(shape)
    return grid_system(nx, ny, nz, logk, active=active, seed=seed,
                       meta={"config": "C2 46x112x22 NORNE-sized"})


def _faults(shape, active, logk, nfault, key_f):
    """Extra symmetric connections between an active cell and an active
    non-neighbour at offset within +-3 in each axis, T = harmonic T * U(0.01,1)."""
    nz, ny, nx = shape
    flat_active = active.ravel()
    act_cells = np.flatnonzero(flat_active)
    idx = np.full(flat_active.shape[0], -1, dtype=np.int64)
    idx[act_cells] = np.arange(act_cells.shape[0])
    kx = np.exp(logk.ravel())
    seen = set()
    fa, fb, ft = [], [], []
    batch = max(4 * nfault, 1024)
    t0 = 0
    while len(fa) < nfault:
        ctr = (np.arange(t0, t0 + batch, dtype=np.uint64)[:, None] * np.uint64(5)
               + np.arange(5, dtype=np.uint64)[None, :])
        u = uniform(key_f, ctr)
        t0 += batch
        ca = np.minimum((u[:, 0] * act_cells.shape[0]).astype(np.int64), act_cells.shape[0] - 1)
        off = np.minimum((u[:, 1:4] * 7).astype(np.int64), 6) - 3
        for r in range(batch):
            g = int(act_cells[ca[r]])
            i, j, k = g % nx, (g // nx) % ny, g // (nx * ny)
            di, dj, dk = int(off[r, 0]), int(off[r, 1]), int(off[r, 2])
            if abs(di) + abs(dj) + abs(dk) <= 1:
                continue
            ii, jj, kk = i + di, j + dj, k + dk
            if not (0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz):
                continue
            h = ii + nx * (jj + ny * kk)
            if not flat_active[h]:
                continue
            a, b = int(idx[g]), int(idx[h])
            key = (min(a, b), max(a, b))
            if key in seen:
                continue
            seen.add(key)
            th = 2.0 * kx[g] * kx[h] / (kx[g] + kx[h])
            fa.append(key[0])
            fb.append(key[1])
            ft.append(th * (0.01 + 0.99 * float(u[r, 4])))
            if len(fa) == nfault:
                break
    return np.array(fa, dtype=np.int64), np.array(fb, dtype=np.int64), np.array(ft)


def config3(n=100, seed=None) -> BsrSystem:
    """n^3 grid (100^3 by default), each cell inactive with probability 0.05,
    plus round(0.01 * active) fault connections, lognormal sigma = 2."""
    seed = config_seed(3) if seed is None else seed
    shape = (n, n, n)
    ncell = n ** 3
    active = (uniform(stream_key(seed, _S_MASK), np.arange(ncell, dtype=np.uint64)) >= 0.05).reshape(shape)
    logk = _lognormal_field(seed, shape, 2.0)
    nact = int(active.sum())
    nfault = int(round(0.01 * nact))
    faults = _faults(shape, active, logk, nfault, stream_key(seed, _S_FAULT))
    return grid_system(n, n, n, logk, active=active, faults=faults, seed=seed,
                       meta={"config": f"C3 {n}^3 faulted", "n_faults": nfault})


def config4_dims(nsys=256, seed=None):
    """Grid dimensions of the batched workload: nx, ny, nz ~ U{5..40},
    rejection-sampled to 500 <= cells <= 20,000."""
    seed = config_seed(4) if seed is None else seed
    key = stream_key(seed, _S_DIMS)
    dims = []
    t = 0
    while len(dims) < nsys:
        u = uniform(key, np.arange(3 * t, 3 * t + 3, dtype=np.uint64))
        t += 1
        d = [5 + min(int(v * 36), 35) for v in u]
        c = d[0] * d[1] * d[2]
        if 500 <= c <= 20000:
            dims.append(tuple(d))
    return dims


def config4_system(s, dims, seed=None) -> BsrSystem:
    """System s of the batched workload, given config4_dims(nsys, seed):
    all active, sigma = 1, its own seed."""
    seed = config_seed(4) if seed is None else seed
    nx, ny, nz = dims[s]
    ss = seed + 1 + s
    return grid_system(nx, ny, nz, _lognormal_field(ss, (nz, ny, nx), 1.0), seed=ss,
                       meta={"config": f"C4 system {s}"})


def config4(nsys=256, seed=None):
    """256 independent all-active systems of uneven size, sigma = 1."""
    dims = config4_dims(nsys, seed)
    return [config4_system(s, dims, seed) for s in range(nsys)]


def config5_dims(npat=32, seed=None):
    """Grid dimensions of the serving patterns: cells log-uniform in
    [5,000, 250,000], nz <= nx, ny."""
    seed = config_seed(5) if seed is None else seed
    key = stream_key(seed, _S_DIMS)
    dims = []
    for p in range(npat):
        u = uniform(key, np.arange(4 * p, 4 * p + 4, dtype=np.uint64))
        cells = math.exp(math.log(5000.0) + u[0] * (math.log(250000.0) - math.log(5000.0)))
        nz = max(2, int(round(cells ** (1.0 / 3.0) * (0.4 + 0.6 * u[1]))))
        rest = cells / nz
        nx = max(nz, int(round(math.sqrt(rest) * (0.8 + 0.45 * u[2]))))
        ny = max(nz, int(round(rest / nx)))
        dims.append((nx, ny, nz))
    return dims


def config5_pattern(p, seed=None) -> BsrSystem:
    seed = config_seed(5) if seed is None else seed
    nx, ny, nz = config5_dims(seed=seed)[p]
    ss = seed + 1 + p
    return grid_system(nx, ny, nz, _lognormal_field(ss, (nz, ny, nx), 1.0), seed=ss,
                       meta={"config": f"C5 pattern {p}"})


def newton_update(base: BsrSystem, request: int, seed=None):
    """A Newton-style value update of a base system: every block scaled by one
    U(0.9, 1.1) factor, and a fresh x_true.  Returns (vals, x_true)."""
    seed = config_seed(5) if seed is None else seed
    key = stream_key(seed * 7919 + request, _S_SCALE)
    f = uniform(key, np.arange(base.nnzb, dtype=np.uint64), 0.9, 1.1)
    vals = base.vals * f[:, None]
    x_true = uniform(stream_key(seed * 7919 + request, _S_X), np.arange(base.nb * 3, dtype=np.uint64), -1.0, 1.0)
    return vals, x_true


def chain_system(nb, seed=SEED_BASE + 17) -> BsrSystem:
    """1-D chain nb x 1 x 1: block tridiagonal, a no-fill pattern."""
    return grid_system(nb, 1, 1, _lognormal_field(seed, (1, 1, nb), 1.0), seed=seed,
                       meta={"config": f"chain {nb}"})


def random_pattern_system(nb, extra_per_row, seed, dense=False) -> BsrSystem:
    """Random pattern with diagonal dominance built like the grid recipe.
    ``dense=True`` gives every block present (all pairs connected)."""
    key = stream_key(seed, _S_FAULT)
    if dense:
        a, b = np.triu_indices(nb, 1)
    else:
        m = nb * extra_per_row
        u = uniform(key, np.arange(2 * m, dtype=np.uint64)).reshape(m, 2)
        a = np.minimum((u[:, 0] * nb).astype(np.int64), nb - 1)
        b = np.minimum((u[:, 1] * nb).astype(np.int64), nb - 1)
        ok = a != b
        a, b = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        pairs = np.unique(a * nb + b)
        a, b = pairs // nb, pairs % nb
    t = uniform(stream_key(seed, _S_PERM), np.arange(a.shape[0], dtype=np.uint64), 0.1, 2.0)
    rowptr, colidx, vals, x_true = _assemble(
        nb, a.astype(np.int64), b.astype(np.int64), t, stream_key(seed, _S_M),
        stream_key(seed, _S_ACC), stream_key(seed, _S_DNOISE), stream_key(seed, _S_X))
    return BsrSystem(nb, rowptr, colidx, vals, x_true, {"config": f"random nb={nb}", "seed": seed})


def one_way_system(base: BsrSystem, frac, seed) -> BsrSystem:
    """base with a seeded fraction of its off-diagonal blocks removed, each
    removal one way only (block (a, b) goes while (b, a) may stay): a
    non-symmetric pattern.  Only off-diagonal blocks go, so every row stays
    diagonally dominant; x_true is kept."""
    u = uniform(stream_key(seed, _S_DROP), np.arange(base.nnzb, dtype=np.uint64))
    rows = np.repeat(np.arange(base.nb), np.diff(base.rowptr))
    keep = (rows == base.colidx) | (u >= frac)
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=base.nb))]).astype(np.int32)
    meta = dict(base.meta, one_way_drop=frac, drop_seed=seed)
    return BsrSystem(base.nb, rowptr, base.colidx[keep].copy(), base.vals[keep].copy(), base.x_true.copy(), meta)


def tree_system(nb, seed) -> BsrSystem:
    """Random tree pattern, each node i < nb-1 joined to one random later node
    (its parent).  Every node then has at most one neighbour after it, so
    eliminating in natural order creates no fill: a no-fill pattern for ILU0."""
    key = stream_key(seed, _S_FAULT)
    u = uniform(key, np.arange(nb, dtype=np.uint64))
    a = np.arange(0, nb - 1, dtype=np.int64)
    span = nb - 1 - a
    b = a + 1 + np.minimum((u[:-1] * span).astype(np.int64), span - 1)
    t = uniform(stream_key(seed, _S_PERM), np.arange(nb - 1, dtype=np.uint64), 0.1, 2.0)
    rowptr, colidx, vals, x_true = _assemble(
        nb, a, b, t, stream_key(seed, _S_M), stream_key(seed, _S_ACC),
        stream_key(seed, _S_DNOISE), stream_key(seed, _S_X))
    return BsrSystem(nb, rowptr, colidx, vals, x_true, {"config": f"tree nb={nb}", "seed": seed})


def block_diagonal_system(nb, seed) -> BsrSystem:
    """Only diagonal blocks: ILU0 is exact and trivially no-fill."""
    e = np.zeros(0, dtype=np.int64)
    rowptr, colidx, vals, x_true = _assemble(
        nb, e, e, np.zeros(0), stream_key(seed, _S_M), stream_key(seed, _S_ACC),
        stream_key(seed, _S_DNOISE), stream_key(seed, _S_X))
    return BsrSystem(nb, rowptr, colidx, vals, x_true, {"config": f"blockdiag nb={nb}", "seed": seed})


def partition_grid(system: BsrSystem, nparts: int) -> np.ndarray:
    """Partition of a grid system's cells into nparts connected boxes,
    weighted by transmissibility (the input the block-Jacobi preconditioner
    of the paper's Section 4.5 takes from the simulator's partitioner):
    recursive bisection; each cut is the grid plane, among those within 5%
    of the balanced position (by active cells), whose faces carry the least
    total transmissibility inside the box (ties to the balanced position,
    then the lower plane), across the box's longest side (ties: x, y, z).
    Returns part[nb] with labels 0..nparts-1."""
    g = system.geom
    if g is None:
        raise ValueError("partition_grid needs a grid system")
    kji = g["kji"]
    part = np.zeros(system.nb, dtype=np.int32)

    def rec(lo, hi, cells, p0, npart):
        if npart <= 1 or cells.size == 0:
            part[cells] = p0
            return
        n1 = npart // 2
        ext = [hi[a] - lo[a] for a in range(3)]
        axis = max((2, 1, 0), key=lambda a: ext[a])  # longest side, ties to x then y then z
        if ext[axis] < 2:
            part[cells] = p0
            return
        coord = kji[cells, axis] - lo[axis]
        layer = np.bincount(coord, minlength=ext[axis])
        cum = np.cumsum(layer)[:-1]  # cells at or below plane c (cut after layer c)
        target = cells.size * n1 / npart
        dev = np.abs(cum - target)
        cand = np.flatnonzero(dev <= max(0.05 * cells.size, dev.min()))
        tf = g["tface"][axis]
        other = [a for a in range(3) if a != axis]
        costs = []
        for c in cand:
            sl = [slice(None)] * 3
            sl[axis] = lo[axis] + c
            for a in other:
                sl[a] = slice(lo[a], hi[a])
            costs.append(float(tf[tuple(sl)].sum()))
        best = min(range(len(cand)), key=lambda q: (costs[q], dev[cand[q]], cand[q]))
        cut = lo[axis] + int(cand[best])
        low = kji[cells, axis] <= cut
        hi1 = list(hi)
        hi1[axis] = cut + 1
        lo2 = list(lo)
        lo2[axis] = cut + 1
        rec(lo, hi1, cells[low], p0, n1)
        rec(lo2, hi, cells[~low], p0 + n1, npart - n1)

    rec([0, 0, 0], list(g["shape"]), np.arange(system.nb), 0, int(nparts))
    return part


@dataclass
class Wells:
    """Standard wells in the separate form of Section 4.6: per well a 4x4
    block D (and its inverse, which the simulator hands over instead of D),
    and one row of 4x3 blocks B and C with a block for every perforated cell.
    Perforations are grouped by well: well w owns perforations
    ptr[w]..ptr[w+1]-1, perforating cells[p] (natural numbering)."""

    ptr: np.ndarray    # int32 [nwells+1]
    cells: np.ndarray  # int32 [nperf]
    B: np.ndarray      # float64 [nperf, 12], 4x3 row-major
    C: np.ndarray      # float64 [nperf, 12], 4x3 row-major
    D: np.ndarray      # float64 [nwells, 16], 4x4 row-major
    Dinv: np.ndarray   # float64 [nwells, 16]

    @property
    def nwells(self) -> int:
        return int(self.ptr.shape[0] - 1)


def wells(system: BsrSystem, nwells: int, layers: int, seed=SEED_BASE + 101, scale=0.1) -> Wells:
    """Vertical wells on a grid system: nwells distinct (i, j) columns drawn
    uniformly; each perforates the active cells of up to `layers` consecutive
    layers starting at a drawn depth.  Well index WI of a perforation:
    scale x the mean face transmissibility of its cell; B and C entries
    -WI x U(0.5, 1.5); D = (sum of the well's WI) x (U(1, 2) I + 0.05 U(-1, 1))
    so that C^T D^-1 B stays small against the cell couplings."""
    g = system.geom
    if g is None:
        raise ValueError("wells need a grid system")
    nz, ny, nx = g["shape"]
    kji = g["kji"]
    cell_of = -np.ones(nz * ny * nx, dtype=np.int64)
    cell_of[(kji[:, 0].astype(np.int64) * ny + kji[:, 1]) * nx + kji[:, 2]] = np.arange(system.nb)
    key = stream_key(seed, _S_WELL)
    # mean face transmissibility per cell (faces of the cell present in the grid)
    tsum = np.zeros((nz, ny, nx))
    tcnt = np.zeros((nz, ny, nx))
    for axis, tf in g["tface"].items():
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, g["shape"][axis] - 1)
        hi[axis] = slice(1, g["shape"][axis])
        for sl in (lo, hi):
            tsum[tuple(sl)] += tf
            tcnt[tuple(sl)] += tf > 0
    tmean = np.where(tcnt > 0, tsum / np.maximum(tcnt, 1), 1.0)
    # columns drawn until nwells distinct ones perforate at least one active cell
    ptr, cells, wi, used = [0], [], [], set()
    u = uniform(key, np.arange(3 * 64 * (nwells + 1), dtype=np.uint64))
    q = 0
    while len(ptr) - 1 < nwells and q + 2 < u.shape[0]:
        i, j = min(int(u[q] * nx), nx - 1), min(int(u[q + 1] * ny), ny - 1)
        top = min(int(u[q + 2] * max(nz - layers, 1)), max(nz - layers, 0))
        q += 3
        if (i, j) in used:
            continue
        perf = [(k, int(cell_of[(k * ny + j) * nx + i])) for k in range(top, min(top + layers, nz))]
        perf = [(k, c) for (k, c) in perf if c >= 0]
        if not perf:
            continue
        used.add((i, j))
        for k, cid in perf:
            cells.append(cid)
            wi.append(scale * tmean[k, j, i])
        ptr.append(len(cells))
    ptr = np.asarray(ptr, dtype=np.int32)
    cells = np.asarray(cells, dtype=np.int32)
    wi = np.asarray(wi)
    nperf = cells.shape[0]
    ctr = np.arange(24 * nperf, dtype=np.uint64) + np.uint64(1 << 20)
    m = uniform(key, ctr, 0.5, 1.5).reshape(nperf, 24)
    B = -wi[:, None] * m[:, :12]
    C = -wi[:, None] * m[:, 12:]
    nw = ptr.shape[0] - 1
    dd = uniform(key, np.arange(4 * nw, dtype=np.uint64) + np.uint64(1 << 24), 1.0, 2.0).reshape(nw, 4)
    dn = 0.05 * uniform(key, np.arange(16 * nw, dtype=np.uint64) + np.uint64(1 << 26), -1.0, 1.0).reshape(nw, 4, 4)
    wsum = np.array([wi[ptr[w]:ptr[w + 1]].sum() for w in range(nw)])
    D = wsum[:, None, None] * (dn + dd[:, :, None] * np.eye(4)[None])
    Dinv = np.linalg.inv(D)
    return Wells(ptr, cells, np.ascontiguousarray(B), np.ascontiguousarray(C),
                 np.ascontiguousarray(D.reshape(nw, 16)), np.ascontiguousarray(Dinv.reshape(nw, 16)))
