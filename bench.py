#!/usr/bin/env python
"""ILU0-BiCGStab solves/s on the 1M-cell synthetic black-oil Jacobian (GB300).

One step = one Newton-step linear solve as the paper's OPM Flow integration
performs it: the new matrix values are permuted into the schedule order and
factorised (ILU0), then BiCGStab runs to a relative residual reduction of
1e-3 (the workload's rtol) and the true residual is computed.  The matrix is
the seeded 100^3 grid with a 5% inactive mask and 1% fault connections
(949,871 cells, 6.33M 3x3 blocks), b = A x_true formed on the GPU with the
library's own SpMV.  Inputs (456 MB of values) are larger than L2.

`value` is device-timed with the inputs resident in HBM; `without_refactor`
times the same solve on the step's factors, without the refactorisation;
`product_reuse_off` the same step with every BiCGStab product walking all of
A.
`e2e` makes the same
calls from pinned host buffers: each step copies the values and b in and
reads x back.  It is measured one step at a time, and again as
`e2e.overlapped`, with two handles on two streams used alternately so that a
step's copies overlap the other handle's kernels; each is the median of three
timed blocks of steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank solves its own replica (the single-system
path does not shard); value = solves of all ranks / the slowest rank's time.
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on the same system: the paper publishes no runnable code.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ILU0-BiCGStab solves/s & HBM roofline frac; FP32-ILU vs FP64; p50/p99 latency"
UNIT = "solves/s"
RTOL = 1e-3


def workload(grid, nb, nnzb):
    """The workload's name: the grid it was generated on and its actual sizes
    (the default 100^3 grid gives the 949,871-cell, 6,328,435-block system)."""
    name = "C3: " if grid == 100 else ""
    return (f"{name}{grid}^3 grid, 5% inactive cells, 1% fault connections, lognormal perm sigma=2; "
            f"{nb:,} cells, {nnzb:,} 3x3 blocks; per step: value permutation + ILU0 factorisation + "
            f"BiCGStab to rtol 1e-3 + true residual")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--schedule", default="auto")
    p.add_argument("--grid", type=int, default=100, help="grid edge (100 = the 1M-cell workload)")
    p.add_argument("--no-autotune", action="store_true", help="batched leg: AUTO options instead of the autotuner")
    p.add_argument("--no-jacobi", action="store_true", help="skip the block-Jacobi ILU0 leg")
    p.add_argument("--no-wells", action="store_true", help="skip the standard-wells leg")
    p.add_argument("--no-gmres", action="store_true", help="skip the restarted-GMRES leg")
    p.add_argument("--no-iterative", action="store_true",
                   help="skip the iterative-ILU0 / Jacobi-triangular-solve leg")
    p.add_argument("--wells", type=int, default=5, help="standard wells of the wells leg")
    p.add_argument("--partitions", type=int, default=150, help="block-Jacobi partitions")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-small", action="store_true", help="skip the C1 / C2 (L2-resident) leg")
    p.add_argument("--no-tight", action="store_true", help="skip the rtol 1e-6 leg")
    p.add_argument("--no-product-reuse", action="store_true",
                   help="FP64 products walk all of A (opm_options.product_reuse = -1)")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--batch-systems", type=int, default=256)
    p.add_argument("--patterns", type=int, default=32)
    p.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    p.add_argument("--serve-s", type=float, default=60.0, help="serving: measured seconds")
    p.add_argument("--serve-warm-s", type=float, default=20.0)
    p.add_argument("--hbm-budget-gb", type=float, default=8.0)
    p.add_argument("--class-size", type=int, default=8, help="serving: patterns per size class")
    p.add_argument("--lanes-per-class", type=int, default=2, help="serving: lanes per size class")
    p.add_argument("--sat-requests", type=int, default=4000, help="serving: requests of the saturating run")
    p.add_argument("--bound-budget-gb", type=float, default=2.0, help="serving: budget of the bound run")
    p.add_argument("--bound-s", type=float, default=10.0, help="serving: seconds of the bound run")
    p.add_argument("--ref-budget-s", type=float, default=90.0,
                   help="reference arm: seconds the timed oracle steps may take")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:  # first sample before timing starts
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def product_terms(info):
    """What a BiCGStab product after an application reads beyond a plain
    matrix pass (opm_options.product_reuse, reported by opm_get_info):
    (blocks of A it walks, rows that add one 3-vector -- p_i where the row
    has no block left of its diagonal, the backward sweep's upper sum where
    the row reuses it -- rows whose upper sum the backward sweep stores).
    Without the reuse: (nnzb, 0, 0)."""
    nprod = getattr(info, "nnzb_product", info.nnzb)
    if nprod >= info.nnzb:
        return info.nnzb, 0, 0
    return nprod, info.rows_identity + info.rows_reuse, info.rows_reuse


class PlainInfo:
    """opm_info seen without the product reuse: every product walks all of A."""

    def __init__(self, info):
        self._info = info
        self.nnzb_product, self.rows_identity, self.rows_reuse = info.nnzb, 0, 0

    def __getattr__(self, k):
        return getattr(self._info, k)


def product_bytes(info) -> int:
    """One product's matrix bytes: 76 per walked block (9 values, a column
    index), A's row pointers; with the reuse also the per-row walk length
    (4), the per-slice row classes (8) and the added 3-vectors (24 each)."""
    n = info.nb
    nprod, extra, _ = product_terms(info)
    nbytes = 76 * nprod + 4 * (n + 1)
    if nprod < info.nnzb:
        nbytes += 4 * n + 8 * ((n + 31) // 32) + 24 * extra
    return nbytes


def algorithmic_apply_bytes(info, fp32: bool) -> int:
    """Bytes one preconditioner application must move at least: every factor
    block once (L, U and the inverted diagonal, 9 values each), L's and U's
    column indices and row pointers, and the vectors: r, p, v read, p and z
    written, the intermediate y written and read back; with the product
    reuse, the row classes (8 per slice) and the stored upper sums (24 per
    reusing row)."""
    n, nnzb = info.nb, info.nnzb
    val = 4 if fp32 else 8
    factors = 9 * val * nnzb + 4 * (nnzb - n) + 2 * 4 * (n + 1)
    vectors = 5 * 24 * n + 2 * 3 * val * n
    nprod, _, stored = product_terms(info)
    if nprod < nnzb:
        vectors += 8 * ((n + 31) // 32) + 24 * stored
    return factors + vectors


def jacobi_apply_work(info, sweeps: int, fp32: bool):
    """Algorithmic work of one preconditioner application by Jacobi sweeps
    (T = sweeps per triangle): the right-hand side (r, v and p read, p
    written; 3.5 vector passes on average over the two BiCGStab
    applications), T forward sweeps (L's blocks and columns, the row
    pointers, the right-hand side, the gathered previous iterate and the new
    one), z_0 = inv(U_ii) y_T (Dinv read, z_0 written), T backward sweeps
    (U's blocks and columns, the row pointers, y_T, the gathered previous z,
    Dinv and the new z).  Returns (bytes, FP64 FMAs)."""
    n, nl, nu = info.nb, info.nnzb_lower, info.nnzb_upper
    val = 4 if fp32 else 8
    blk, vec, d = 9 * val + 4, 3 * val, 9 * val
    nbytes = 3.5 * 24 * n + sweeps * (blk * nl + 4 * n + 24 * n + 2 * vec * n) + (d + 24) * n \
        + sweeps * (blk * nu + 4 * n + vec * n + 2 * 24 * n + d * n)
    fma = 4.5 * n + (0 if fp32 else 9 * sweeps * (nl + nu) + 9 * n * (sweeps + 1))
    return int(nbytes), int(fma)


# FP64 FMA peak of the GB300: 2 FP64 lanes per SM per clock (the FP64 pipe's
# issue rate) x 152 SMs x 2.07 GHz maximum SM clock = 629 G FMA/s, i.e.
# 1.259 TFLOP/s (the nominal 1.25 TFLOP/s FP64 of the part).
FP64_FMA_PEAK = 2 * 152 * 2.07e9


def iteration_work(info, fp32: bool):
    """Algorithmic work of one BiCGStab + ILU0 iteration: HBM bytes (two
    products, two factor passes, 27 fused vector passes of 24 n bytes) and
    FP64 FMAs (two products of 9 per walked block; two preconditioner
    applications of 9 per factor block when the factors are FP64; the dot
    products, right-hand sides and vector updates: 36 per block row).  A
    product walks all of A, or with the reuse only the blocks of
    product_terms (product_bytes)."""
    n, nnzb = info.nb, info.nnzb
    nprod, _, stored = product_terms(info)
    factor = (40 if fp32 else 76) * nnzb + 4 * n
    if nprod < nnzb:
        factor += 8 * ((n + 31) // 32) + 24 * stored
    nbytes = 2 * (product_bytes(info) - 4) + 2 * factor + 27 * 24 * n
    fma = 18 * nprod + (0 if fp32 else 18 * nnzb) + 36 * n
    return nbytes, fma


def factor_work(info, fp32: bool):
    """Algorithmic work of one refactorisation with the value permutation
    fused (Algorithm 2 with Algorithm 3's index copy).  Bytes: the caller's
    blocks read once through their gather index (72 + 4 per block); the
    permuted copy of A written (72 per block); every factor slot written
    once (9 values per kept block, with its 8-byte slot location); per L
    block its column and update-list pointer (8) and one gathered inverse
    pivot (9 values); per update product its two slots (16) and one gathered
    U block (9 values); the row pointers of A and L.  FP64 FMAs (FP64
    factors; with FP32 factors the arithmetic is FP32): 27 per L block (the
    product with the inverse pivot), 27 per update product, about 30 per
    3x3 pivot inverse."""
    n, nnzb, nl, nu = info.nb, info.nnzb, info.nnzb_lower, info.nupdates
    val = 4 if fp32 else 8
    kept = nl + info.nnzb_upper + n
    nbytes = 76 * nnzb + 72 * nnzb + (9 * val + 8) * kept + (8 + 9 * val) * nl + (16 + 9 * val) * nu \
        + 2 * 4 * (n + 1)
    fma = 0 if fp32 else 27 * nl + 27 * nu + 30 * n
    return int(nbytes), int(fma)


def kernel_work(info, fp32: bool):
    """Algorithmic HBM bytes and FP64 FMAs per launch of the other kernel
    groups.  A matrix pass is 76 bytes per block (9 values and a column
    index) plus the row pointers; vectors are 24 bytes per row.
      spmv (v = A p^ with (r^, v); t = A s^ with (t, s), (t, t), (s, s)):
        a product (product_bytes: all of A, or with the reuse the walked
        blocks and the added 3-vectors), 3 vector passes; 9 FMAs per walked
        block, 3 or 9 per row (the average of the two kinds is reported);
      update (x += alpha p^ + omega s^, r = s - omega t, ||r||, (r^, r)):
        6 vectors read, 2 written; 15 FMAs per row;
      finish (true residual and x back to the caller's order): a matrix
        pass, x gathered, b and the permutation read, x written; 9 FMAs per
        block and 3 per row;
      setup (b gathered through the permutation; r, r^, x, p, v written):
        6 vector passes and the permutation; 3 FMAs per row."""
    n, nnzb = info.nb, info.nnzb
    mat = 76 * nnzb + 4 * (n + 1)
    return {"factor": factor_work(info, fp32),
            "apply": (algorithmic_apply_bytes(info, fp32), 0 if fp32 else int(9 * nnzb + 4.5 * n)),
            "spmv": (product_bytes(info) + 72 * n, 9 * product_terms(info)[0] + 6 * n),
            "update": (192 * n, 15 * n),
            "setup": (148 * n, 3 * n),
            "finish": (mat + 76 * n, 9 * nnzb + 3 * n)}


def kernel_source_hash() -> str:
    """Hash of what fixes the sweep kernels' DRAM traffic: their device code
    and the layout the symbolic analysis gives the factors."""
    h = hashlib.sha256()
    for f in ("sweeps.cuh", "symbolic.cpp"):
        with open(os.path.join(ROOT, "paper_2309_11488_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, precision: str):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary (the
    JSON block of profiles/apply_traffic_c3_949871cells.md), if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "apply_traffic_c3_949871cells.md")
    try:
        with open(path) as f:
            txt = f.read()
        d = json.loads(txt.split("```json", 1)[1].split("```", 1)[0])
    except (OSError, ValueError, IndexError):
        return None
    e = d.get(f"{kernel}_{precision}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def make_system(grid):
    from paper_2309_11488_gb300 import synth
    return synth.config3(grid)


def rank_sync(dist, sync_device, device):
    """The replicas' timing plumbing: barrier() waits for every rank and then
    for this rank's device; max_over_ranks(v) is the largest v over the
    ranks (the slowest replica's time), reduced on `device` ("cuda" with
    NCCL, "cpu" with gloo).  Without a process group both act on this rank
    alone."""
    def barrier():
        if dist:
            dist.barrier()
        sync_device()

    def max_over_ranks(v):
        if not dist:
            return v
        import torch
        tt = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        return float(tt.item())
    return barrier, max_over_ranks


def run_ours(args, rank, world, dist):
    import torch
    from paper_2309_11488_gb300 import opm

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s = make_system(args.grid)
    rp, ci, vals = dev(s.rowptr), dev(s.colidx), dev(s.vals)
    xt = dev(s.x_true)

    barrier, max_over_ranks = rank_sync(dist, torch.cuda.synchronize, "cuda")

    def tuned(precision):
        """Launch options for this workload: the autotuner's choice, or the
        schedule given on the command line."""
        if args.schedule != "auto" or args.no_autotune:
            return {"schedule": args.schedule}, {"candidates": 0}
        with opm.Solver(s.nb, rp, ci, vals) as h:
            b = h.spmv(xt)
        t0 = time.perf_counter()
        st, kw, cands, bi = opm.autotune(s.nb, rp, ci, vals, b, rtol=RTOL, maxit=200, repeats=2,
                                         precision=precision)
        best_of = lambda sc: min((c["ms"] for c in cands if c["schedule"] == sc and c["status"] == 0),
                                 default=None)
        rep = {"status": st, "chosen": kw, "candidates": len(cands), "tune_s": round(time.perf_counter() - t0, 1),
               "ms_per_solve_best_level": best_of("level"), "ms_per_solve_best_colour": best_of("colour")}
        if st != opm.OPM_OK:
            return {"schedule": "auto"}, rep
        return kw, rep

    def measure(precision):
        kw, tune = tuned(precision)
        if args.no_product_reuse:
            kw = dict(kw, product_reuse=-1)
        sv = opm.Solver(s.nb, rp, ci, vals, precision=precision, **kw)
        b = sv.spmv(xt)  # b = A x_true on the GPU
        x = torch.empty_like(b)
        info = sv.info()
        stat = {}

        def step(h):
            # refactor + solve enqueued by one call, one host wait per step
            h.launch(vals, b, x, rtol=RTOL, maxit=200)
            st2, it, rr = h.wait()
            stat.update(st=opm.OPM_ERR_ZERO_PIVOT if st2 == opm.OPM_ERR_ZERO_PIVOT else 0, st2=st2, iters=it,
                        relres=rr)

        def step_profiled(h):
            st = h.factor(vals)
            _, st2, it, rr = h.solve(b, x, rtol=RTOL, maxit=200)

        for _ in range(max(3, args.warmup)):
            step(sv)
        sv.reset_timing()
        barrier()
        # an event after every step: the whole region gives the rate, the
        # per-step times its spread
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        with ClockSampler(local) as clk:
            evs[0].record()
            for k in range(args.steps):
                step(sv)
                evs[k + 1].record()
            torch.cuda.synchronize()
        barrier()
        ms = evs[0].elapsed_time(evs[-1])
        per = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)])
        spread = {"median_ms": round(float(np.median(per)), 4), "p10_ms": round(float(np.percentile(per, 10)), 4),
                  "p90_ms": round(float(np.percentile(per, 90)), 4), "min_ms": round(float(per.min()), 4),
                  "max_ms": round(float(per.max()), 4), "steps": int(args.steps)}
        launches = sv.timing().launches
        x_host = x.cpu().numpy()
        # the same solve without the refactorisation (opm_bicgstab_solve on
        # the factors of the last step): one host wait per solve
        xs = torch.empty_like(b)
        for _ in range(3):
            sv.solve(b, xs, rtol=RTOL, maxit=200)
        barrier()
        sevs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        sevs[0].record()
        for k in range(args.steps):
            _, sst, sit, _ = sv.solve(b, xs, rtol=RTOL, maxit=200)
            sevs[k + 1].record()
        torch.cuda.synchronize()
        barrier()
        sper = np.array([sevs[k].elapsed_time(sevs[k + 1]) for k in range(args.steps)])
        solve_only = {"ms_total": float(sevs[0].elapsed_time(sevs[-1])), "median_ms": round(float(np.median(sper)), 4),
                      "iters": int(sit), "status": int(sst),
                      "x_equal_to_step": bool(np.array_equal(xs.cpu().numpy(), x_host))}
        err = float(np.linalg.norm(x_host - s.x_true) / np.linalg.norm(s.x_true))
        # per-kernel device time from a second handle that records events
        # around every kernel group (a host-driven loop, so not the timed one)
        with opm.Solver(s.nb, rp, ci, vals, precision=precision, profile_kernels=True, **kw) as sp:
            for _ in range(2):
                step_profiled(sp)
            sp.reset_timing()
            for _ in range(max(3, min(args.steps, 30))):
                step_profiled(sp)
            t = sp.timing()
        return sv, dict(ms=ms, timing=t, launches=launches, info=info, clocks=clk.summary(), err=err, options=kw,
                        autotune=tune, spread=spread, x=x_host, solve_only=solve_only, **stat)

    sv64, r64 = measure("fp64")
    sv32, r32 = measure("fp32")
    ms64 = max_over_ranks(r64["ms"])
    ms32 = max_over_ranks(r32["ms"])

    # end to end through the C ABI from pinned host buffers: per step the
    # values and b go host -> device and x comes back, all enqueued by one
    # opm_solve_launch and awaited by opm_solve_wait
    vals_h = torch.from_numpy(np.ascontiguousarray(s.vals)).pin_memory()
    b_h = sv64.spmv(xt).cpu().pin_memory()
    x_h = torch.empty_like(b_h).pin_memory()

    def e2e_step():
        sv64.launch(vals_h, b_h, x_h, rtol=RTOL, maxit=200)
        st, it, rr = sv64.wait()
        assert st == 0, st

    for _ in range(2):
        e2e_step()
    # three timed blocks of n_e2e steps, the median block: a block lasts a
    # few tens of ms and crosses the host link, so one host stall would
    # otherwise decide the figure
    n_e2e = max(10, args.steps // 2)
    e2e_blocks = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        e2e_blocks.append(max_over_ranks(time.perf_counter() - t0))
        barrier()
    e2e_s = float(np.median(e2e_blocks))

    # the same calls through two handles of the pattern, each on its own
    # stream, used alternately: step k+1's host -> device copies overlap step
    # k's kernels.  Every step still copies its values and b from pinned host
    # memory and reads x back; a handle is reused only after its wait.
    pair, streams = [], [torch.cuda.Stream(), torch.cuda.Stream()]
    for q in range(2):
        h = opm.Solver(s.nb, rp, ci, vals, precision="fp64", stream=streams[q], **r64["options"])
        pair.append((h, torch.empty_like(b_h).pin_memory()))

    def e2e_overlapped(n):
        busy = [False, False]
        for k in range(n):
            h, xh = pair[k % 2]
            if busy[k % 2]:
                st, it, rr = h.wait()
                assert st == 0, st
            h.launch(vals_h, b_h, xh, rtol=RTOL, maxit=200)
            busy[k % 2] = True
        for q in (0, 1):
            if busy[q]:
                st, it, rr = pair[q][0].wait()
                assert st == 0, st

    # timed as the one-handle figure: the median of three blocks
    e2e_overlapped(4)
    blocks = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        e2e_overlapped(n_e2e)
        torch.cuda.synchronize()
        blocks.append(max_over_ranks(time.perf_counter() - t0))
        barrier()
    e2e2_s = float(np.median(blocks))
    x_ok = all(np.array_equal(xh.numpy(), x_h.numpy()) for _, xh in pair)
    for h, _ in pair:
        h.close()

    def solve_only_line(r):
        so = r["solve_only"]
        return {"value": round(world * args.steps / (max_over_ranks(so["ms_total"]) * 1e-3), 3), "unit": UNIT,
                "median_ms": so["median_ms"], "iters": so["iters"], "status": so["status"],
                "x_equal_to_step": so["x_equal_to_step"],
                "form": "BiCGStab + ILU0 application on the step's factors (opm_bicgstab_solve), setup and true "
                        "residual included, no refactorisation; one host wait per solve"}

    def roofline(r, precision):
        t = r["timing"]
        ms, cnt = t.kernel_ms[1], t.kernel_count[1]
        avg = ms / max(cnt, 1)
        nbytes = algorithmic_apply_bytes(r["info"], precision == "fp32")
        peak, src = peaks()
        ach = nbytes / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        # FP64 FMAs of one application: 9 per factor block (L and U blocks
        # in the sweeps, the inverse pivot once per row) and the right-hand
        # side (6 per row for p^, 3 for s^); with FP64 factors the HBM and
        # FP64 floors are within 1% of each other, so both are reported
        info = r["info"]
        fmas = 0 if precision == "fp32" else 9 * info.nnzb + 4.5 * info.nb
        return {"kernel": f"k_apply<{'float' if precision == 'fp32' else 'double'}> (ILU0 forward+backward)",
                "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_source": f"{src} (MEMORY copy, MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_launch": int(nbytes), "avg_launch_us": round(avg * 1e3, 2), "launches": int(cnt),
                "traffic": measured_traffic("apply", precision) if args.grid == 100 else None,
                "fp64_fma": {"fmas_per_launch": int(fmas),
                             "frac": round(fmas / (avg * 1e-3) / FP64_FMA_PEAK, 4) if avg > 0 else 0.0,
                             "peak_source": "derived: 2 FP64 FMA lanes/SM/clock x 152 SMs x 2.07 GHz"}}

    def iteration(r, ms_total, precision):
        """Per-iteration time of the timed run (its refactorisation, setup
        and final residual taken out at their profiled averages) against the
        HBM and FP64 FMA rooflines."""
        t = r["timing"]
        avg = lambda q: t.kernel_ms[q] / max(t.kernel_count[q], 1)
        per_step = ms_total / args.steps - avg(0) - avg(4) - avg(5)
        t_it = per_step / max(r["iters"], 1)
        nbytes, fma = iteration_work(r["info"], precision == "fp32")
        peak, src = peaks()
        gbs = nbytes / (t_it * 1e-3) / 1e9
        fmas = fma / (t_it * 1e-3)
        out = {"ms": round(t_it, 4), "iters_per_solve": r["iters"],
               "hbm": {"bytes": int(nbytes), "achieved_gbs": round(gbs, 1), "peak_gbs": peak,
                       "frac": round(gbs / peak, 4), "peak_source": src},
               "fp64_fma": {"fmas": int(fma), "achieved_tflops": round(2 * fmas / 1e12, 4),
                            "peak_tflops": round(2 * FP64_FMA_PEAK / 1e12, 4), "frac": round(fmas / FP64_FMA_PEAK, 4),
                            "peak_source": "derived: 2 FP64 FMA lanes/SM/clock x 152 SMs x 2.07 GHz"}}
        if product_terms(r["info"])[0] < r["info"].nnzb:
            tb, tf = iteration_work(PlainInfo(r["info"]), precision == "fp32")
            out["textbook_count"] = {
                "bytes": int(tb), "fmas": int(tf),
                "hbm_frac": round(tb / (t_it * 1e-3) / 1e9 / peak, 4),
                "fp64_frac": round(tf / (t_it * 1e-3) / FP64_FMA_PEAK, 4),
                "note": "the same iteration time against the bytes and FMAs of the iteration with every "
                        "product walking all of A (product_reuse off): the work the reuse saves counted "
                        "as done, so an effective rate, not a roofline fraction"}
        return out

    def kernels(r, precision):
        """Per-kernel device time from the profiled handle, with each kernel
        group's algorithmic bytes and FP64 FMAs per launch against the
        measured HBM copy bandwidth and the derived FP64 FMA peak."""
        t = r["timing"]
        work = kernel_work(r["info"], precision == "fp32")
        peak, src = peaks()
        out = {}
        for q, k in enumerate(opm.KERNELS):
            avg_ms = t.kernel_ms[q] / max(t.kernel_count[q], 1)
            e = {"ms_total": round(t.kernel_ms[q], 3), "launches": int(t.kernel_count[q]),
                 "avg_us": round(1e3 * avg_ms, 2)}
            if k in work and avg_ms > 0:
                nbytes, fma = work[k]
                e.update({"bytes_per_launch": nbytes, "hbm_frac": round(nbytes / (avg_ms * 1e-3) / 1e9 / peak, 4),
                          "fmas_per_launch": fma, "fp64_frac": round(fma / (avg_ms * 1e-3) / FP64_FMA_PEAK, 4)})
            out[k] = e
        out["peaks"] = {"hbm_gbs": peak, "hbm_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
                        "fp64_fma_per_s": FP64_FMA_PEAK,
                        "fp64_source": "derived: 2 FP64 FMA lanes/SM/clock x 152 SMs x 2.07 GHz"}
        return out

    out = {
        "metric": METRIC,
        "value": round(world * args.steps / (ms64 * 1e-3), 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": round(ms64 / args.steps, 4),
        "step_spread": r64["spread"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded generator shaped like the paper's 1M-cell model)",
        "config": {"workload": workload(args.grid, s.nb, len(s.colidx)), "options": r64["options"], "nsets": r64["info"].nsets,
                   "precision": "fp64 factors and Krylov", "rtol": RTOL, "parallelism": f"replicas x{world}",
                   "l2": (f"inputs larger than L2 (A values {len(s.colidx) * 72 / 1e6:.0f} MB, factors "
                          f"{len(s.colidx) * 72 / 1e6:.0f} MB)" if len(s.colidx) * 72 > 129e6 else
                          "inputs smaller than L2: not flushed")},
        "iters": r64["iters"], "relres": r64["relres"], "status": [r64["st"], r64["st2"]],
        "x_err_vs_x_true": r64["err"],
        "roofline": roofline(r64, "fp64"),
        "e2e": {"value": round(world * n_e2e / e2e_s, 3), "unit": UNIT,
                "h2d_bytes_per_step": int(s.vals.nbytes + 24 * s.nb), "d2h_bytes_per_step": int(24 * s.nb),
                "form": "one handle; each step's copies, refactor and solve, then its wait",
                "blocks_s": [round(v, 5) for v in e2e_blocks], "steps_per_block": n_e2e,
                "overlapped": {"value": round(world * n_e2e / e2e2_s, 3), "unit": UNIT,
                               "blocks_s": [round(v, 5) for v in blocks], "steps_per_block": n_e2e,
                               "form": "two handles on two streams used alternately: a step's copies overlap "
                                       "the other handle's kernels; same copies per step",
                               "x_equal_to_one_handle": bool(x_ok)}},
        "gpu_launches": int(r64["launches"]),
        "clocks": r64["clocks"],
        "kernels": kernels(r64, "fp64"),
        "iteration": iteration(r64, ms64, "fp64"),
        "without_refactor": solve_only_line(r64),
        "fp32_factors": {"value": round(world * args.steps / (ms32 * 1e-3), 3), "unit": UNIT,
                         "ms_per_step": round(ms32 / args.steps, 4), "step_spread": r32["spread"],
                         "iters": r32["iters"],
                         "relres": r32["relres"], "x_err_vs_x_true": r32["err"], "dtype": "f64 Krylov + f32 factors",
                         "roofline": roofline(r32, "fp32"), "kernels": kernels(r32, "fp32"), "options": r32["options"],
                         "iteration": iteration(r32, ms32, "fp32"), "without_refactor": solve_only_line(r32),
                         "autotune": r32["autotune"], "gpu_launches": int(r32["launches"]), "clocks": r32["clocks"]},
        "autotune": r64["autotune"],
    }
    sv64.close()
    sv32.close()
    del vals_h, b_h, x_h
    if r64["info"].nnzb_product < r64["info"].nnzb:
        out["product_reuse_off"] = measure_reuse_off(args, s, r64, barrier, max_over_ranks, world)
    tight_x = None
    if not args.no_tight:
        out["c3_rtol1e-6"], tight_x = measure_tight(args, s, r64, r32, barrier, max_over_ranks, world)
    if not args.no_jacobi:
        out["block_jacobi"] = measure_jacobi(args, s, barrier, max_over_ranks, world)
    if not args.no_wells:
        out["wells"] = measure_wells(args, s, out["config"]["options"], barrier, max_over_ranks, world)
    if not args.no_gmres:
        out["gmres"] = measure_gmres(args, s, out["config"]["options"], barrier, max_over_ranks, world)
    if not args.no_iterative:
        out["iterative"] = measure_iterative(args, s, barrier, max_over_ranks, world)
    if not args.no_small:
        try:
            out["small_configs"] = measure_small(args, barrier, world, rank)
        except Exception as e:  # the other figures stand without it
            out["small_configs"] = {"unavailable": f"{type(e).__name__}: {e}"}
    if not args.no_batched:
        out["batched"] = measure_batched(args, barrier, max_over_ranks, world)
    if not args.no_serving:
        out["serving"] = measure_serving(args, barrier, max_over_ranks, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sched = {v: k for k, v in opm.SCHEDULES.items()}[r64["info"].schedule]
        out["cpu_baseline"] = cpu_baseline(s, n_solves=2, schedule=sched, xs={"fp64": r64["x"], "fp32": r32["x"]})
        if tight_x is not None:
            out["c3_rtol1e-6"]["cpu_baseline"] = cpu_baseline_tight(s, out["c3_rtol1e-6"]["schedule"], tight_x)
    return out


def measure_reuse_off(args, s, r64, barrier, max_over_ranks, world):
    """The headline step (FP64, the same launch options) with every product
    walking all of A (opm_options.product_reuse = -1): the product reuse's
    effect measured beside the headline, and x against the headline's."""
    import torch
    from paper_2309_11488_gb300 import opm
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, vals = dev(s.rowptr), dev(s.colidx), dev(s.vals)
    kw = dict(r64["options"], product_reuse=-1)
    with opm.Solver(s.nb, rp, ci, vals, precision="fp64", **kw) as sv:
        b = sv.spmv(dev(s.x_true))
        x = torch.empty_like(b)

        def step():
            sv.launch(vals, b, x, rtol=RTOL, maxit=200)
            return sv.wait()
        for _ in range(max(3, args.warmup)):
            step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            st, it, rr = step()
        e1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1))
        xo = x.cpu().numpy()
    xr = r64["x"]
    return {"value": round(world * args.steps / (ms * 1e-3), 3), "unit": UNIT,
            "ms_per_step": round(ms / args.steps, 4), "iters": int(it), "status": int(st),
            "options": kw, "product_blocks": int(r64["info"].nnzb),
            "x_rel_diff_vs_reuse": float(np.linalg.norm(xo - xr) / np.linalg.norm(xr)),
            "form": "the headline step with every BiCGStab product walking all of A "
                    "(opm_options.product_reuse = -1); the headline's products walk "
                    f"{int(r64['info'].nnzb_product):,} of {int(r64['info'].nnzb):,} blocks"}


def measure_jacobi(args, s, barrier, max_over_ranks, world):
    """Block-Jacobi ILU0 (Section 4.5) on the same system: the preconditioner
    keeps the blocks inside each of args.partitions transmissibility-weighted
    partitions (the paper's 150-partition configurations), the SpMV all of A;
    refactor + solve to the same rtol, against the plain preconditioner, for
    level scheduling and the Kempe-reduced colouring."""
    import torch
    from paper_2309_11488_gb300 import opm, synth
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, vals, xt = dev(s.rowptr), dev(s.colidx), dev(s.vals), dev(s.x_true)
    part = synth.partition_grid(s, args.partitions)
    rows = np.repeat(np.arange(s.nb), np.diff(s.rowptr))
    dropped = int((part[rows] != part[s.colidx]).sum())
    res = {"partitions": int(args.partitions), "blocks_dropped": dropped,
           "blocks_dropped_frac": round(dropped / s.nnzb, 4)}
    reps = max(3, args.steps // 20)
    for sched in ("level", "colour_kempe"):
        for name, p in (("plain", None), ("jacobi", part)):
            with opm.Solver(s.nb, rp, ci, vals, schedule=sched, part=p) as sv:
                b = sv.spmv(xt)
                x = torch.empty_like(b)
                for _ in range(2):
                    sv.factor(vals)
                    _, st, it, rr = sv.solve(b, x, rtol=RTOL, maxit=200)
                barrier()
                t0 = time.perf_counter()
                for _ in range(reps):
                    sv.factor(vals)
                    _, st, it, rr = sv.solve(b, x, rtol=RTOL, maxit=200)
                torch.cuda.synchronize()
                dt = max_over_ranks(time.perf_counter() - t0)
                info = sv.info()
            res[f"{sched}_{name}"] = {"solves_per_s": round(world * reps / dt, 2), "iters": it, "status": st,
                                      "relres": rr, "nsets": info.nsets, "nphases": info.nphases}
    return res


def measure_wells(args, s, options, barrier, max_over_ranks, world):
    """Standard wells applied separately (Section 4.6): args.wells vertical
    wells of up to 20 perforated layers on the same system; the solver's
    operator is A - sum C^T inv(D) B, preconditioned by ILU0 of A; refactor +
    solve at the same rtol with the headline launch options, against no
    wells."""
    import torch
    from paper_2309_11488_gb300 import opm, synth
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, vals, xt = dev(s.rowptr), dev(s.colidx), dev(s.vals), dev(s.x_true)
    w = synth.wells(s, args.wells, 20)
    res = {"wells": int(w.nwells), "perforations": int(w.ptr[-1])}
    reps = max(3, args.steps // 20)
    for name, ww in (("without", None), ("with", w)):
        with opm.Solver(s.nb, rp, ci, vals, **options) as sv:
            if ww is not None:
                sv.set_wells(ww)
            b = sv.spmv(xt)  # b = (A - sum C^T inv(D) B) x_true
            x = torch.empty_like(b)
            for _ in range(2):
                sv.factor(vals)
                _, st, it, rr = sv.solve(b, x, rtol=RTOL, maxit=200)
            barrier()
            t0 = time.perf_counter()
            for _ in range(reps):
                sv.factor(vals)
                _, st, it, rr = sv.solve(b, x, rtol=RTOL, maxit=200)
            torch.cuda.synchronize()
            dt = max_over_ranks(time.perf_counter() - t0)
            err = float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt))
        res[name] = {"solves_per_s": round(world * reps / dt, 2), "iters": it, "status": st, "relres": rr,
                     "x_err_vs_x_true": err}
    return res


def measure_gmres(args, s, options, barrier, max_over_ranks, world):
    """Restarted GMRES(30) with the same ILU0 on the same system (headline
    launch options), beside BiCGStab: refactor + solve to the same rtol per
    step, and the solve alone per preconditioner application (the factors
    computed once)."""
    import torch
    from paper_2309_11488_gb300 import opm
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, vals, xt = dev(s.rowptr), dev(s.colidx), dev(s.vals), dev(s.x_true)
    reps = max(3, args.steps // 4)
    res = {"restart": 30}
    with opm.Solver(s.nb, rp, ci, vals, **options) as sv:
        b = sv.spmv(xt)
        x = torch.empty_like(b)
        for name, solve in (("gmres", lambda: sv.gmres(b, x, rtol=RTOL, maxit=300, restart=30)),
                            ("bicgstab", lambda: sv.solve(b, x, rtol=RTOL, maxit=200))):
            for _ in range(2):
                sv.factor(vals)
                _, st, it, rr = solve()
            barrier()
            t0 = time.perf_counter()
            for _ in range(reps):
                sv.factor(vals)
                _, st, it, rr = solve()
            torch.cuda.synchronize()
            dt = max_over_ranks(time.perf_counter() - t0)
            t0 = time.perf_counter()
            for _ in range(reps):
                _, st, it, rr = solve()
            torch.cuda.synchronize()
            ds = max_over_ranks(time.perf_counter() - t0)
            apps = it + (1 if name == "gmres" else it)
            res[name] = {"solves_per_s": round(world * reps / dt, 2), "iters": it, "status": st, "relres": rr,
                         "preconditioner_applications": apps, "solve_ms": round(1e3 * ds / reps, 4),
                         "ms_per_application": round(1e3 * ds / reps / max(apps, 1), 4)}
        res["gmres_vs_bicgstab_per_application"] = round(res["gmres"]["ms_per_application"] /
                                                         res["bicgstab"]["ms_per_application"], 3)
    return res


RTOL_TIGHT = 1e-6


def measure_tight(args, s, r64, r32, barrier, max_over_ranks, world):
    """The iteration-dominated regime: the same workload and launch options
    at rtol 1e-6 (about five times the iterations of rtol 1e-3), FP64 and
    FP32 factors.  Each step is one refactorisation + solve through
    opm_solve_launch / opm_solve_wait, event-timed.  The iteration share is
    the step's time outside the refactorisation, setup and final residual
    (their profiled averages from the headline run).  Returns the figures
    and the two solutions (host arrays) for the oracle comparison."""
    import torch
    from paper_2309_11488_gb300 import opm
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, vals, xt = dev(s.rowptr), dev(s.colidx), dev(s.vals), dev(s.x_true)
    reps = max(5, args.steps // 2)
    out, xs = {}, {}
    for precision, r in (("fp64", r64), ("fp32", r32)):
        with opm.Solver(s.nb, rp, ci, vals, precision=precision, **r["options"]) as sv:
            b = sv.spmv(xt)
            x = torch.empty_like(b)
            for _ in range(2):
                sv.launch(vals, b, x, rtol=RTOL_TIGHT, maxit=200)
                st, it, rr = sv.wait()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                sv.launch(vals, b, x, rtol=RTOL_TIGHT, maxit=200)
                st, it, rr = sv.wait()
            e1.record()
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1)) / reps
            barrier()
            t = r["timing"]
            avg = lambda q: t.kernel_ms[q] / max(t.kernel_count[q], 1)
            outside = avg(0) + avg(4) + avg(5)
            xs[precision] = x.cpu().numpy()
            nbytes, _ = iteration_work(r["info"], precision == "fp32")
            t_it = (ms - outside) / max(it, 1)
            peak, src = peaks()
            out[precision] = {"value": round(world * 1e3 / ms, 3), "unit": UNIT, "ms_per_step": round(ms, 4),
                              "iters": it, "status": st, "relres": rr,
                              "iteration_share": round(1.0 - outside / ms, 4),
                              "ms_per_iteration": round(t_it, 4),
                              "iteration_hbm_frac": round(nbytes / (t_it * 1e-3) / 1e9 / peak, 4),
                              "x_err_vs_x_true": float(np.linalg.norm(xs[precision] - s.x_true)
                                                       / np.linalg.norm(s.x_true))}
    out["schedule"] = {v: k for k, v in opm.SCHEDULES.items()}[r64["info"].schedule]
    out["rtol"] = RTOL_TIGHT
    return out, xs


def cpu_baseline_tight(s, schedule, xs):
    """The oracle at rtol 1e-6 in the library's order, one full step on one
    host core: its rate, and the GPU solutions' distance from its x (the FP64
    path's parity at this rtol, the FP32-factor path's accuracy)."""
    import oracle as O
    b = O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true)
    perm, _ = O.schedule_perm(s.nb, s.rowptr, s.colidx, schedule)
    pb = b.reshape(-1, 3)[perm].ravel()
    t0 = time.perf_counter()
    prow, pcol, pval = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    fac = O.ilu0(s.nb, prow, pcol, pval)
    res = O.bicgstab(s.nb, prow, pcol, pval, fac, pb, RTOL_TIGHT, 200)
    dt = time.perf_counter() - t0
    x = np.empty(3 * s.nb)
    x.reshape(-1, 3)[perm] = res.x.reshape(-1, 3)
    nx = np.linalg.norm(x)
    return {"value": round(1.0 / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle", "iters": res.iters,
            "sample": f"1 full step at rtol 1e-6 ({res.iters} iterations) in the {schedule} order, "
                      f"single-threaded C",
            "x_err_fp64_vs_oracle": float(np.linalg.norm(xs["fp64"] - x) / nx),
            "x_err_fp32_factors_vs_oracle": float(np.linalg.norm(xs["fp32"] - x) / nx)}


def small_config_cases():
    """(name, generator, rtol, schedule) of the configurations that fit in L2:
    C1 (10x10x5, natural order) and C2 (the 44,431-cell NORNE stand-in, graph
    colouring, rtol 1e-2 and 1e-6), each also in the library's default order."""
    from paper_2309_11488_gb300 import synth
    return [("C1", synth.config1, 1e-2, "natural"), ("C1", synth.config1, 1e-2, "auto"),
            ("C2", synth.config2, 1e-2, "colour"), ("C2", synth.config2, 1e-6, "colour"),
            ("C2", synth.config2, 1e-2, "auto"), ("C2", synth.config2, 1e-6, "auto")]


def oracle_small(q, rtol, schedule, repeats=5):
    """The oracle, single-threaded, on one small configuration in the order
    the library used: median seconds of `repeats` steps (value permutation,
    ILU0, BiCGStab), the order's setup untimed."""
    import oracle as O
    b = O.spmv(q.nb, q.rowptr, q.colidx, q.vals, q.x_true)
    perm, _ = O.schedule_perm(q.nb, q.rowptr, q.colidx, schedule)
    pb = b.reshape(-1, 3)[perm].ravel()
    times, res = [], None
    for _ in range(repeats):
        t0 = time.perf_counter()
        prow, pcol, pval = O.permute(q.nb, q.rowptr, q.colidx, q.vals, perm)
        fac = O.ilu0(q.nb, prow, pcol, pval)
        res = O.bicgstab(q.nb, prow, pcol, pval, fac, pb, rtol, 200)
        times.append(time.perf_counter() - t0)
    return float(np.median(times)), res


def measure_small(args, barrier, world, rank):
    """C1 and C2, which fit in L2: per step one refactorisation and one
    solve (two synchronous calls), each step timed with CUDA events, median
    of at least 20 steps;
    beside it the oracle, single-threaded, median of 5 steps in the same
    order (rank 0 at one GPU only)."""
    import torch
    from paper_2309_11488_gb300 import opm
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    names = {v: k for k, v in opm.SCHEDULES.items()}
    reps = max(20, args.steps // 10)
    out, cache = [], {}
    for name, gen, rtol, schedule in small_config_cases():
        if name not in cache:
            cache[name] = gen()
        q = cache[name]
        rp, ci, va, xt = dev(q.rowptr), dev(q.colidx), dev(q.vals), dev(q.x_true)
        with opm.Solver(q.nb, rp, ci, va, schedule=schedule,
                        product_reuse=-1 if args.no_product_reuse else 0) as sv:
            used = names[sv.info().schedule]
            b = sv.spmv(xt)
            x = torch.empty_like(b)

            def step():
                # refactor, then solve: the calls the parity tests make on
                # these configurations and orders
                sv.factor(va)
                _, st, it, rr = sv.solve(b, x, rtol=rtol, maxit=200)
                return st, it, rr
            for _ in range(5):
                step()
            barrier()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for e0, e1 in ev:
                e0.record()
                st, it, rr = step()
                e1.record()
            torch.cuda.synchronize()
            ms = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
        p50 = float(np.median(ms))
        row = {"config": name, "cells": q.nb, "blocks": q.nnzb, "schedule": used, "rtol": rtol, "iters": it,
               "status": st, "relres": rr, "p50_ms": round(p50, 4), "p90_ms": round(float(np.percentile(ms, 90)), 4),
               "solves_per_s": round(world * 1e3 / p50, 2), "repeats": reps}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            t, res = oracle_small(q, rtol, used)
            row["oracle"] = {"p50_ms": round(1e3 * t, 3), "solves_per_s": round(1.0 / t, 3), "iters": res.iters,
                             "cores": 1, "repeats": 5, "kind": "oracle"}
        out.append(row)
    return {"cases": out, "l2": "inputs smaller than L2, not flushed: L2-resident latency per refactor + solve"}


def measure_iterative(args, s, barrier, max_over_ranks, world):
    """Chow-Patel iterative ILU0 (cp sweeps) and Jacobi triangular solves
    (tri sweeps per triangle), the "Chow Patel ILU0" of Section 3's library
    table, on the same system: factorisation time, solve time and iterations
    to the same rtol, against the exact factorisation and substitution, for
    level scheduling (the natural-order ILU0, many phases) and smallest-last
    colouring (few phases)."""
    import torch
    from paper_2309_11488_gb300 import opm
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, vals, xt = dev(s.rowptr), dev(s.colidx), dev(s.vals), dev(s.x_true)
    reps = max(3, args.steps // 20)
    res = {}
    for sched in ("level", "colour_sl"):
        for cp, tri in ((0, 0), (0, 3), (3, 0), (2, 2), (3, 3)):
            with opm.Solver(s.nb, rp, ci, vals, schedule=sched, cp_sweeps=cp, tri_sweeps=tri) as sv:
                b = sv.spmv(xt)
                x = torch.empty_like(b)
                for _ in range(2):
                    sv.factor(vals)
                    _, st, it, rr = sv.solve(b, x, rtol=RTOL, maxit=300)
                barrier()
                t0 = time.perf_counter()
                for _ in range(reps):
                    sv.factor(vals)
                torch.cuda.synchronize()
                tf = max_over_ranks(time.perf_counter() - t0)
                barrier()
                t0 = time.perf_counter()
                for _ in range(reps):
                    _, st, it, rr = sv.solve(b, x, rtol=RTOL, maxit=300)
                torch.cuda.synchronize()
                ts = max_over_ranks(time.perf_counter() - t0)
                err = float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt))
            res[f"{sched}_cp{cp}_tri{tri}"] = {
                "solves_per_s": round(world * reps / (tf + ts), 2), "factor_ms": round(1e3 * tf / reps, 3),
                "solve_ms": round(1e3 * ts / reps, 3), "iters": it, "status": st, "relres": rr,
                "x_err_vs_x_true": err}
    # one Jacobi application (3 sweeps per triangle) against the HBM and FP64
    # rooflines, timed by the profiled handle's events (level order)
    with opm.Solver(s.nb, rp, ci, vals, schedule="level", cp_sweeps=3, tri_sweeps=3, profile_kernels=True) as sv:
        b = sv.spmv(xt)
        x = torch.empty_like(b)
        sv.factor(vals)
        sv.solve(b, x, rtol=RTOL, maxit=300)
        sv.reset_timing()
        for _ in range(reps):
            sv.factor(vals)
            sv.solve(b, x, rtol=RTOL, maxit=300)
        t = sv.timing()
        info = sv.info()
    avg_ms = t.kernel_ms[1] / max(t.kernel_count[1], 1)
    nbytes, fma = jacobi_apply_work(info, 3, False)
    peak, src = peaks()
    gbs = nbytes / (avg_ms * 1e-3) / 1e9
    fmas = fma / (avg_ms * 1e-3)
    res["jacobi_apply_level_tri3"] = {
        "avg_launch_group_us": round(avg_ms * 1e3, 2), "applications": int(t.kernel_count[1]),
        "kernels_per_application": 7,
        "hbm": {"bytes": nbytes, "achieved_gbs": round(gbs, 1), "peak_gbs": peak, "frac": round(gbs / peak, 4),
                "peak_source": src},
        "fp64_fma": {"fmas": fma, "frac": round(fmas / FP64_FMA_PEAK, 4),
                     "peak_source": "derived: 2 FP64 FMA lanes/SM/clock x 152 SMs x 2.07 GHz"},
        "factor_ms_cp3": round(t.kernel_ms[0] / max(t.kernel_count[0], 1), 3)}
    return res


def measure_batched(args, barrier, max_over_ranks, world):
    """256 independent systems of uneven size (grids 5..40 per axis, 500 to
    20,000 cells), FP32 factors + FP64 Krylov, rtol 1e-2 each, refactored and
    solved by the same kernel launches (one batch); against the plain FP64
    path solving the same systems one after another."""
    import torch
    from paper_2309_11488_gb300 import opm, synth
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    syss = synth.config4(nsys=args.batch_systems)
    data = [(dev(q.rowptr), dev(q.colidx), dev(q.vals), dev(q.x_true)) for q in syss]
    # right-hand sides b = A x_true with the library's FP64 SpMV
    bs = []
    for q, (rp, ci, va, xt) in zip(syss, data):
        with opm.Solver(q.nb, rp, ci, va) as h:
            bs.append(h.spmv(xt))
    res = {}
    for precision in ("fp32", "fp64"):
        # launch configuration: the autotuner on every fourth system (or the
        # schedule given on the command line)
        if args.schedule == "auto" and not args.no_autotune:
            sub = list(range(0, len(syss), 4))
            t_tune = time.perf_counter()
            tst, kw, cands, bi = opm.autotune_batch(
                [(syss[k].nb, data[k][0], data[k][1], data[k][2], bs[k]) for k in sub], rtol=[1e-2] * len(sub),
                maxit=200, repeats=2, precision=precision)
            tune = {"status": tst, "chosen": kw, "candidates": len(cands), "tuned_on_systems": len(sub),
                    "tune_s": round(time.perf_counter() - t_tune, 2)}
            if tst != opm.OPM_OK:
                kw = {"schedule": "auto", "sweep_launch": "auto", "chunk": 0, "small_phase_slices": 0}
        else:
            kw = {"schedule": args.schedule, "sweep_launch": "auto", "chunk": 0, "small_phase_slices": 0}
            tune = {"chosen": kw, "candidates": 0}
        hs = [opm.Solver(q.nb, rp, ci, va, schedule=kw["schedule"], precision=precision)
              for q, (rp, ci, va, xt) in zip(syss, data)]
        xs = [torch.empty_like(b) for b in bs]
        vals = [d[2] for d in data]
        with opm.Batch([h.h for h in hs], chunk=kw["chunk"], sweep_launch=kw["sweep_launch"],
                       small_phase_slices=kw["small_phase_slices"]) as bt:
            def step():
                bt.factor(vals)
                return bt.solve(bs, xs, rtol=1e-2, maxit=200)
            for _ in range(3):
                step()
            barrier()
            reps = max(3, args.steps // 30)
            t0 = time.perf_counter()
            for _ in range(reps):
                st_all, st, it, rr = step()
            torch.cuda.synchronize()
            dt = max_over_ranks(time.perf_counter() - t0)
        # the same systems one at a time through the single-system path
        t1 = time.perf_counter()
        for h, v, b, x in zip(hs, vals, bs, xs):
            h.factor(v)
            h.solve(b, x, rtol=1e-2, maxit=200)
        torch.cuda.synchronize()
        dt_seq = max_over_ranks(time.perf_counter() - t1)
        err = max(float(torch.linalg.norm(x - d[3]) / torch.linalg.norm(d[3])) for x, d in zip(xs, data))
        res[precision] = {"solves_per_s": round(world * len(syss) * reps / dt, 2),
                          "ms_per_batch": round(1e3 * dt / reps, 3),
                          "sequential_solves_per_s": round(world * len(syss) / dt_seq, 2),
                          "iters_mean": float(np.mean(it)), "iters_max": int(max(it)),
                          "status_ok": int(sum(1 for v in st if v == 0)), "max_rel_err_vs_x_true": err,
                          "autotune": tune}
        for h in hs:
            h.close()
    cells = sum(q.nb for q in syss)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_batched(len(syss))
        except Exception as e:  # the GPU figures stand without it
            cpu = {"kind": "oracle", "unavailable": f"{type(e).__name__}: {e}"}
    return {"cpu_baseline": cpu,
            "workload": f"{len(syss)} independent systems, {cells} cells total, grids 5..40 per axis, "
                        f"per step: batched refactor + BiCGStab to rtol 1e-2 for every system",
            "value": res["fp32"]["solves_per_s"], "unit": "solves/s", "dtype": "f64 Krylov + f32 factors",
            "fp32_factors": res["fp32"], "fp64": res["fp64"],
            "vs_plain_fp64_sequential": round(res["fp32"]["solves_per_s"] / res["fp64"]["sequential_solves_per_s"], 3)}


def measure_serving(args, barrier, max_over_ranks, world):
    """Poisson request stream over 32 sparsity patterns of 5k-250k cells; each
    request is a Newton-step value update (blocks scaled by U(0.9, 1.1)) that
    needs ILU0 refactorisation + BiCGStab to rtol 1e-2.  Analyses are kept per
    pattern, instances stay resident in lanes admitted by an HBM budget, and
    the ready requests of a size class share one batched launch; latency =
    completion - arrival.  Three runs after the warm one: the offered rate
    (the headline p50/p99), a saturating stream (offered far above capacity:
    the serving capacity), and a short run under a budget that binds (lanes
    evicted and remade from the kept analyses)."""
    import torch
    from paper_2309_11488_gb300 import serve, synth
    pats = [synth.config5_pattern(p) for p in range(args.patterns)]
    tmpl = serve.request_templates(pats, 2, "fp32")

    def requests(rate, duration, seed):
        t = serve.poisson_arrivals(rate, duration, seed)
        pick = serving_picks(len(pats), len(t), seed)
        return [serve.Request(i, float(ti), int(pick[i]), *tmpl[int(pick[i])][i % 2]) for i, ti in enumerate(t)]

    def engine(budget_gb, class_size, lanes):
        return serve.ServingEngine(pats, precision="fp32", hbm_budget_bytes=int(budget_gb * (1 << 30)),
                                   class_size=class_size, lanes_per_class=lanes)

    eng = engine(args.hbm_budget_gb, args.class_size, args.lanes_per_class)
    t0 = time.perf_counter()
    eng.warm()
    warm_setup_s = time.perf_counter() - t0
    eng.run(requests(args.rate, args.serve_warm_s, 31))          # warm: lanes, clocks
    barrier()
    stats = eng.run(requests(args.rate, args.serve_s, 32))
    barrier()
    summ = stats.summary()
    sat_rate = 1e6  # every request arrives within a few ms: the run measures the capacity
    sat = eng.run(requests(sat_rate, args.sat_requests / sat_rate, 33)).summary()
    barrier()
    eng.close()
    # a budget below one instance of every pattern (a lane per pattern, so
    # that an eviction frees one pattern's memory): lanes are evicted and
    # remade from the kept analyses while the run goes on
    bound_gb = args.bound_budget_gb
    eng = engine(bound_gb, 1, 1)
    eng.warm()
    bound = eng.run(requests(args.rate, args.bound_s, 34)).summary()
    eng.close()
    if world == 1 and not args.no_cpu_baseline:
        try:
            summ["cpu_baseline"] = cpu_baseline_serving(len(pats))
        except Exception as e:  # the GPU figures stand without it
            summ["cpu_baseline"] = {"kind": "oracle", "unavailable": f"{type(e).__name__}: {e}"}
    cells = [q.nb for q in pats]
    summ.update({"workload": f"{len(pats)} patterns of {min(cells)}..{max(cells)} cells, Poisson arrivals "
                             f"{args.rate:g} req/s for {args.serve_s:g} s (after {args.serve_warm_s:g} s warm), "
                             f"refactor + BiCGStab rtol 1e-2 per request, FP32 factors + FP64 Krylov",
                 "engine": f"size classes of {args.class_size} patterns, up to {args.lanes_per_class} lanes per "
                           f"class, analyses kept per pattern, ready requests of a class in one batched launch",
                 "analysis_and_warm_lanes_s": round(warm_setup_s, 2),
                 "hbm_budget_bytes": int(args.hbm_budget_gb * (1 << 30)), "offered_rate": args.rate,
                 "solves_per_s_all_ranks": round(world * summ["solves_per_s"], 2),
                 "max_solves_per_s": round(sat["solves_per_s"], 2),
                 "saturated": {**{k: sat[k] for k in ("requests", "completed", "failed", "solves_per_s", "p50_ms",
                                                      "p99_ms", "mean_batch", "launches", "max_in_flight")},
                               "offered_rate": sat_rate},
                 "budget_bound": {**{k: bound[k] for k in ("requests", "completed", "failed", "solves_per_s",
                                                           "p50_ms", "p99_ms", "max_ms", "evictions",
                                                           "lanes_created_in_run", "hbm_bytes_peak")},
                                  "hbm_budget_bytes": int(bound_gb * (1 << 30)), "seconds": args.bound_s,
                                  "engine": "one lane per pattern (a size class of one)"}})
    return summ


def cpu_oracle_setup(s, schedule="colour_kempe"):
    """The oracle's inputs for the workload: b = A x_true and the schedule's
    permutation (by default the smallest-last colouring reduced by Kempe
    exchanges, the library's default)."""
    import oracle as O
    b = O.spmv(s.nb, s.rowptr, s.colidx, s.vals, s.x_true)
    perm, _ = O.schedule_perm(s.nb, s.rowptr, s.colidx, schedule)
    pb = b.reshape(-1, 3)[perm].ravel()
    return O, perm, pb


def oracle_solve(O, s, perm, pb):
    """One step of the workload on the oracle: the value permutation, ILU0,
    BiCGStab to rtol 1e-3 and the true residual."""
    prow, pcol, pval = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    fac = O.ilu0(s.nb, prow, pcol, pval)
    return O.bicgstab(s.nb, prow, pcol, pval, fac, pb, RTOL, 200)


def cpu_baseline(s, n_solves=2, schedule="colour_kempe", xs=None):
    """The oracle's rate on one host core; with xs (the GPU solutions of the
    headline step, FP64 and FP32 factors), their distance from the oracle's
    x in the same row order."""
    O, perm, pb = cpu_oracle_setup(s, schedule)
    t0 = time.perf_counter()
    for _ in range(n_solves):
        res = oracle_solve(O, s, perm, pb)
    dt = time.perf_counter() - t0
    out = {"value": round(n_solves / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n_solves} full steps (value permutation, ILU0, BiCGStab to rtol 1e-3 in {res.iters} "
                     f"iterations, true residual) of the same system in the library's order ({schedule}), "
                     f"single-threaded C, {os.cpu_count()} host cores present", "iters": res.iters}
    if xs:
        x = np.empty(3 * s.nb)
        x.reshape(-1, 3)[perm] = res.x.reshape(-1, 3)
        nx = np.linalg.norm(x)
        for k, v in xs.items():
            out[f"x_err_{k}_vs_oracle"] = float(np.linalg.norm(v - x) / nx)
    return out


def _oracle_worker(conn, kind, jobs, nsys, rtol, repeats):
    """One host core of a multi-core oracle baseline.  Builds its share of the
    workload and sets it up untimed (b = A x_true, the colour_kempe order),
    reports ready, then on "go" times `repeats` passes of value permutation
    + ILU0 + BiCGStab over its jobs and sends (seconds, statuses,
    iterations).  kind "batched": jobs are indices of the batched workload's
    systems; kind "serving": jobs are (pattern, template) requests, the
    values of a template made once and shared by its requests."""
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2309_11488_gb300 import synth
    systems, prepared, perms = {}, {}, {}
    dims = synth.config4_dims(nsys) if kind == "batched" else None
    work = []
    for job in jobs:
        if job not in prepared:
            if kind == "batched":
                q = synth.config4_system(job, dims)
                vals, xt = q.vals, q.x_true
                pk = ("s", job)
            else:
                p, k = job
                if p not in systems:
                    systems[p] = synth.config5_pattern(p)
                q = systems[p]
                vals, xt = synth.newton_update(q, 1000 * p + k)
                pk = ("p", p)
            if pk not in perms:
                perms[pk] = O.schedule_perm(q.nb, q.rowptr, q.colidx, "colour_kempe")[0]
            perm = perms[pk]
            b = O.spmv(q.nb, q.rowptr, q.colidx, vals, xt)
            prepared[job] = (q, vals, perm, b.reshape(-1, 3)[perm].ravel())
        work.append(prepared[job])
    conn.send("ready")
    conn.recv()
    st, its = [], []
    t0 = time.perf_counter()
    for rep in range(repeats):
        for q, vals, perm, pb in work:
            prow, pcol, pval = O.permute(q.nb, q.rowptr, q.colidx, vals, perm)
            fac = O.ilu0(q.nb, prow, pcol, pval)
            res = O.bicgstab(q.nb, prow, pcol, pval, fac, pb, rtol, 200)
            if rep == 0:
                st.append(int(res.status))
                its.append(int(res.iters))
    conn.send((time.perf_counter() - t0, st, its))
    conn.close()


def _run_oracle_processes(kind, shards, nsys, rtol, repeats, timeout_s):
    """One spawned process per shard, all started on the same signal; returns
    (the slowest process's seconds, statuses, iterations)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    procs = []
    try:
        for jobs in shards:
            parent, child = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(child, kind, jobs, nsys, rtol, repeats), daemon=True)
            p.start()
            procs.append((p, parent))
        for p, c in procs:
            if not c.poll(timeout_s) or c.recv() != "ready":
                raise RuntimeError("an oracle process did not get ready")
        for p, c in procs:
            c.send("go")
        out = []
        for p, c in procs:
            if not c.poll(timeout_s):
                raise RuntimeError("an oracle process did not finish")
            out.append(c.recv())
    finally:
        for p, c in procs:
            p.join(5)
            if p.is_alive():
                p.terminate()
    return (max(o[0] for o in out), [v for o in out for v in o[1]], [v for o in out for v in o[2]])


def cpu_baseline_batched(nsys, rtol=1e-2, repeats=5, cores=None, timeout_s=600.0):
    """The oracle on all host cores for the batched workload: one spawned
    process per core, systems dealt round-robin, every process started on
    the same signal; solves/s = repeats x nsys / the slowest process's time."""
    cores = max(1, min(cores or os.cpu_count() or 1, nsys))
    shards = [list(range(w, nsys, cores)) for w in range(cores)]
    wall, st, its = _run_oracle_processes("batched", shards, nsys, rtol, repeats, timeout_s)
    return {"value": round(repeats * nsys / wall, 2), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{repeats} passes over all {nsys} systems (value permutation, ILU0, BiCGStab to rtol {rtol:g} "
                      f"in the colour_kempe order, FP64), one single-threaded C oracle process per core, systems "
                      f"dealt round-robin; time of the slowest process",
            "status_ok": sum(1 for v in st if v == 0), "iters_mean": float(np.mean(its)) if its else 0.0}


def serving_picks(npat, nreq, seed=32):
    """Patterns of the first nreq requests of the serving run's request
    stream (the same counter-based draw the serving leg makes)."""
    from paper_2309_11488_gb300 import synth
    u = synth.uniform(synth.stream_key(seed, 5), np.arange(nreq, dtype=np.uint64))
    return np.minimum((u * npat).astype(int), npat - 1)


def cpu_baseline_serving(npat, nreq=256, rtol=1e-2, repeats=1, cores=None, timeout_s=600.0):
    """The oracle on all host cores for the serving workload, closed loop (no
    arrival process): the first nreq requests of the serving stream, each a
    refactorisation + solve of its pattern with the request's values.  A
    pattern's requests stay on one process; patterns are dealt to the least
    loaded process by cells x requests.  solves/s = repeats x nreq / the
    slowest process's time."""
    from paper_2309_11488_gb300 import synth
    pick = serving_picks(npat, nreq)
    cells = {p: int(np.prod(d)) for p, d in enumerate(synth.config5_dims(npat))}
    jobs = {}
    for i, p in enumerate(pick.tolist()):
        jobs.setdefault(p, []).append((p, i % 2))
    cores = max(1, min(cores or os.cpu_count() or 1, len(jobs)))
    shards, load = [[] for _ in range(cores)], [0] * cores
    for p in sorted(jobs, key=lambda p: -cells[p] * len(jobs[p])):
        w = int(np.argmin(load))
        shards[w] += jobs[p]
        load[w] += cells[p] * len(jobs[p])
    wall, st, its = _run_oracle_processes("serving", shards, npat, rtol, repeats, timeout_s)
    return {"value": round(repeats * nreq / wall, 2), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {nreq} requests of the serving stream over {len(jobs)} of {npat} patterns, "
                      f"closed loop (value permutation, ILU0, BiCGStab to rtol {rtol:g} in the colour_kempe "
                      f"order, FP64), one single-threaded C oracle process per core; time of the slowest process",
            "status_ok": sum(1 for v in st if v == 0), "iters_mean": float(np.mean(its)) if its else 0.0}


def run_reference(args, rank, world):
    """The oracle on the host cores, one full step of the workload per timed
    step.  At most as many steps as fit args.ref_budget_s are timed (K when
    they fit): a full C3 step takes over a second on one core, and the arm
    must end within minutes."""
    if rank != 0:
        return None
    s = make_system(args.grid)
    O, perm, pb = cpu_oracle_setup(s)
    t0 = time.perf_counter()
    for _ in range(max(1, args.warmup)):
        oracle_solve(O, s, perm, pb)
    t_one = (time.perf_counter() - t0) / max(1, args.warmup)
    n = max(1, min(args.steps, int(args.ref_budget_s / max(t_one, 1e-9))))
    t0 = time.perf_counter()
    for _ in range(n):
        res = oracle_solve(O, s, perm, pb)
    dt = time.perf_counter() - t0
    v = round(n / dt, 4)
    sample = (f"{n} full steps of the workload timed" + ("" if n == args.steps else
              f" ({args.steps} requested; the steps that fit {args.ref_budget_s:.0f} s)") +
              ", single-threaded C oracle")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": n,
            "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / n, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.grid, s.nb, len(s.colidx)), "schedule": "colour_kempe", "rtol": RTOL},
            "iters": res.iters, "relres": res.relres,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    from paper_2309_11488_gb300 import build
    build.build()
    out = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
