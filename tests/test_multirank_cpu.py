"""The replicas path (one process per GPU, no data-path collective) on the
CPU with world size 2 over gloo: the bench's barrier waits for both ranks and
then for the rank's device, the timing reduction returns the slowest rank's
time on every rank, and the reference arm runs on rank 0 alone while the
other rank exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import importlib.util, json, os, sys, time
import torch.distributed as dist
spec = importlib.util.spec_from_file_location("bench_rank", os.path.join(sys.argv[1], "bench.py"))
b = importlib.util.module_from_spec(spec)
sys.argv = ["bench.py"]
spec.loader.exec_module(b)
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
synced = []
barrier, max_over_ranks = b.rank_sync(dist, lambda: synced.append(time.perf_counter()), "cpu")
t0 = time.perf_counter()
if rank == 1:
    time.sleep(0.5)           # the slow replica
barrier()
waited = time.perf_counter() - t0
slowest = max_over_ranks(0.25 + rank)
alone = b.rank_sync(None, lambda: None, "cpu")[1](0.25 + rank)
print(json.dumps({"rank": rank, "waited": waited, "slowest": slowest, "alone": alone, "synced": len(synced)}))
dist.destroy_process_group()
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(args, world, extra_env=None):
    env0 = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_port()), WORLD_SIZE=str(world))
    procs = []
    for r in range(world):
        env = dict(env0, RANK=str(r), LOCAL_RANK=str(r), **(extra_env or {}))
        procs.append(subprocess.Popen(args, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        outs.append((p.returncode, o, e))
    return outs


def test_barrier_and_max_over_ranks_with_gloo():
    outs = _launch([sys.executable, "-c", _WORKER, ROOT], 2)
    res = {}
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        d = json.loads(o.strip().splitlines()[-1])
        res[d["rank"]] = d
    for r in (0, 1):
        assert res[r]["slowest"] == 1.25          # rank 1's value on both ranks
        assert res[r]["alone"] == 0.25 + r        # no group: the rank's own value
        assert res[r]["synced"] == 1              # the device sync ran after the barrier
    assert res[0]["waited"] >= 0.45               # rank 0 waited for the slow rank


def test_reference_arm_runs_on_rank_zero_only():
    outs = _launch([sys.executable, "bench.py", "--impl", "reference", "--grid", "8", "--steps", "2",
                    "--warmup", "1"], 2)
    (rc0, o0, e0), (rc1, o1, e1) = outs
    assert rc0 == 0 and rc1 == 0, (e0[-1000:], e1[-1000:])
    assert o1.strip() == ""
    lines = [ln for ln in o0.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
