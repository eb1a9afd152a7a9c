"""Host-side logic of bench.py that needs no GPU: the reference (oracle) arm's
JSON line, its behaviour under two ranks, and the max-over-ranks reduction on
the gloo backend."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(cmd, env=None, timeout=300):
    e = dict(os.environ)
    if env:
        e.update(env)
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=e)


def test_reference_arm_line():
    r = run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "0",
             "--ref-seconds", "1"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("naca0012_4096x2048")
    # the contract's K and W: K timed steps after W warm-up steps, each a bounded sample
    assert d["steps"] == 2 and d["warmup"] == 0 and "band" in d["cpu_baseline"]["sample"]


def test_reference_arm_two_ranks_only_rank0_prints():
    r = run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
             "--master-addr", "127.0.0.1", "--master-port", "29517", "bench.py", "--impl",
             "reference", "--gpus", "2", "--steps", "2", "--warmup", "0", "--ref-seconds", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["n_gpus"] == 2


def _max_rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    q.put((rank, bench.reduce_max(10.0 + 5 * rank)))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_max_rank, args=(r, 2, 29531, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: 15.0, 1: 15.0}


def test_reduce_max_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5


def test_reference_arm_band_sample():
    # the reference arm's bounded sample: a thin band takes the all-fluid top
    # rows; a band of at least half the height is centred and holds the airfoil
    sys.path.insert(0, ROOT)
    import bench
    from paper_2210_10377_gb300 import inputs
    w = inputs.LARGE_F32
    thin, y0 = bench.oracle_band(w, 3)
    assert thin.shape == (3, w.nx) and y0 == w.ny - 3 and thin.sum() == 0
    thick, y0 = bench.oracle_band(w, w.ny // 2)
    assert thick.shape == (w.ny // 2, w.nx) and y0 == w.ny // 4
    import oracle
    full = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    assert thick.sum() == full.sum() > 0
