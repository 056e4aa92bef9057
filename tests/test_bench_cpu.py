"""bench.py's reference arm runs on the host (the oracle on a z-slab of the
roofline workload) and prints the one JSON line of the benchmark contract; checked
here on a small sample, without a GPU."""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "3", "--cpu-rows", "64"],
                         cwd=ROOT, capture_output=True, text=True, check=True, timeout=600)
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    # value = cell-updates (2 species x 64 rows x 256 beams per step) per second
    assert abs(d["value"] * d["ms_per_step"] * 1e-3 - 2 * 64 * 256) < 1e-6 * 2 * 64 * 256
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_reference_arm_two_ranks_gloo():
    """Launched as the benchmark contract launches N > 1 (torchrun, one process per
    rank, rendezvous on 127.0.0.1): rank 0 alone runs the sample and prints the one
    line; the other rank exits 0 without output."""
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                          "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                          "--master-port", "29517", os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
                          "--cpu-rows", "32"],
                         cwd=ROOT, capture_output=True, text=True, check=True, timeout=600)
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, out.stdout + out.stderr
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def _max_over_ranks(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier(world)
    q.put((rank, bench.dist_max(float(10 * rank + 1), world)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    """The timing reduction of the N > 1 path (barrier, then the maximum over
    ranks) on two gloo ranks: every rank gets the larger value."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_max_over_ranks, args=(r, 2, 29519, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 11.0, 1: 11.0}
