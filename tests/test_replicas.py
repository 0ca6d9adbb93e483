"""The multi-process (N > 1) bench path on CPU with gloo, world size 2:
replicas share nothing but the barrier and the max / sum reductions around
the timed region; under torchrun the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, w, _ = bench.dist_init()
    bench.barrier(w)
    t_max = bench.allreduce_max(1.0 + r, w)          # per-rank step time
    conv = bench.allreduce_sum(81 * (r + 1), w)      # per-rank converged plans
    out.put((r, w, t_max, conv, conv / t_max))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_reductions():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, t_max, conv, value) in enumerate(res):
        assert rank == r and world == 2
        assert t_max == 2.0                          # the slowest rank's time
        assert conv == 81 + 162                      # all ranks' plans
        assert value == pytest.approx(243 / 2.0)     # whole-job throughput


@pytest.mark.slow
def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "cfg0", "--steps", "2", "--warmup", "1", "--gpus", "2"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
