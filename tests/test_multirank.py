"""Multi-rank (replica) path of the benchmark on CPU, world size 2 over gloo.

The workload does not shard (each rank runs whole images on its own GPU), so
the only cross-rank steps are the barrier and the max-reduce of the timed
region; those, the whole-job throughput and the reference arm's rank-0-only
output are checked here without a GPU."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import bench
    D = bench.Dist(world, torch.device("cpu"))
    D.barrier()
    t_max = D.max(10.0 + rank)          # per-rank timed region, ms
    v = bench.replica_throughput(1 << 20, 5, world, t_max)
    D.barrier()
    D.close()
    with open(os.path.join(out, "r%d.json" % rank), "w") as f:
        json.dump({"t_max": t_max, "value": v}, f)


def test_two_gloo_ranks_agree_on_the_slowest_rank(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / ("r%d.json" % k))) for k in range(2)]
    assert r[0]["t_max"] == r[1]["t_max"] == 11.0
    # whole-job throughput: both replicas' pixels over the slowest rank's time
    assert abs(r[0]["value"] - (1 << 20) * 5 * 2 / 11.0e-3 / 1e6) < 1e-9
    assert r[0]["value"] == r[1]["value"]


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
