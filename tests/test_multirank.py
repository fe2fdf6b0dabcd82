"""The N > 1 benchmark path on the CPU: two ranks over gloo (weak scaling,
no data-path collective: only the step-time maximum crosses ranks), and the
reference arm launched under torchrun (rank 0 prints the one JSON line,
the other rank exits without work)."""
import json
import os
import socket
import subprocess
import sys
import tempfile

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sec = bench.max_over_ranks(0.001 * (rank + 1), dist)  # rank 1 is the slower one
    value = bench.aggregate_value(1e9, sec, world)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"sec": sec, "value": value}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step_and_sum_units():
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        r = [json.load(open(os.path.join(d, f"r{k}.json"))) for k in range(2)]
    assert r[0]["sec"] == r[1]["sec"] == 0.002
    assert abs(r[0]["value"] - 2 * 1e9 / 0.002) < 1e-3


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "0", "--ref-sample", "4096"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    lines = [json.loads(x) for x in r.stdout.decode().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
