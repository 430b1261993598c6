"""The multi-process path on CPU (gloo, world size 2): the bench's weak-scaling
shards (independent populations per rank, no data-path collective), the
max-over-ranks step time and the whole-job rate, and the reference arm under
torchrun, where rank 0 alone runs and prints one line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1511_02166_gb300 import inputs
    spec = bench.rank_population_spec(inputs.SPECS["naca_b64_n100"], rank)
    pop = inputs.make_population(spec, batch=6)
    nodes = torch.from_numpy(np.ascontiguousarray(pop.nodes).ravel())
    got = [torch.empty_like(nodes) for _ in range(world)]
    dist.all_gather(got, nodes)
    ms = bench.max_over_ranks(10.0 + rank)
    np.savez(os.path.join(outdir, "rank%d.npz" % rank), nodes=np.stack([g.numpy() for g in got]),
             ms=ms, rate=bench.whole_job_rate(world, pop.batch, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_and_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]
    for r in res:
        assert float(r["ms"]) == 11.0  # the slowest rank's time on every rank
        assert abs(float(r["rate"]) - world * 6 / 11.0e-3) < 1e-9
        a, b = r["nodes"]
        assert a.shape == b.shape and not np.array_equal(a, b)  # independent shards
    assert np.array_equal(res[0]["nodes"], res[1]["nodes"])


def test_reference_arm_rank0_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-seconds", "1",
           "--config", "naca_b64_n100"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["steps"] == 1
