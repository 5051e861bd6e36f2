"""The multi-process side of bench.py on CPU (gloo, world size 2): the barrier, the
max-over-ranks timing reduction, and the reference arm's rank-0-only rule."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        t = bench.max_over_ranks(1.5 + rank, ws)            # rank times 1.5 s and 2.5 s
        rc = bench.run_reference(None, rank, ws) if rank != 0 else 0   # non-zero ranks return at once
        out.put((rank, t, rc))
    finally:
        dist.destroy_process_group()


def test_replicas_barrier_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [2.5, 2.5]      # both ranks see the slowest rank's time
    assert [r[2] for r in res] == [0, 0]


def test_reference_arm_prints_one_contract_line(capsys):
    """Rank 0 of `bench.py --impl reference` times the FP64 oracle on the host and prints
    one JSON line with the keys of the bench contract, the reference tag, a cpu_baseline
    describing itself and an e2e entry with no host-device traffic."""
    import argparse
    import json
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(argparse.Namespace(gpus=1, steps=1, warmup=0), 0, 1) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
