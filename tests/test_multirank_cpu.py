"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Every rank decomposes its own tensor (no data-path collective); the ranks
only meet at barriers and in the max-over-ranks reduction of the timings,
and rank 0 alone prints.  These run the same helpers bench.py uses, and the
reference arm end to end under torch.distributed.run.
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    r, w, loc = bench.rank_env()
    dist = bench.init_ranks(w)
    bench.barrier(dist)
    slowest = bench.max_over_ranks(10.0 + 2.5 * r, dist)  # rank r "took" 10 + 2.5 r ms
    bench.barrier(dist)
    dist.destroy_process_group()
    q.put((r, w, loc, slowest))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 0, 12.5), (1, 2, 1, 12.5)]


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.init_ranks(1) is None
    assert bench.max_over_ranks(3.25, None) == 3.25


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-n", "40"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["unit"] == "ms"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
