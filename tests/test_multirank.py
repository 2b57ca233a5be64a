"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The solver runs replicas only (one independent problem per GPU, no
collective on the data path); what spans ranks is the bench's bookkeeping:
the barrier, the max-over-ranks time, the sum-over-ranks work, and the rule
that rank 0 alone prints the JSON line (the reference arm: rank 0 alone runs
the oracle, the other ranks exit 0 without work)."""
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


def _reduce_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    w, r, _, pg = bench.dist_setup(world)
    assert (w, r) == (world, rank)
    bench.barrier(pg)
    out[rank] = (bench.max_over_ranks(pg, 10.0 * (rank + 1)), bench.sum_over_ranks(pg, rank + 1.5))
    pg.destroy_process_group()


def test_rank_reductions_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        procs = [mp.Process(target=_reduce_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(world):
            assert out[r] == (20.0, 1.5 + 2.5)  # max of 10, 20; sum of 1.5, 2.5


def test_reference_arm_two_ranks_prints_one_line():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--N", "12", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
