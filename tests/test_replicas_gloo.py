"""The N > 1 path of bench.py on the CPU: world size 2 over gloo.

Games are independent (no exchange step in the iteration), so ranks run
replicas with no collective on the data path; the only collectives are the
barrier around the timed region and the max / sum reductions of the timing.
Each rank's work must not depend on the other rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_1810_03063_b300 import synth
    w, r, _ = bench.dist_setup()
    n, _, steps = bench.oracle_iterations(0, max_iters=2, seed=synth.BASE_SEED + r)
    bench.barrier(w)
    mx = bench.allreduce_max(w, float(r + 1))
    total = bench.allreduce_sum(w, float(n))
    q.put((r, w, mx, total, n))
    dist.destroy_process_group()


def test_two_replicas_reduce_time_and_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 2.0 for o in out)            # max over ranks
    assert all(o[3] == 4.0 for o in out)            # iterations of both replicas
    assert all(o[4] == 2 for o in out)
