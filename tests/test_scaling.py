"""Multi-rank bookkeeping of the benchmark on CPU: two gloo ranks, each with
its own molecule (weak scaling), reduce the job's time (max) and work (sum)
exactly as the GPU ranks do under torchrun with NCCL."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    from paper_1809_04352_gb300 import inputs, scaling

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = scaling.rank_env()
        xyz, _ = inputs.workload_atoms(1, molecule=r)  # the bench's per-rank molecule choice
        secs = 1.5 + r
        pts = 1000.0 * (r + 1)
        t, n = scaling.job_totals(secs, pts, "cpu")
        out.put((r, w, t, n, scaling.throughput(n, 4, t), float(xyz[:, 0].sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_points():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, t, n, v, xs) in enumerate(res):
        assert rank == r and world == 2
        assert t == 2.5 and n == 3000.0
        assert v == pytest.approx(3000.0 * 4 / 2.5)
    assert res[0][5] != res[1][5]  # every rank computes its own molecule


def test_single_rank_is_identity():
    from paper_1809_04352_gb300 import scaling

    assert scaling.job_totals(3.0, 7.0) == (3.0, 7.0)
    assert scaling.throughput(7.0, 2, 3.0) == pytest.approx(14.0 / 3.0)
    assert np.isfinite(scaling.job_max(1.0))
