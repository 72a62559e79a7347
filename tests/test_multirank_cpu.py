"""Host-side logic of the N-rank benchmark on CPU with the gloo backend
(world size 2): each rank renders its own ring view (independent problems,
no data-path collective) and the step time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", world_size=world, rank=rank)
    try:
        w, r, lr = bench.dist_env()
        t = bench.max_over_ranks(10.0 + 5.0 * rank, device="cpu")
        cam = bench.ring_view_for_rank(rank, world, 64, 48)
        bench.barrier()
        centre = -np.asarray(cam.R).T @ np.asarray(cam.T)
        q.put((rank, w, r, t, centre.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_distinct_views():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[3] == pytest.approx(15.0) for o in out)          # max over ranks
    # the two ranks render different cameras of the ring (same distance)
    assert not np.allclose(out[0][4], out[1][4])
    assert np.linalg.norm(out[0][4]) == pytest.approx(np.linalg.norm(out[1][4]))


def test_single_process_helpers_without_a_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    bench.barrier()
    w, r, lr = bench.dist_env()
    assert w >= 1 and r >= 0
