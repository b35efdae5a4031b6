"""The multi-rank logic of bench.py on CPU: world_size-2 gloo ranks (one replica per rank, no
data-path collective).  Whole-job throughput is every rank's units over the slowest rank's time,
the barrier and the max-over-ranks reduction work, each rank seeds its own independent problem, and
the reference arm does no work on ranks other than 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist("gloo")
    try:
        d.barrier()
        t_local = 1.0 + rank             # rank 1 is the slow one
        value, t = bench.whole_job(d, 100.0, t_local)
        ref = bench.reference_arm(type("A", (), {"warmup": 3, "steps": 1})(), d) if rank else "skipped"
        q.put((rank, d.world, value, t, ref))
        d.barrier()
    finally:
        d.close()


@pytest.mark.timeout(120)
def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, world, value, t, ref in out:
        assert world == 2
        assert t == 2.0                  # the slowest rank's time
        assert value == 2 * 100.0 / 2.0  # all ranks' units over that time
    assert out[1][4] is None             # rank 1 returns from the reference arm without work


def test_single_rank_needs_no_process_group():
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    d = bench.Dist("gloo")
    assert d.world == 1 and d.pg is None
    assert bench.whole_job(d, 50.0, 2.0) == (25.0, 2.0)


def test_replicas_draw_independent_initial_states():
    from paper_2605_23812_gb300 import synth
    a = synth.cavity_ic(64, 32, seed=1234)
    b = synth.cavity_ic(64, 32, seed=1235)
    assert a[0].shape == b[0].shape and not (a[0] == b[0]).all()
