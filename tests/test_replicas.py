"""The replica bookkeeping of multi-GPU runs (paper_2605_19796_gb300/replicas.py)
on two CPU processes with the gloo backend: max-over-ranks timing, the
whole-job rate, distinct seeds, barriers, root-only reporting, and a rank
that leaves: the others' next barrier fails within the group timeout.  The data path
has no collective (independent replicas), so this is all there is to shard."""
import multiprocessing as mp
import os
import socket

import pytest

from paper_2605_19796_gb300.replicas import Replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    try:
        rep = Replicas("gloo")
        rep.barrier()
        t = rep.max_over_ranks(1.0 + rank)  # per-rank times 1 s and 2 s
        rate = rep.whole_job_rate(100.0, t)
        seeds = [rep.seed(b, 3) for b in range(3)]
        rep.barrier()
        q.put((rank, rep.world, rep.root, t, rate, seeds))
        rep.close()
    except Exception as e:  # reported to the parent
        q.put((rank, "error", repr(e)))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in ps)
    res = sorted(res)
    for rank, world, root, t, rate, seeds in res:
        assert world == 2 and root == (rank == 0)
        assert t == 2.0  # the slowest rank
        assert rate == pytest.approx(100.0 * 2 / 2.0)
    assert sorted(res[0][5] + res[1][5]) == list(range(6))  # distinct seeds over ranks and boxes


def _leaving_worker(rank, world, port, q):
    """Rank 1 leaves between steps (no collective in flight) without telling
    anyone; rank 0's next barrier must fail within the group's timeout."""
    import time

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    rep = Replicas("gloo", timeout_s=5.0)
    rep.barrier()  # both ranks are up
    if rank == 1:
        q.put((rank, "left", 0.0))
        q.close()
        q.join_thread()  # the message is out before the process goes
        os._exit(0)
    t0 = time.perf_counter()
    try:
        rep.barrier()
        q.put((rank, "no error", time.perf_counter() - t0))
    except Exception as e:  # the expected outcome
        q.put((rank, "error: " + type(e).__name__, time.perf_counter() - t0))
    q.close()
    q.join_thread()
    os._exit(0)


def test_rank_that_leaves_fails_the_others_next_barrier():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict((r, (what, dt)) for r, what, dt in (q.get(timeout=120) for _ in ps))
    for p in ps:
        p.join(timeout=60)
    assert res[1][0] == "left"
    assert res[0][0].startswith("error"), res[0]
    assert res[0][1] < 30.0  # bounded by the group timeout, not a hang


def test_single_process_needs_no_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    rep = Replicas()
    assert rep.world == 1 and rep.root and rep.dist is None
    assert rep.max_over_ranks(3.5) == 3.5 and rep.whole_job_rate(10.0, 2.0) == 5.0
    rep.barrier()
    rep.close()
