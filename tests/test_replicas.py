"""Multi-process tests (world size 2, gloo on CPU) of the replica
coordination used by the multi-GPU form (paper_1103_3373_gb300/replicas.py):
contiguous shards covering the work, the whole-job rate taken over the
slowest rank, and a rank that leaves before the collective: the other rank
gets an error from a short process-group timeout instead of waiting."""
import datetime
import multiprocessing
import os
import socket
import time

import pytest

from paper_1103_3373_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_1103_3373_gb300 import replicas as R
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    r, w, local = R.rank_info()
    if mode == "rate":
        start, stop = R.shard(4096, r, w)
        units = (stop - start) * 16 ** 3
        rate, max_ms, total = R.job_rate(10.0 * (r + 1), units, dist, device="cpu")
        q.put((r, w, local, start, stop, rate, max_ms, total))
        dist.destroy_process_group()
    else:
        if r == 1:
            q.put((r, "left"))
            q.close()
            q.join_thread()  # the message is out before the process goes
            os._exit(0)  # leaves between steps, with nothing in flight
        t0 = time.perf_counter()
        try:
            R.job_rate(1.0, 1.0, dist, device="cpu")
            q.put((r, "no error"))
        except Exception as e:  # the collective fails: the peer is gone
            q.put((r, "error", type(e).__name__, time.perf_counter() - t0))


def _run(mode, world=2, timeout=60):
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=timeout) for _ in range(world)]
    for p in ps:
        p.join(timeout=timeout)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda x: x[0])


def test_shards_cover_the_work():
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def test_single_process_rate():
    rate, ms, units = replicas.job_rate(20.0, 1000.0)
    assert (rate, ms, units) == (50000.0, 20.0, 1000.0)


def test_two_ranks_rate_over_the_slowest():
    out = _run("rate")
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert out[0][3:5] == (0, 2048) and out[1][3:5] == (2048, 4096)
    for o in out:
        assert o[6] == 20.0                         # max over ranks
        assert o[7] == 4096 * 16 ** 3               # sum over ranks
        assert o[5] == pytest.approx(4096 * 16 ** 3 / 0.020)


def test_rank_leaving_before_the_collective_is_reported():
    out = _run("fail")
    assert out[1] == (1, "left")
    assert out[0][0] == 0 and out[0][1] == "error"
    assert out[0][3] < 8.0  # within the process-group timeout
