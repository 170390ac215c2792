"""bench.py's multi-rank aggregation on CPU: two gloo ranks with different
times; every rank gets the slowest time and the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, ms = bench.combine_ranks(100.0 * (rank + 1), 10, dist, device="cpu")
        q.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in out:
        assert ms == pytest.approx(200.0)            # the slower rank's time
        assert value == pytest.approx(2 * 10 / 0.2)  # units of both ranks / max time


def test_combine_ranks_single_process():
    import bench

    value, ms = bench.combine_ranks(250.0, 5)
    assert ms == 250.0 and value == pytest.approx(20.0)


class _FakeSession:
    """Counts steps; every feature is decided at the third iteration."""

    def __init__(self):
        self.t, self.writes = 0, 0

    def read(self):
        return {"t": 0}

    def write(self, state):
        self.t = state["t"]
        self.writes += 1

    def step(self):
        self.t += 1
        return 0 if self.t == 3 else 5

    def kernel_launches(self):
        return 100 + self.t  # the library's count for the step just taken


def test_stepper_restarts_finished_runs_outside_the_step():
    import bench

    S = _FakeSession()
    R = bench.Stepper(S, max_iter=10)
    ts = []
    for _ in range(7):
        R.ready()  # restart (untimed) only when the last step finished the run
        R.step()
        ts.append(S.t)
    assert ts == [1, 2, 3, 1, 2, 3, 1]
    assert S.writes == 2
    assert R.launches == sum(100 + t for t in ts)  # counted over restarts too
    R2 = bench.Stepper(_FakeSession(), max_iter=2)  # t = max_iter also ends a run
    for _ in range(3):
        R2.ready()
        R2.step()
    assert R2.S.writes == 1
