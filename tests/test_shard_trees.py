"""Tree sharding of one iteration, simulated on the host with two gloo
ranks: each rank computes the importance rows of the trees tau = rank mod 2
(every rank builds the same shadows from the same counter-based streams),
the rows are all-gathered and put back in tree order, and the result equals
the single-process iteration row for row -- so the statistic and the test,
computed redundantly from them, are identical on every rank.  (The GPU
build runs one process per GPU as replicas; this pins the exchange a
sharded run would need.)"""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp

from paper_2605_09950_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(importance):
    import oracle

    w = synth.binary_small(N=300, p=10, n_inf=3, n_trees=6, max_depth=5, max_iter=4, importance=importance)
    return w, oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)


def _worker(rank, world, port, importance, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, P = _problem(importance)
        live = np.arange(w.p, dtype=np.int32)
        sha = P.shadow(1, live)
        p_aug = w.p + sha.shape[0]
        mine = list(range(rank, w.n_trees, world))
        rows = np.zeros((len(mine), p_aug))
        for k, tau in enumerate(mine):
            _, ti, pm = P.tree(1, live, sha, tau, nodes=False, treeimp=importance == synth.TREEIMP,
                               permut=importance == synth.PERMUT)
            rows[k] = ti if importance == synth.TREEIMP else pm
        per_rank = (w.n_trees + world - 1) // world
        buf = torch.zeros((per_rank, p_aug), dtype=torch.float64)
        buf[: len(mine)] = torch.from_numpy(rows)
        parts = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        full = np.zeros((w.n_trees, p_aug))
        for r in range(world):
            for k, tau in enumerate(range(r, w.n_trees, world)):
                full[tau] = parts[r][k].numpy()
        q.put((rank, full))
    finally:
        dist.destroy_process_group()


def _run(importance):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, importance, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w, P = _problem(importance)
    want = P.iteration(1, np.zeros(w.p, np.int8), np.zeros(w.p, np.int32))["imp"]
    for rank in (0, 1):
        np.testing.assert_array_equal(out[rank], want)


def test_tree_sharding_treeimp_rows_match_single_process():
    _run(synth.TREEIMP)


def test_tree_sharding_permut_rows_match_single_process():
    _run(synth.PERMUT)
