"""Multi-rank PML/TVaR over trial shards: each rank sends its m largest year
losses with their global trial indices, one all-gather, and the C-ABI merge
(ara_merge_top, host code, no GPU) gives the PML/TVaR of the whole YLT.

Run as world_size-2 gloo ranks on CPU.  A rank's top m comes from the
oracle's sort here (on the GPU it is ara_top_m, tested in test_gpu_parity.py);
the merged result is checked against the oracle on the concatenated YLT
(Section 2.3).
"""

import os
import socket

import numpy as np
import pytest

import oracle

RPS = (2.0, 100.0, 250.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard(rank, n):
    rng = np.random.default_rng(100 + rank)
    y = np.round(rng.lognormal(6, 2, n), 1)  # ties within and across shards
    y[rng.random(n) < 0.3] = 0.0
    return y


def _local_top(y, m, offset):
    order = oracle.sort_desc(y)[:m]
    vals = np.full(m, -np.inf)
    trials = np.full(m, -1, np.int64)
    vals[: order.size] = y[order]
    trials[: order.size] = offset + order
    return vals, trials


def _worker(rank, world, port, n, q):
    import torch
    import torch.distributed as dist

    from paper_1501_06326_gb300 import ara

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        y = _shard(rank, n)
        m = int(np.ceil(world * n / min(RPS)))
        vals, trials = _local_top(y, m, rank * n)
        gv = [torch.empty(m, dtype=torch.float64) for _ in range(world)]
        gt = [torch.empty(m, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gv, torch.from_numpy(vals))
        dist.all_gather(gt, torch.from_numpy(trials))
        pml, tvar = ara.merge_top(torch.cat(gv).numpy(), torch.cat(gt).numpy(), world * n, RPS)
        q.put((rank, pml, tvar))
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_matches_oracle():
    import multiprocessing as mp

    world, n = 2, 5000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = np.concatenate([_shard(r, n) for r in range(world)])
    rpml, rtvar = oracle.pml_tvar(full, RPS)
    for _, pml, tvar in results:
        assert np.array_equal(pml, rpml)
        assert np.allclose(tvar, rtvar, rtol=1e-14, atol=0)


@pytest.mark.parametrize("world", [1, 3, 8])
def test_merge_of_uneven_shards_matches_oracle(world):
    from paper_1501_06326_gb300 import ara

    rng = np.random.default_rng(world)
    sizes = rng.integers(1, 3000, world)
    shards = [np.round(rng.lognormal(5, 1.5, s), 0) for s in sizes]  # many ties
    n_total = int(sizes.sum())
    rps = np.array([1.0, 3.0, 100.0, 1e6])
    m = int(np.ceil(n_total / rps.min()))
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    tops = [_local_top(y, m, o) for y, o in zip(shards, offs)]
    pml, tvar = ara.merge_top(np.concatenate([t[0] for t in tops]), np.concatenate([t[1] for t in tops]),
                              n_total, rps)
    rpml, rtvar = oracle.pml_tvar(np.concatenate(shards), rps)
    assert np.array_equal(pml, rpml)
    assert np.allclose(tvar, rtvar, rtol=1e-14, atol=0)


def test_merge_rejects_too_few_values():
    from paper_1501_06326_gb300 import ara

    with pytest.raises(ara.AraError):
        ara.merge_top(np.array([3.0, 1.0, -np.inf]), np.array([0, 1, -1]), 6, [1.0])
    with pytest.raises(ara.AraError):
        ara.merge_top(np.array([3.0]), np.array([0]), 1, [0.5])
