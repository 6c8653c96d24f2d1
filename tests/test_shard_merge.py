"""Multi-rank PML/TVaR merge (trial shards, one all-gather of top-m values),
run as world_size-2 gloo ranks on CPU and checked against the oracle on the
concatenated YLT."""

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1501_06326_gb300.shard import global_pml_tvar, local_top

RPS = (2.0, 100.0, 250.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard(rank, n):
    rng = np.random.default_rng(100 + rank)
    y = np.round(rng.lognormal(6, 2, n), 1)
    y[rng.random(n) < 0.3] = 0.0
    return y


def _worker(rank, world, port, n, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        y = _shard(rank, n)
        m = int(np.ceil(world * n / min(RPS)))
        top = torch.from_numpy(local_top(y, m))
        gathered = [torch.empty_like(top) for _ in range(world)]
        dist.all_gather(gathered, top)
        pml, tvar = global_pml_tvar([g.numpy() for g in gathered], world * n, RPS)
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


def test_local_top_pads_short_shards():
    t = local_top(np.array([3.0, 1.0]), 4)
    assert t[0] == 3.0 and t[1] == 1.0 and np.isneginf(t[2:]).all()
    with pytest.raises(ValueError):
        global_pml_tvar([t], 6, (1.0,))
