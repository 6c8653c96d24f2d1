"""GPU tests of the serving loop (ara_submit / ara_serve_step / ara_poll):
each request's PML/TVaR against the FP64 oracle on its own trial prefix
(1e-4 relative), results identical alone and in a mix of requests, and the
batch-forming rules."""

import numpy as np
import pytest

import oracle
from paper_1501_06326_gb300 import synth

pytestmark = pytest.mark.gpu

PML_TOL = 1e-4
RPS = (10.0, 40.0)


@pytest.fixture(scope="module")
def eng():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1501_06326_gb300 import ara

    e = ara.Ara(0)
    yield e
    e.close()


@pytest.fixture(scope="module")
def world():
    # 1,000 trials x Poisson(100) over 10,000 events; a pool of 16 ELTs x 1,000 records;
    # 12 requests of 1..6 ELTs with trial prefixes of 40..1000 and percentile terms
    yet = synth.make_yet(1000, 100.0, 10_000, 515)
    pool = synth.make_elt_pool(16, 1000, 10_000, 516)
    rng = np.random.default_rng(517)
    reqs = []
    for ids in synth.draw_layers(12, pool.elt_ids, 6, 518):
        sub = pool.subset([int(i) for i in ids])
        t_end = int(rng.integers(40, 1001))
        terms = oracle.calibrate_layer_terms(yet, sub, t_end=t_end)
        reqs.append((ids, terms, t_end, sub))
    return yet, pool, reqs


def _load(eng, yet, pool):
    eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)
    eng.load_pool(pool)


def _serve_all(eng, reqs, seed=0):
    tickets = [eng.submit(ids, terms, seed, t_end, RPS) for ids, terms, t_end, _ in reqs]
    steps = 0
    while True:
        n = eng.serve_step()
        if n == 0:
            break
        steps += 1
    return [eng.poll(tk, len(RPS)) for tk in tickets], steps


def test_served_requests_match_the_oracle(eng, world):
    yet, pool, reqs = world
    _load(eng, yet, pool)
    got, steps = _serve_all(eng, reqs, seed=3)
    assert steps >= 1
    for (ids, terms, t_end, sub), res in zip(reqs, got):
        assert res is not None
        ref = oracle.run_layer(yet, sub, terms, seed=3, trials=np.arange(t_end))
        pml, tvar = oracle.pml_tvar(ref["ylt"], RPS)
        assert np.allclose(res[0], pml, rtol=PML_TOL, atol=1e-9)
        assert np.allclose(res[1], tvar, rtol=PML_TOL, atol=1e-9)


def test_results_identical_alone_and_in_a_mix(eng, world):
    yet, pool, reqs = world
    _load(eng, yet, pool)
    mixed, _ = _serve_all(eng, reqs, seed=7)
    for req, res in zip(reqs, mixed):
        alone, _ = _serve_all(eng, [req], seed=7)
        assert np.array_equal(alone[0][0], res[0]) and np.array_equal(alone[0][1], res[1])


def test_batches_follow_the_rules(eng, world):
    yet, pool, reqs = world
    _load(eng, yet, pool)
    ids, terms, t_end, _ = reqs[0]
    # at most ARA_MAX_BATCH_LAYERS requests per batch
    tk = [eng.submit(ids, terms, 0, t_end, RPS) for _ in range(40)]
    assert eng.serve_step() == 32
    assert eng.serve_step() == 8
    assert eng.serve_step() == 0
    first = [eng.poll(t, len(RPS)) for t in tk]
    assert all(np.array_equal(first[0][0], r[0]) for r in first)
    # one seed per batch: requests of another seed wait for a later batch
    a = [eng.submit(ids, terms, 1, t_end, RPS) for _ in range(3)]
    b = [eng.submit(ids, terms, 2, t_end, RPS) for _ in range(3)]
    assert eng.poll(a[0], len(RPS)) is None
    assert eng.serve_step() == 3
    assert eng.poll(b[0], len(RPS)) is None
    assert eng.serve_step() == 3
    for t in a + b:
        assert eng.poll(t, len(RPS)) is not None


def test_serving_errors(eng, world):
    from paper_1501_06326_gb300 import ara

    yet, pool, reqs = world
    _load(eng, yet, pool)
    ids, terms, t_end, _ = reqs[0]
    with pytest.raises(ara.AraError) as e:
        eng.submit([999], terms, 0, t_end, RPS)
    assert e.value.code == ara.ARA_ENOTLOADED
    with pytest.raises(ara.AraError) as e:
        eng.submit(ids, terms, 0, yet.n_trials + 1, RPS)
    assert e.value.code == ara.ARA_EINVAL
    with pytest.raises(ara.AraError) as e:
        eng.submit(ids, terms, 0, t_end, [0.5])
    assert e.value.code == ara.ARA_EINVAL
    with pytest.raises(ara.AraError) as e:
        eng.poll(123456789, len(RPS))
    assert e.value.code == ara.ARA_EINVAL


def test_wait_serves_until_the_request_is_done(eng, world):
    from paper_1501_06326_gb300 import ara

    yet, pool, reqs = world
    _load(eng, yet, pool)
    # requests of two seeds: waiting for a later one runs the steps before it
    t_a = [eng.submit(ids, terms, 11, t_end, RPS) for ids, terms, t_end, _ in reqs[:3]]
    t_b = eng.submit(reqs[3][0], reqs[3][1], 12, reqs[3][2], RPS)
    pml, tvar = eng.wait(t_b, len(RPS))
    ids, terms, t_end, sub = reqs[3]
    ref = oracle.run_layer(yet, sub, terms, seed=12, trials=np.arange(t_end))
    rpml, rtvar = oracle.pml_tvar(ref["ylt"], RPS)
    assert np.allclose(pml, rpml, rtol=PML_TOL) and np.allclose(tvar, rtvar, rtol=PML_TOL)
    for t in t_a:  # finished by the steps that ran before t_b's
        assert eng.poll(t, len(RPS)) is not None
    # a timeout that has passed before the first step: the request stays queued
    t_c = eng.submit(ids, terms, 13, t_end, RPS)
    with pytest.raises(ara.AraError) as e:
        eng.wait(t_c, len(RPS), timeout_ns=1)
    assert e.value.code == ara.ARA_ETIMEOUT
    assert eng.wait(t_c, len(RPS)) is not None
