"""GPU tests of the serving loop (ara_submit / ara_serve_step / ara_poll /
ara_wait): continuous batching of layer requests over trial chunks.

Each request's PML/TVaR against the FP64 oracle on its own trial prefix (1e-4
relative); results bit-identical alone and in a mix of requests; a short
request submitted while a long one is in flight finishes first; the rules that
form a round's passes; admission by the HBM budget (a request that does not
fit yet waits, one that can never fit is refused at submit); errors.
"""

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


@pytest.fixture(scope="module")
def long_world():
    # 900,000 trials x Poisson(20) over 50,000 events: a whole-YET request spans several chunks
    yet = synth.make_yet(900_000, 20.0, 50_000, 611)
    pool = synth.make_elt_pool(6, 3000, 50_000, 612)
    return yet, pool


def _load(eng, yet, pool):
    eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)
    eng.load_pool(pool)


def _serve_all(eng, reqs, seed=0):
    tickets = [eng.submit(ids, terms, seed, t_end, RPS) for ids, terms, t_end, _ in reqs]
    return [eng.wait(tk, len(RPS)) for tk in tickets]


def test_served_requests_match_the_oracle(eng, world):
    yet, pool, reqs = world
    _load(eng, yet, pool)
    got = _serve_all(eng, reqs, seed=3)
    for (ids, terms, t_end, sub), res in zip(reqs, got):
        ref = oracle.run_layer(yet, sub, terms, seed=3, trials=np.arange(t_end))
        pml, tvar = oracle.pml_tvar(ref["ylt"], RPS)
        assert np.allclose(res[0], pml, rtol=PML_TOL, atol=1e-9)
        assert np.allclose(res[1], tvar, rtol=PML_TOL, atol=1e-9)
    st = eng.serve_stats()
    assert st["queued"] == 0 and st["active"] == 0 and st["rounds_in_flight"] == 0


def test_results_identical_alone_and_in_a_mix(eng, world):
    yet, pool, reqs = world
    _load(eng, yet, pool)
    mixed = _serve_all(eng, reqs, seed=7)
    for req, res in zip(reqs, mixed):
        alone = _serve_all(eng, [req], seed=7)
        assert np.array_equal(alone[0][0], res[0]) and np.array_equal(alone[0][1], res[1])


def test_batched_selects_give_the_selects_bits(eng, world):
    """The requests that a pass finishes get their PML/TVaR from one batched
    select.  40 requests at once (passes of 32 and 8) with 1, 2, 5 or 16 return
    periods (one to four groups of periods each, so that a pass's selects span
    two batches); each result equals ara_pml_tvar over the request's year losses
    from ara_run_layers, bit for bit."""
    yet, pool, reqs = world
    _load(eng, yet, pool)
    rp_sets = [(10.0,), (10.0, 40.0), (2.0, 5.0, 10.0, 40.0, 100.0), tuple(np.geomspace(1.0, 900.0, 16))]
    subs = [(*reqs[i % len(reqs)][:3], rp_sets[i % 4]) for i in range(40)]
    s0 = eng.serve_stats()
    tks = [eng.submit(ids, terms, 13, t_end, rps) for ids, terms, t_end, rps in subs]
    got = [eng.wait(tk, len(rps)) for tk, (_, _, _, rps) in zip(tks, subs)]
    assert eng.serve_stats()["passes_launched"] - s0["passes_launched"] == 2
    for (ids, terms, t_end, rps), res in zip(subs, got):
        ylt = np.zeros((1, t_end))
        eng.run_layers([(ids, terms)], 13, 0, t_end, ylt)
        pml, tvar = eng.pml_tvar(ylt[0], rps)
        assert np.array_equal(pml, res[0]) and np.array_equal(tvar, res[1])


def test_a_short_request_overtakes_a_long_one_in_flight(eng, long_world):
    """A whole-YET request is launched; a 10,000-trial request submitted while its
    first round is on the device joins the next round and finishes first.  Both
    results are bit-identical to each request served alone."""
    yet, pool = long_world
    _load(eng, yet, pool)
    chunk = eng.serve_stats()["chunk_trials"]
    assert yet.n_trials > 3 * chunk
    long_ids, short_ids = pool.elt_ids[:4], pool.elt_ids[2:5]
    terms = (2e5, 5e6, 1e6, 1e9)
    t_long = eng.submit(long_ids, terms, 5, yet.n_trials, RPS)
    assert eng.serve_step() == 0  # launches the long request's first round and returns
    assert eng.serve_stats()["rounds_in_flight"] >= 1
    t_short = eng.submit(short_ids, terms, 5, 10_000, RPS)
    order, res = [], {}
    while len(order) < 2:
        eng.serve_step()
        for tk in (t_long, t_short):
            if tk not in res:
                r = eng.poll(tk, len(RPS))
                if r is not None:
                    res[tk] = r
                    order.append(tk)
    assert order == [t_short, t_long]
    alone_long = _serve_all(eng, [(long_ids, terms, yet.n_trials, None)], seed=5)[0]
    alone_short = _serve_all(eng, [(short_ids, terms, 10_000, None)], seed=5)[0]
    for a, b in ((alone_long, res[t_long]), (alone_short, res[t_short])):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # the short request against the oracle
    sub = pool.subset([int(i) for i in short_ids])
    ref = oracle.run_layer(yet, sub, terms, seed=5, trials=np.arange(10_000))
    pml, tvar = oracle.pml_tvar(ref["ylt"], RPS)
    assert np.allclose(res[t_short][0], pml, rtol=PML_TOL) and np.allclose(res[t_short][1], tvar, rtol=PML_TOL)


def test_rounds_follow_the_rules(eng, world):
    yet, pool, reqs = world
    _load(eng, yet, pool)
    ids, terms, t_end, _ = reqs[0]
    # 40 requests at the same chunk, one seed: passes of at most 32 layers, one round
    s0 = eng.serve_stats()
    tk = [eng.submit(ids, terms, 0, t_end, RPS) for _ in range(40)]
    res = [eng.wait(t, len(RPS)) for t in tk]
    s1 = eng.serve_stats()
    assert s1["passes_launched"] - s0["passes_launched"] == 2
    assert s1["rounds_launched"] - s0["rounds_launched"] == 1
    assert all(np.array_equal(res[0][0], r[0]) and np.array_equal(res[0][1], r[1]) for r in res)
    # one seed per pass: two seeds share the round in two passes
    a = [eng.submit(ids, terms, 1, t_end, RPS) for _ in range(3)]
    b = [eng.submit(ids, terms, 2, t_end, RPS) for _ in range(3)]
    assert eng.poll(a[0], len(RPS)) is None
    for t in a + b:
        eng.wait(t, len(RPS))
    s2 = eng.serve_stats()
    assert s2["passes_launched"] - s1["passes_launched"] == 2
    assert s2["rounds_launched"] - s1["rounds_launched"] == 1


def test_admission_follows_the_hbm_budget(world):
    """Under a budget whose arena holds one large request but not two, a second
    large request waits for the first to finish (it is not failed) and the small
    requests behind it go first; every result is bit-identical to serving it
    alone without a budget; a request that could never fit is refused at submit
    with ARA_ENOMEM."""
    from paper_1501_06326_gb300 import ara

    yet, pool, reqs = world
    free_ctx = ara.Ara(0)
    _load(free_ctx, yet, pool)
    probe = ara.Ara(0, 1 << 40)  # a budget that binds nothing: arena = budget - used - workspace
    _load(probe, yet, pool)
    fixed = (1 << 40) - probe.serve_stats()["arena_bytes"]
    probe.close()
    big, small = 1000, 100
    arena = 8 * big + 8 * big // 2  # one big request (8 KB), not two
    eng = ara.Ara(0, fixed + arena)
    _load(eng, yet, pool)
    assert 8 * big <= eng.serve_stats()["arena_bytes"] < 16 * big
    ids, terms, _, _ = reqs[1]
    tk = [eng.submit(ids, terms, 4, t, RPS) for t in (big, big, small, small)]
    eng.serve_step()
    st = eng.serve_stats()
    assert st["active"] == 3 and st["queued"] == 1  # the second big request waits
    res = [eng.wait(t, len(RPS)) for t in tk]
    for t_end, r in zip((big, big, small, small), res):
        alone = free_ctx.wait(free_ctx.submit(ids, terms, 4, t_end, RPS), len(RPS))
        assert np.array_equal(alone[0], r[0]) and np.array_equal(alone[1], r[1])
    bad = ara.Ara(0, fixed + 4096)
    _load(bad, yet, pool)
    with pytest.raises(ara.AraError) as e:
        bad.submit(ids, terms, 4, big, RPS)
    assert e.value.code == ara.ARA_ENOMEM
    for e_ in (eng, bad, free_ctx):
        e_.close()


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
    # the YET cannot be replaced under queued requests
    tk = eng.submit(ids, terms, 0, t_end, RPS)
    with pytest.raises(ara.AraError) as e:
        eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)
    assert e.value.code == ara.ARA_EINVAL
    eng.wait(tk, len(RPS))
    eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)


def test_wait_serves_until_the_request_is_done(eng, world):
    from paper_1501_06326_gb300 import ara

    yet, pool, reqs = world
    _load(eng, yet, pool)
    t_a = [eng.submit(ids, terms, 11, t_end, RPS) for ids, terms, t_end, _ in reqs[:3]]
    t_b = eng.submit(reqs[3][0], reqs[3][1], 12, reqs[3][2], RPS)
    pml, tvar = eng.wait(t_b, len(RPS))
    ids, terms, t_end, sub = reqs[3]
    ref = oracle.run_layer(yet, sub, terms, seed=12, trials=np.arange(t_end))
    rpml, rtvar = oracle.pml_tvar(ref["ylt"], RPS)
    assert np.allclose(pml, rpml, rtol=PML_TOL) and np.allclose(tvar, rtvar, rtol=PML_TOL)
    for t in t_a:  # they shared t_b's round
        assert eng.wait(t, len(RPS)) is not None
    # a timeout that has passed before the first step: the request stays pending
    t_c = eng.submit(ids, terms, 13, t_end, RPS)
    with pytest.raises(ara.AraError) as e:
        eng.wait(t_c, len(RPS), timeout_ns=1)
    assert e.value.code == ara.ARA_ETIMEOUT
    assert eng.wait(t_c, len(RPS)) is not None


def test_direct_selects_while_rounds_are_in_flight(eng, world):
    """ara_pml_tvar on the same context while serving rounds are in flight: the
    requests' selects run on their own stream with their own scratch, so the
    served results equal those of serving alone, and the direct calls match
    the oracle."""
    yet, pool, reqs = world
    _load(eng, yet, pool)
    alone = _serve_all(eng, reqs[:6], seed=21)
    tickets = [eng.submit(ids, terms, 21, t_end, RPS) for ids, terms, t_end, _ in reqs[:6]]
    rng = np.random.default_rng(22)
    done = {}
    while len(done) < len(tickets):
        eng.serve_step()
        y = np.round(rng.lognormal(5.0, 2.0, int(rng.integers(10, 20_000))), 2)
        pml, tvar = eng.pml_tvar(y, RPS)
        rpml, rtvar = oracle.pml_tvar(y, RPS)
        assert np.array_equal(pml, rpml) and np.allclose(tvar, rtvar, rtol=1e-12, atol=0)
        for tk in tickets:
            if tk not in done:
                r = eng.poll(tk, len(RPS))
                if r is not None:
                    done[tk] = r
    for a, tk in zip(alone, tickets):
        assert np.array_equal(a[0], done[tk][0]) and np.array_equal(a[1], done[tk][1])


def test_served_through_the_yet_index(world):
    """Serving with the YET's event-major index built (the passes take the
    indexed work item) gives each request the bits it gets without it; the
    index cannot be built while requests are queued."""
    from paper_1501_06326_gb300 import ara

    yet, pool, reqs = world
    plain = ara.Ara(0)
    _load(plain, yet, pool)
    want = _serve_all(plain, reqs, seed=31)
    plain.close()
    e = ara.Ara(0)
    _load(e, yet, pool)
    tk = e.submit(reqs[0][0], reqs[0][1], 31, reqs[0][2], RPS)
    with pytest.raises(ara.AraError) as err:
        e.build_yet_index()
    assert err.value.code == ara.ARA_EINVAL
    e.wait(tk, len(RPS))
    e.build_yet_index()
    got = _serve_all(e, reqs, seed=31)
    assert e.stats()["batch_item"] == ara.ARA_BATCH_ITEM_INDEXED
    for a, b in zip(want, got):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    e.close()
