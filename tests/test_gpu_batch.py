"""GPU parity of batched layers (ara_run_layers: several layers in one pass
over the YET) against the FP64 oracle run layer by layer, and against the
single-layer path.  Same tolerances as the single-layer parity tests: each
year loss within 1e-5 of max(|Y|, gross loss) of its layer's oracle run.
"""

import numpy as np
import pytest

import oracle
from paper_1501_06326_gb300 import synth

pytestmark = pytest.mark.gpu

YLT_TOL = 1e-5


@pytest.fixture(scope="module")
def eng():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1501_06326_gb300 import ara

    e = ara.Ara(0)
    yield e
    e.close()


def check_ylt(ylt, ref, tol=YLT_TOL):
    scale = np.maximum(np.abs(ref["ylt"]), ref["gross"])
    err = np.abs(ylt - ref["ylt"])
    bad = err > tol * scale
    worst = float(np.max(err / np.where(scale > 0, scale, 1.0))) if err.size else 0.0
    assert not bad.any(), f"{bad.sum()} trials out of tolerance, worst {worst:.3e}"
    return worst


def _batch_case(n_trials, catalogue, mean_events, n_elts, entries, n_layers, max_elts, seed, recipe="plain"):
    yet = synth.make_yet(n_trials, mean_events, catalogue, seed)
    pool = synth.make_elt_pool(n_elts, entries, catalogue, seed + 1, recipe=recipe)
    layer_ids = synth.draw_layers(n_layers, pool.elt_ids, max_elts, seed + 2)
    layers = []
    for ids in layer_ids:
        sub = pool.subset([int(np.flatnonzero(pool.elt_ids == i)[0]) for i in ids])
        layers.append((ids, oracle.calibrate_layer_terms(yet, sub), sub))
    return yet, pool, layers


def _run_batch(eng, yet, pool, layers, seed, t0=0, t1=None, index=False, **kw):
    t1 = yet.n_trials if t1 is None else t1
    eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)
    if index:
        eng.build_yet_index()
    eng.load_pool(pool)
    out = np.zeros((len(layers), t1 - t0))
    eng.run_layers([(ids, terms) for ids, terms, _ in layers], seed, t0, t1, out, **kw)
    return out


@pytest.fixture(scope="module")
def small_batch():
    # 1,000 trials x Poisson(100) over a catalogue of 10,000; a pool of 12 ELTs x 1,000
    # records; 6 layers of 1..8 ELTs (overlapping), terms per layer
    return _batch_case(1000, 10_000, 100.0, 12, 1000, 6, 8, 4242)


def test_batch_matches_oracle_layer_by_layer(eng, small_batch):
    yet, pool, layers = small_batch
    for seed in (0, 77):
        out = _run_batch(eng, yet, pool, layers, seed)
        for l, (ids, terms, sub) in enumerate(layers):
            ref = oracle.run_layer(yet, sub, terms, seed=seed)
            check_ylt(out[l], ref)


def test_batch_matches_the_single_layer_path(eng, small_batch):
    # the two paths differ only in the FP32 rounding of multi-ELT event sums and in
    # how a trial's sum is carried, so they agree well inside the oracle tolerance
    # (scaled, as there, by the trial's gross loss: terms are 1-Lipschitz)
    yet, pool, layers = small_batch
    out = _run_batch(eng, yet, pool, layers, 5)
    for l, (ids, terms, sub) in enumerate(layers):
        single = np.zeros(yet.n_trials)
        eng.run_layer(ids, terms, 5, 0, yet.n_trials, single)
        gross = oracle.run_layer(yet, sub, terms, seed=5)["gross"]
        scale = np.maximum(np.abs(single), gross)
        assert np.all(np.abs(out[l] - single) <= 1e-6 * scale + 1e-300)


def test_batch_is_deterministic_and_order_free(eng, small_batch):
    yet, pool, layers = small_batch
    a = _run_batch(eng, yet, pool, layers, 3)
    b = _run_batch(eng, yet, pool, layers, 3)
    assert np.array_equal(a, b)
    # listing the layers in another order permutes the outputs exactly
    perm = [3, 0, 5, 1, 4, 2]
    c = _run_batch(eng, yet, pool, [layers[i] for i in perm], 3)
    assert np.array_equal(c, a[perm])


def test_batch_subrange_primary_only_and_halley(eng, small_batch):
    yet, pool, layers = small_batch
    t0, t1 = 137, 911
    out = _run_batch(eng, yet, pool, layers, 9, t0, t1, primary_only=True)
    for l, (ids, terms, sub) in enumerate(layers):
        ref = oracle.run_layer(yet, sub, terms, seed=9, primary_only=True, trials=np.arange(t0, t1))
        check_ylt(out[l], ref)
    out = _run_batch(eng, yet, pool, layers, 9, 0, 300, newton_only=True)
    for l, (ids, terms, sub) in enumerate(layers):
        ref = oracle.run_layer(yet, sub, terms, seed=9, trials=np.arange(0, 300))
        check_ylt(out[l], ref)


def test_batch_of_one_layer_and_of_full_layers(eng):
    # one layer; then 32 layers, all 32 ELTs each (the batch limits), over a small YET
    yet, pool, layers = _batch_case(300, 5000, 60.0, 32, 400, 1, 32, 777)
    out = _run_batch(eng, yet, pool, layers, 1)
    check_ylt(out[0], oracle.run_layer(yet, layers[0][2], layers[0][1], seed=1))
    ids = pool.elt_ids
    terms = oracle.calibrate_layer_terms(yet, pool)
    full = [(ids, terms, pool)] * 32
    out = _run_batch(eng, yet, pool, full, 1)
    ref = oracle.run_layer(yet, pool, terms, seed=1)
    for l in range(32):
        check_ylt(out[l], ref)


def test_paper_shaped_batch_sampled(eng):
    # the paper-1m YET (first 2,000 trials), a pool of 64 ELTs x 10,000 records,
    # 16 layers of 1..32 ELTs: the shapes of the batched workload
    spec = synth.WORKLOADS["paper-1m"]
    yet = synth.make_yet(2000, spec["mean_events"], spec["catalogue"], spec["seed"])
    pool = synth.make_elt_pool(64, spec["entries"], spec["catalogue"], spec["seed"] + 7)
    layer_ids = synth.draw_layers(16, pool.elt_ids, 32, spec["seed"] + 8)
    layers = []
    for ids in layer_ids:
        sub = pool.subset([int(np.flatnonzero(pool.elt_ids == i)[0]) for i in ids])
        layers.append((ids, oracle.calibrate_layer_terms(yet, sub), sub))
    out = _run_batch(eng, yet, pool, layers, 0)
    for l, (ids, terms, sub) in enumerate(layers):
        check_ylt(out[l], oracle.run_layer(yet, sub, terms, seed=0))


def test_a_layer_alone_and_in_a_batch_agree(eng):
    # each layer of a 16-layer batch (about 320 hit records per trial) against the
    # layer alone (at most about 160): the same fixed-point sums, so each layer's
    # year losses are identical bit for bit
    spec = synth.WORKLOADS["paper-1m"]
    yet = synth.make_yet(1200, spec["mean_events"], spec["catalogue"], spec["seed"])
    pool = synth.make_elt_pool(64, spec["entries"], spec["catalogue"], spec["seed"] + 7)
    layer_ids = synth.draw_layers(16, pool.elt_ids, 32, spec["seed"] + 8)
    layers = [(ids, (50.0, 5e6, 1e4, 5e7), None) for ids in layer_ids]
    both = _run_batch(eng, yet, pool, layers, 5)
    for l, layer in enumerate(layers):
        alone = _run_batch(eng, yet, pool, [layer], 5)
        assert np.array_equal(alone[0], both[l])
    assert np.count_nonzero(both) > both.size // 2


def test_batch_errors(eng, small_batch):
    from paper_1501_06326_gb300 import ara

    yet, pool, layers = small_batch
    eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)
    eng.load_pool(pool)
    out = np.zeros((40, 10))
    spec = [(l[0], l[1]) for l in layers]
    with pytest.raises(ara.AraError) as e:  # too many layers
        eng.run_layers(spec * 7, 0, 0, 10, out)
    assert e.value.code == ara.ARA_EINVAL
    with pytest.raises(ara.AraError) as e:  # an ELT that is not loaded
        eng.run_layers(spec + [([999], spec[0][1])], 0, 0, 10, out)
    assert e.value.code == ara.ARA_ENOTLOADED
    with pytest.raises(ara.AraError) as e:  # bad range
        eng.run_layers(spec, 0, 5, 5, out)
    assert e.value.code == ara.ARA_EINVAL
    big = synth.make_elt_pool(70, 20, yet.catalogue_size, 5)
    big.elt_ids = big.elt_ids + 1000
    eng.load_pool(big)
    wide = [(big.elt_ids[:32], spec[0][1]), (big.elt_ids[32:64], spec[0][1]), (big.elt_ids[64:], spec[0][1])]
    with pytest.raises(ara.AraError) as e:  # union of 70 ELTs
        eng.run_layers(wide, 0, 0, 10, out)
    assert e.value.code == ara.ARA_EINVAL


def test_batch_with_empty_and_long_trials(eng):
    # empty trials (also at tile starts and ends), a trial longer than a gather step,
    # a partial last tile: the per-trial record ranges of each tile
    rng = np.random.default_rng(11)
    C = 2003
    lens = [0, 0, 3, 0, 4097, 0, 0, 0, 0, 1, 0, 250] + list(rng.integers(0, 40, 203)) + [0, 0]
    offsets = np.zeros(len(lens) + 1, np.int64)
    offsets[1:] = np.cumsum(lens)
    yet = synth.YET(offsets, rng.integers(0, C, offsets[-1]).astype(np.int32), C)
    pool = synth.make_elt_pool(6, 300, C, 31)
    layer_ids = [np.array([0, 1, 2], np.int32), np.array([2, 3, 4, 5], np.int32), np.array([5], np.int32)]
    layers = []
    for ids in layer_ids:
        sub = pool.subset([int(i) for i in ids])
        layers.append((ids, (100.0, 5e5, 1e3, 5e6), sub))
    out = _run_batch(eng, yet, pool, layers, 2)
    for l, (ids, terms, sub) in enumerate(layers):
        check_ylt(out[l], oracle.run_layer(yet, sub, terms, seed=2))
    out = _run_batch(eng, yet, pool, layers, 2, 3, 200)
    for l, (ids, terms, sub) in enumerate(layers):
        check_ylt(out[l], oracle.run_layer(yet, sub, terms, seed=2, trials=np.arange(3, 200)))


def test_autotuner_keeps_the_results_and_caches_its_choice(eng, small_batch):
    """ARA_AUTOTUNE measures the losses kernel's configurations on the first pass
    of a batch shape and keeps the fastest; every configuration gives the same
    bits, so the tuned pass equals the default one, and a later pass of the same
    shape (without the flag) reuses the choice."""
    yet, pool, layers = small_batch
    t1 = yet.n_trials - 3  # a shape of its own: nothing cached for it yet
    base = _run_batch(eng, yet, pool, layers, 5, t1=t1)
    assert eng.stats()["batch_tuned"] == 0
    tuned = _run_batch(eng, yet, pool, layers, 5, t1=t1, autotune=True)
    st = eng.stats()
    assert st["batch_tuned"] == 1 and st["batch_item"] in (0, 1, 2) and 2 <= st["batch_blocks_per_sm"] <= 16
    again = _run_batch(eng, yet, pool, layers, 5, t1=t1)
    st2 = eng.stats()
    assert st2["batch_tuned"] == 1
    assert (st2["batch_item"], st2["batch_blocks_per_sm"]) == (st["batch_item"], st["batch_blocks_per_sm"])
    assert np.array_equal(base, tuned) and np.array_equal(base, again)


def _run_items(eng, yet, pool, layers, seed, t0=0, t1=None, blocks=(0,), **kw):
    """The pass under each work item (and CTAs per SM) pinned by ara_set_batch_config;
    the indexed item after the YET's event-major index is built."""
    from paper_1501_06326_gb300 import ara

    outs = {}
    try:
        for item in (ara.ARA_BATCH_ITEM_TILE, ara.ARA_BATCH_ITEM_TRIAL, ara.ARA_BATCH_ITEM_DENSE,
                     ara.ARA_BATCH_ITEM_INDEXED):
            for b in blocks:
                eng.set_batch_config(item, b)
                outs[(item, b)] = _run_batch(eng, yet, pool, layers, seed, t0, t1,
                                             index=item == ara.ARA_BATCH_ITEM_INDEXED, **kw)
                st = eng.stats()
                assert st["batch_item"] == item and st["batch_tuned"] == 0
                assert b == 0 or st["batch_blocks_per_sm"] == b
    finally:
        eng.set_batch_config(ara.ARA_BATCH_AUTO)
    return outs


def _assert_same_bits(outs):
    ref = next(iter(outs.values()))
    for key, out in outs.items():
        assert np.array_equal(out, ref), f"work item / blocks {key} differs"
    return ref


def test_work_items_give_the_same_bits(eng):
    """The three losses kernels (a lane per record over a tile or over one trial,
    a lane per pair over a tile) add the same fixed-point numbers: identical
    bits on the paper-shaped 16-layer batch, at 2 CTAs per SM and at the most
    an SM holds; the dense kernel's result against the oracle."""
    spec = synth.WORKLOADS["paper-1m"]
    yet = synth.make_yet(600, spec["mean_events"], spec["catalogue"], spec["seed"] + 3)
    pool = synth.make_elt_pool(64, spec["entries"], spec["catalogue"], spec["seed"] + 7)
    layer_ids = synth.draw_layers(16, pool.elt_ids, 32, spec["seed"] + 8)
    layers = []
    for ids in layer_ids:
        sub = pool.subset([int(np.flatnonzero(pool.elt_ids == i)[0]) for i in ids])
        layers.append((ids, oracle.calibrate_layer_terms(yet, sub), sub))
    out = _assert_same_bits(_run_items(eng, yet, pool, layers, 4, blocks=(0, 2)))
    for l in (0, 7, 15):
        check_ylt(out[l], oracle.run_layer(yet, layers[l][2], layers[l][1], seed=4))
    # a subrange whose first tile is partial, and the Halley path for every pair
    _assert_same_bits(_run_items(eng, yet, pool, layers, 4, 13, 470))
    out = _assert_same_bits(_run_items(eng, yet, pool, layers[:4], 4, 0, 100, newton_only=True))
    for l in range(4):
        check_ylt(out[l], oracle.run_layer(yet, layers[l][2], layers[l][1], seed=4, trials=np.arange(100)))


def test_work_items_on_events_with_64_pairs(eng):
    """Every ELT of a 64-ELT pool holds every event of a 300-event catalogue, so
    each hit event has one pair per ELT (64, the most a record holds): long
    records cross the dense kernel's compute rounds and fill its pair ring; one
    trial has 4,097 such events.  32 layers of up to 32 ELTs; all work items
    agree, and match the oracle."""
    C = 300
    base = synth.make_yet(160, 40.0, C, 91)
    # and a 4,097-event trial (262,208 pairs in one tile) between empty ones
    rng = np.random.default_rng(94)
    lens = np.diff(base.offsets).tolist()
    lens[17:17] = [0, 4097, 0]
    offsets = np.zeros(len(lens) + 1, np.int64)
    offsets[1:] = np.cumsum(lens)
    ev = np.concatenate([base.event_ids[: base.offsets[17]], rng.integers(0, C, 4097).astype(np.int32),
                         base.event_ids[base.offsets[17]:]])
    yet = synth.YET(offsets, ev, C)
    pool = synth.make_elt_pool(64, C, C, 92)
    layer_ids = synth.draw_layers(32, pool.elt_ids, 32, 93)
    layers = []
    for ids in layer_ids:
        sub = pool.subset([int(np.flatnonzero(pool.elt_ids == i)[0]) for i in ids])
        layers.append((ids, oracle.calibrate_layer_terms(yet, sub), sub))
    out = _assert_same_bits(_run_items(eng, yet, pool, layers, 6))
    for l in (0, 13, 31):
        check_ylt(out[l], oracle.run_layer(yet, layers[l][2], layers[l][1], seed=6))


def test_work_items_on_empty_and_long_trials(eng):
    """Empty trials (at tile starts and ends), a 4,097-event trial, a partial last
    tile, and a subrange: all work items agree."""
    rng = np.random.default_rng(12)
    C = 2003
    lens = [0, 0, 3, 0, 4097, 0, 0, 0, 0, 1, 0, 250] + list(rng.integers(0, 40, 203)) + [0, 0]
    offsets = np.zeros(len(lens) + 1, np.int64)
    offsets[1:] = np.cumsum(lens)
    yet = synth.YET(offsets, rng.integers(0, C, offsets[-1]).astype(np.int32), C)
    pool = synth.make_elt_pool(6, 300, C, 32)
    layers = [(np.array(ids, np.int32), (100.0, 5e5, 1e3, 5e6), None)
              for ids in ([0, 1, 2], [2, 3, 4, 5], [5], [0, 5])]
    _assert_same_bits(_run_items(eng, yet, pool, layers, 2))
    _assert_same_bits(_run_items(eng, yet, pool, layers, 2, 3, 200))
    _assert_same_bits(_run_items(eng, yet, pool, layers, 2, 4, 5))


def test_indexed_pass_across_slices_and_grid_cells(eng):
    """A YET of 600,000 trials and 32 layers: the indexed pass runs in three
    slices of 262,144 trials, over three cells of the index's trial grid.
    Passes whose bounds are on the grid, inside a cell, inside one cell at both
    ends, and up to the YET's end; the indexed item gives the dense item's bits
    on each, and sampled trials match the oracle."""
    yet = synth.make_yet(600_000, 4.0, 3000, 61)
    pool = synth.make_elt_pool(8, 1000, 3000, 62)
    layer_ids = synth.draw_layers(32, pool.elt_ids, 4, 63)
    layers = [(ids, (10.0, 5e5, 1e2, 5e6), pool.subset([int(i) for i in ids])) for ids in layer_ids]
    for t0, t1 in ((0, 600_000), (262_144, 524_288), (70_001, 590_001), (262_145, 262_999),
                   (262_143, 600_000), (599_999, 600_000)):
        out = _assert_same_bits(_run_items(eng, yet, pool, layers, 8, t0, t1))
        assert np.count_nonzero(out) > 0
    # trials on both sides of a grid and slice bound, against the oracle
    t0, t1 = 262_000, 262_300
    out = _assert_same_bits(_run_items(eng, yet, pool, layers, 8, t0, t1))
    for l in (0, 11, 31):
        ids, terms, sub = layers[l]
        check_ylt(out[l], oracle.run_layer(yet, sub, terms, seed=8, trials=np.arange(t0, t1)))


def test_yet_index_by_radix_sort_where_an_event_is_frequent(eng):
    """An event in every trial of a 3,000-trial YET (a bucket of 3,000
    occurrences, above the bucket build's 2,048) has the index built by the
    radix sort; the indexed passes give the dense item's bits there, and on
    the same YET without the frequent event, built by buckets."""
    pool = synth.make_elt_pool(6, 400, 1500, 72)
    e_hot = int(pool.event_ids[0])  # an event of ELT 0
    base = synth.make_yet(3000, 30.0, 1500, 71)
    lens = np.diff(base.offsets) + 1
    offsets = np.zeros(len(lens) + 1, np.int64)
    offsets[1:] = np.cumsum(lens)
    ev = np.empty(offsets[-1], np.int32)
    for t in range(base.n_trials):  # the frequent event first in every trial, then the trial's own events
        ev[offsets[t]] = e_hot
        ev[offsets[t] + 1: offsets[t + 1]] = base.event_ids[base.offsets[t]: base.offsets[t + 1]]
    hot = synth.YET(offsets, ev, 1500)
    layers = [(np.array(ids, np.int32), (10.0, 5e5, 1e2, 5e6), None) for ids in ([0, 1], [1, 2, 3], [0, 4, 5])]
    for yet, method in ((hot, "radix sort"), (base, "buckets")):
        for t0, t1 in ((0, yet.n_trials), (17, 2903)):
            _assert_same_bits(_run_items(eng, yet, pool, layers, 3, t0, t1))
            assert eng.yet_index_info()["method"] == method


def test_batch_config_errors(eng):
    from paper_1501_06326_gb300 import ara

    for item, blocks in ((4, 0), (-2, 0), (ara.ARA_BATCH_ITEM_DENSE, -1), (ara.ARA_BATCH_ITEM_TILE, 17)):
        with pytest.raises(ara.AraError) as e:
            eng.set_batch_config(item, blocks)
        assert e.value.code == ara.ARA_EINVAL
    eng.set_batch_config(ara.ARA_BATCH_AUTO)


def test_yet_index_default_and_errors(eng, small_batch):
    """Without an index the indexed item is refused; once built, batched passes
    default to it and give the same bits as the dense item; a new YET load drops
    the index; building needs a YET."""
    from paper_1501_06326_gb300 import ara

    yet, pool, layers = small_batch
    fresh = ara.Ara(0)
    with pytest.raises(ara.AraError) as e:
        fresh.build_yet_index()
    assert e.value.code == ara.ARA_ENOTLOADED
    fresh.close()
    dense = _run_batch(eng, yet, pool, layers, 8)
    assert eng.stats()["batch_item"] == ara.ARA_BATCH_ITEM_DENSE
    eng.set_batch_config(ara.ARA_BATCH_ITEM_INDEXED)
    try:
        with pytest.raises(ara.AraError) as e:
            _run_batch(eng, yet, pool, layers, 8)
        assert e.value.code == ara.ARA_EINVAL
    finally:
        eng.set_batch_config(ara.ARA_BATCH_AUTO)
    indexed = _run_batch(eng, yet, pool, layers, 8, index=True)
    assert eng.stats()["batch_item"] == ara.ARA_BATCH_ITEM_INDEXED
    info = eng.yet_index_info()
    assert info["built"] and info["bytes"] >= 8 * yet.n_events and info["method"] == "buckets"
    assert np.array_equal(dense, indexed)
    eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)
    assert not eng.yet_index_info()["built"] and eng.yet_index_info()["method"] is None
