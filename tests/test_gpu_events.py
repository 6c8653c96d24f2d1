"""GPU parity of the per-event output (ara_run_layer_events: the Algorithm 1
loop of Section 2.2 read per event) against the FP64 oracle.  Rows (trial,
event index, event id) bit-exact in (trial, k) order; O_k, inc_k and each
trial's largest O_k within 1e-5 of the trial's scale max(|Y|, gross loss),
the bar of the year losses; a trial's increments add up to the GPU's own year
loss; occurrence exceedance through ara_pml_tvar on max_occ within 1e-4."""

import numpy as np
import pytest

import oracle
from paper_1501_06326_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def eng():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1501_06326_gb300 import ara

    e = ara.Ara(0)
    yield e
    e.close()


def _load(eng, yet, pool):
    eng.load_yet(yet.offsets, yet.event_ids, yet.catalogue_size)
    eng.load_pool(pool)


def _run(eng, ids, terms, seed, t0, t1, cap=None, **kw):
    n = t1 - t0
    cap = (1 << 20) if cap is None else cap
    out = {"trial": np.full(cap, -7, np.int64), "k": np.full(cap, -7, np.int32), "event": np.full(cap, -7, np.int32),
           "occ": np.full(cap, -7.0), "inc": np.full(cap, -7.0), "max_occ": np.full(n, -7.0)}
    ylt = np.zeros(n)
    n_rows = eng.run_layer_events(ids, terms, seed, t0, t1, ylt, out["trial"], out["k"], out["event"], out["occ"],
                                  out["inc"], out["max_occ"], **kw)
    return n_rows, ylt, out


def check_rows(n_rows, ylt, got, ref, ref_layer, t0):
    assert n_rows == len(ref["trial"])
    assert np.array_equal(got["trial"][:n_rows], ref["trial"])
    assert np.array_equal(got["k"][:n_rows], ref["k"])
    assert np.array_equal(got["event"][:n_rows], ref["event"])
    scale_t = np.maximum(np.abs(ref_layer["ylt"]), ref_layer["gross"])
    scale = scale_t[ref["trial"] - t0]
    assert np.all(np.abs(got["occ"][:n_rows] - ref["occ"]) <= TOL * scale)
    assert np.all(np.abs(got["inc"][:n_rows] - ref["inc"]) <= TOL * scale)
    assert np.all(np.abs(got["max_occ"] - ref["max_occ"]) <= TOL * scale_t)
    # the GPU's increments add up to its own year losses
    sums = np.zeros(len(ylt))
    np.add.at(sums, got["trial"][:n_rows] - t0, got["inc"][:n_rows])
    assert np.all(np.abs(sums - ylt) <= 1e-9 * np.maximum(scale_t, 1.0))
    assert np.all(np.abs(ylt - ref_layer["ylt"]) <= TOL * scale_t)


@pytest.fixture(scope="module")
def world():
    # 1,000 trials x Poisson(100) over 10,000 events; 8 ELTs x 1,000 records (many
    # events held by several ELTs); a layer of 5 ELTs with percentile terms
    yet = synth.make_yet(1000, 100.0, 10_000, 801)
    pool = synth.make_elt_pool(8, 1000, 10_000, 802)
    ids = [0, 2, 3, 5, 7]
    sub = pool.subset(ids)
    terms = oracle.calibrate_layer_terms(yet, sub)
    return yet, pool, ids, sub, terms


def test_event_rows_match_the_oracle(eng, world):
    yet, pool, ids, sub, terms = world
    _load(eng, yet, pool)
    for seed in (0, 13):
        n_rows, ylt, got = _run(eng, ids, terms, seed, 0, yet.n_trials)
        ref = oracle.run_layer_events(yet, sub, terms, seed=seed)
        check_rows(n_rows, ylt, got, ref, oracle.run_layer(yet, sub, terms, seed=seed), 0)
        assert np.all(got["trial"][n_rows:] == -7)


def test_event_rows_halley_path_subrange_and_primary_only(eng, world):
    # every pair through the deferred Halley path; a trial range that starts and
    # ends inside tiles
    yet, pool, ids, sub, terms = world
    _load(eng, yet, pool)
    t0, t1 = 203, 517
    n_rows, ylt, got = _run(eng, ids, terms, 4, t0, t1, newton_only=True)
    trials = np.arange(t0, t1)
    ref = oracle.run_layer_events(yet, sub, terms, seed=4, t_begin=t0, t_end=t1)
    check_rows(n_rows, ylt, got, ref, oracle.run_layer(yet, sub, terms, seed=4, trials=trials), t0)
    n_rows, ylt, got = _run(eng, ids, terms, 4, t0, t1, primary_only=True)
    ref = oracle.run_layer_events(yet, sub, terms, seed=4, primary_only=True, t_begin=t0, t_end=t1)
    check_rows(n_rows, ylt, got, ref, oracle.run_layer(yet, sub, terms, seed=4, primary_only=True, trials=trials), t0)


def test_event_rows_aggregate_terms_beyond_fp32(eng, world):
    # an aggregate limit beyond the FP32 range: the running sums in FP64
    yet, pool, ids, sub, terms = world
    _load(eng, yet, pool)
    big = (terms[0], terms[1], terms[2], 1e300)
    n_rows, ylt, got = _run(eng, ids, big, 3, 0, yet.n_trials)
    ref = oracle.run_layer_events(yet, sub, big, seed=3)
    check_rows(n_rows, ylt, got, ref, oracle.run_layer(yet, sub, big, seed=3), 0)


def test_event_rows_empty_and_long_trials(eng):
    rng = np.random.default_rng(811)
    C = 2003
    lens = [0, 0, 3, 0, 4097, 0, 0, 0, 0, 1, 0, 250] + list(rng.integers(0, 40, 203)) + [0, 0]
    offsets = np.zeros(len(lens) + 1, np.int64)
    offsets[1:] = np.cumsum(lens)
    yet = synth.YET(offsets, rng.integers(0, C, offsets[-1]).astype(np.int32), C)
    pool = synth.make_elt_pool(4, 300, C, 812)
    _load(eng, yet, pool)
    ids = [0, 1, 2, 3]
    terms = (100.0, 5e5, 1e3, 5e6)
    n_rows, ylt, got = _run(eng, ids, terms, 2, 0, yet.n_trials)
    ref = oracle.run_layer_events(yet, pool, terms, seed=2)
    check_rows(n_rows, ylt, got, ref, oracle.run_layer(yet, pool, terms, seed=2), 0)
    assert got["max_occ"][0] == 0.0 and got["max_occ"][1] == 0.0


def test_capacity_and_device_outputs(eng, world):
    import torch

    yet, pool, ids, sub, terms = world
    _load(eng, yet, pool)
    n_all, ylt, full = _run(eng, ids, terms, 6, 0, yet.n_trials)
    # fewer rows than the range holds: the first ones are written, n_rows is the total
    n, _, part = _run(eng, ids, terms, 6, 0, yet.n_trials, cap=1000)
    assert n == n_all
    assert np.array_equal(part["trial"], full["trial"][:1000]) and np.array_equal(part["inc"], full["inc"][:1000])
    # device arrays give the same rows
    dev = torch.device("cuda", 0)
    d = {k: torch.full((n_all,), -1, dtype=dt, device=dev)
         for k, dt in (("trial", torch.int64), ("k", torch.int32), ("event", torch.int32), ("occ", torch.float64),
                       ("inc", torch.float64))}
    d_max = torch.zeros(yet.n_trials, dtype=torch.float64, device=dev)
    d_ylt = torch.zeros(yet.n_trials, dtype=torch.float64, device=dev)
    assert eng.run_layer_events(ids, terms, 6, 0, yet.n_trials, d_ylt, d["trial"], d["k"], d["event"], d["occ"],
                                d["inc"], d_max) == n_all
    torch.cuda.synchronize()
    for k in d:
        assert np.array_equal(d[k].cpu().numpy(), full[k][:n_all])
    assert np.array_equal(d_max.cpu().numpy(), full["max_occ"])
    assert np.array_equal(d_ylt.cpu().numpy(), ylt)
    # only max_occ requested
    m = np.zeros(yet.n_trials)
    assert eng.run_layer_events(ids, terms, 6, 0, yet.n_trials, np.zeros(yet.n_trials), max_occ=m) == n_all
    assert np.array_equal(m, full["max_occ"])


def test_occurrence_exceedance_pml(eng, world):
    # OEP: PML/TVaR of each trial's largest occurrence loss
    yet, pool, ids, sub, terms = world
    _load(eng, yet, pool)
    m = np.zeros(yet.n_trials)
    eng.run_layer_events(ids, terms, 1, 0, yet.n_trials, np.zeros(yet.n_trials), max_occ=m)
    rps = np.array([10.0, 50.0, 200.0])
    pml, tvar = np.zeros(3), np.zeros(3)
    eng.pml_tvar(m, rps, pml, tvar)
    ref_pml, ref_tvar = oracle.pml_tvar(oracle.run_layer_events(yet, sub, terms, seed=1)["max_occ"], rps)
    assert np.allclose(pml, ref_pml, rtol=1e-4) and np.allclose(tvar, ref_tvar, rtol=1e-4)


def test_paper_shaped_event_rows_sampled(eng):
    # the paper-1m YET (first 1,500 trials) and a layer of its 15 ELTs x 10,000 records
    spec = synth.WORKLOADS["paper-1m"]
    yet = synth.make_yet(1500, spec["mean_events"], spec["catalogue"], spec["seed"])
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["seed"],
                               recipe=spec["recipe"])
    _load(eng, yet, pool)
    terms = oracle.calibrate_layer_terms(yet, pool)
    n_rows, ylt, got = _run(eng, pool.elt_ids, terms, 0, 0, yet.n_trials)
    ref = oracle.run_layer_events(yet, pool, terms, seed=0)
    check_rows(n_rows, ylt, got, ref, oracle.run_layer(yet, pool, terms, seed=0), 0)


def test_event_rows_errors(eng, world):
    from paper_1501_06326_gb300 import ara

    yet, pool, ids, sub, terms = world
    _load(eng, yet, pool)
    with pytest.raises(ara.AraError) as e:
        eng.run_layer_events(ids, terms, 0, 0, 10, np.zeros(10), capacity=-1)
    assert e.value.code == ara.ARA_EINVAL
    with pytest.raises(ara.AraError) as e:
        eng.run_layer_events(ids, terms, 0, 5, 5, np.zeros(1))
    assert e.value.code == ara.ARA_EINVAL
