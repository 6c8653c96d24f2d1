"""Pins of the oracle's ARA loop (Algorithm 1, Section 2.2, with secondary
uncertainty inserted after the lookup as Section 3.3 states) and of its
PML/TVaR (Section 2.3).

Hand-summed year losses of tiny YETs (tests/golden/tiny_ara_cases.json),
closed-form secondary-uncertainty records, the sigma -> 0 limit, the
order-free identity of the year loss, monotonicity in the terms, ELT
permutation invariance, brute-force hit counts and brute-force sorting.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1501_06326_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_ara_cases.json")


def _f(v):
    return float("inf") if v == "inf" else float(v)


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def tiny_inputs(g, elt_terms=None):
    trials = g["yet"]
    offsets = np.zeros(len(trials) + 1, np.int64)
    offsets[1:] = np.cumsum([len(t) for t in trials])
    ids = np.array([e for t in trials for e in t], np.int32)
    yet = synth.YET(offsets=offsets, event_ids=ids, catalogue_size=g["catalogue"])
    pids = g["elts"]["pool_ids"]
    ev, mu, offs = [], [], [0]
    for pid in pids:
        recs = g["elts"]["records"][str(pid)]
        ev += [r[0] for r in recs]
        mu += [r[1] for r in recs]
        offs.append(len(ev))
    mu = np.array(mu, np.float32)
    terms = np.array([[_f(v) for v in (elt_terms or {}).get(str(p), [0.0, "inf", 1.0])] for p in pids], np.float32)
    pool = synth.ELTPool(
        elt_ids=np.array(pids, np.int32), rec_offsets=np.array(offs, np.int64),
        event_ids=np.array(ev, np.int32), mean=mu, sigma=np.zeros_like(mu),
        exposure=(2.0 * mu).astype(np.float32), terms=terms,
    )
    return yet, pool


@pytest.mark.parametrize("case", [c["name"] for c in golden()["cases"]])
def test_hand_summed_year_losses(case):
    g = golden()
    c = next(c for c in g["cases"] if c["name"] == case)
    yet, pool = tiny_inputs(g, c["elt_terms"])
    lt = [_f(v) for v in c["layer_terms"]]
    for primary_only in (True, False):  # sigma = 0 records: SU leaves the loss at mu
        r = oracle.run_layer(yet, pool, lt, seed=123, primary_only=primary_only)
        assert np.array_equal(r["ylt"], np.array(c["ylt"]))
        assert np.array_equal(r["gross"], np.array(c["gross"]))
        assert np.array_equal(r["hits"], np.array(c["hits"]))


@pytest.mark.parametrize("rec", golden()["su_closed_forms"]["records"], ids=lambda r: r["name"])
def test_secondary_uncertainty_closed_forms(rec):
    max_l = rec["max"]
    sigma = max_l * math.sqrt(rec["sigma_sq_over_max_sq"])
    n = 200
    offsets = np.arange(n + 1, dtype=np.int64)
    yet = synth.YET(offsets=offsets, event_ids=np.full(n, 2, np.int32), catalogue_size=4)
    pool = synth.ELTPool(
        elt_ids=np.array([5], np.int32), rec_offsets=np.array([0, 1], np.int64),
        event_ids=np.array([2], np.int32), mean=np.array([rec["mu"]], np.float32),
        sigma=np.array([sigma], np.float32), exposure=np.array([max_l], np.float32),
        terms=np.array([[0.0, np.inf, 1.0]], np.float32),
    )
    seed = 99
    r = oracle.run_layer(yet, pool, (0.0, np.inf, 0.0, np.inf), seed=seed)
    z = oracle.uniform_batch(seed, np.arange(n), np.zeros(n, np.int32), np.full(n, 5, np.int32))
    want = max_l * (z if rec["quantile"] == "z" else np.sqrt(z))
    # the record's float32 rounding moves the shapes by ~1e-7 relative
    assert np.allclose(r["ylt"], want, rtol=2e-6, atol=0)


def _su_under_terms_closed_form(c, z5, z8):
    """The year loss that tests/golden/tiny_ara_cases.json's su_under_terms
    states as a closed form of the two uniforms."""
    (r5, r8) = c["records"]
    occ_r, occ_l = c["layer_terms"][0], c["layer_terms"][1]

    def elt(rec, z):
        ret, lim, share = rec["terms"]
        loss = rec["max"] * (z if rec["quantile"] == "z" else np.sqrt(z))
        return share * np.minimum(np.maximum(loss - ret, 0.0), lim)

    return np.minimum(np.maximum(elt(r5, z5) + elt(r8, z8) - occ_r, 0.0), occ_l)


def test_secondary_uncertainty_sits_before_elt_terms():
    """Section 3.3: the Beta loss is drawn for the looked-up record, and the
    ELT financial terms (Section 2.2) act on the drawn loss, then the sum
    over ELTs, then the occurrence terms."""
    c = golden()["su_under_terms"]
    for h in c["hand_checks"]:
        got = _su_under_terms_closed_form(c, np.array(h["z"][0]), np.array(h["z"][1]))
        assert abs(float(got) - h["year_loss"]) <= 1e-9
    n = 400
    offsets = np.arange(n + 1, dtype=np.int64)
    yet = synth.YET(offsets=offsets, event_ids=np.full(n, 2, np.int32), catalogue_size=4)
    recs = c["records"]
    pool = synth.ELTPool(
        elt_ids=np.array([r["pool_id"] for r in recs], np.int32), rec_offsets=np.array([0, 1, 2], np.int64),
        event_ids=np.array([2, 2], np.int32), mean=np.array([r["mu"] for r in recs], np.float32),
        sigma=np.array([r["max"] * math.sqrt(r["sigma_sq_over_max_sq"]) for r in recs], np.float32),
        exposure=np.array([r["max"] for r in recs], np.float32),
        terms=np.array([r["terms"] for r in recs], np.float32),
    )
    lt = [_f(v) for v in c["layer_terms"]]
    seed = 31
    r = oracle.run_layer(yet, pool, lt, seed=seed)
    tr = np.arange(n)
    z5 = oracle.uniform_batch(seed, tr, np.zeros(n, np.int32), np.full(n, recs[0]["pool_id"], np.int32))
    z8 = oracle.uniform_batch(seed, tr, np.zeros(n, np.int32), np.full(n, recs[1]["pool_id"], np.int32))
    want = _su_under_terms_closed_form(c, z5, z8)
    # the records' float32 rounding moves the shapes by ~1e-7 relative; the
    # terms are 1-Lipschitz, so the year loss moves by at most that share of
    # the two maxima
    assert np.allclose(r["ylt"], want, rtol=0, atol=2e-6 * (recs[0]["max"] + recs[1]["max"]))
    # the case exercises every regime of both ELTs' terms and of the occurrence terms
    l5 = recs[0]["max"] * z5
    assert (l5 < 200).any() and ((l5 > 200) & (l5 < 700)).any() and (l5 > 700).any()
    l8 = recs[1]["max"] * np.sqrt(z8)
    assert (l8 < 50).any() and ((l8 > 50) & (l8 < 200)).any() and (l8 > 200).any()
    assert (want == 0).any() and ((want > 0) & (want < 400)).any()


def _small(n_trials=150, seed_shift=0):
    spec = synth.WORKLOADS["plain-1k"]
    yet = synth.make_yet(n_trials, spec["mean_events"], spec["catalogue"], spec["seed"] + seed_shift)
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["seed"] + seed_shift)
    return yet, pool


def test_sigma_to_zero_reduces_to_primary_uncertainty():
    yet, pool = _small(60)
    lt = oracle.calibrate_layer_terms(yet, pool)
    prim = oracle.run_layer(yet, pool, lt, primary_only=True)
    exact = synth.ELTPool(**{**pool.__dict__, "sigma": np.zeros_like(pool.sigma)})
    r0 = oracle.run_layer(yet, exact, lt, seed=1)
    assert np.array_equal(r0["ylt"], prim["ylt"])
    # small sigma: each loss moves by O(sigma), and the terms are 1-Lipschitz
    small = synth.ELTPool(**{**pool.__dict__, "sigma": (pool.sigma * 1e-3).astype(np.float32)})
    rs = oracle.run_layer(yet, small, lt, seed=1)
    bound = 1e-2 * prim["gross"] + 1e-9
    assert np.all(np.abs(rs["ylt"] - prim["ylt"]) <= bound)
    assert np.abs(rs["ylt"] - prim["ylt"]).max() > 0.0


def test_year_loss_is_aggregate_terms_of_total_occurrence_loss():
    # O_k >= 0 makes S non-decreasing, so Y = min(max(S_final - AggR, 0), AggL)
    yet, pool = _small(40)
    occ_r, occ_l, agg_r, agg_l = oracle.calibrate_layer_terms(yet, pool)
    r = oracle.run_layer(yet, pool, (occ_r, occ_l, agg_r, agg_l), seed=4)
    for t in range(yet.n_trials):
        g = oracle.event_losses(yet, pool, seed=4, primary_only=False, t_begin=t, t_end=t + 1)
        s = float(np.sum(np.minimum(np.maximum(g - occ_r, 0.0), occ_l)))
        y = min(max(s - agg_r, 0.0), agg_l)
        assert abs(r["ylt"][t] - y) <= 1e-12 * max(1.0, abs(y))


def test_event_order_within_a_trial_does_not_change_primary_year_loss():
    yet, pool = _small(80)
    lt = oracle.calibrate_layer_terms(yet, pool)
    base = oracle.run_layer(yet, pool, lt, primary_only=True)["ylt"]
    rng = np.random.default_rng(8)
    ids = yet.event_ids.copy()
    for t in range(yet.n_trials):
        lo, hi = yet.offsets[t], yet.offsets[t + 1]
        ids[lo:hi] = rng.permutation(ids[lo:hi])
    shuf = synth.YET(offsets=yet.offsets, event_ids=ids, catalogue_size=yet.catalogue_size)
    got = oracle.run_layer(shuf, pool, lt, primary_only=True)["ylt"]
    assert np.allclose(got, base, rtol=1e-12, atol=0)


def test_elt_order_within_a_layer_does_not_matter():
    yet, pool = _small(80)
    lt = oracle.calibrate_layer_terms(yet, pool)
    base = oracle.run_layer(yet, pool, lt, seed=3)
    perm = pool.subset([2, 0, 1])
    got = oracle.run_layer(yet, perm, lt, seed=3)
    assert np.allclose(got["ylt"], base["ylt"], rtol=1e-13, atol=0)
    assert np.array_equal(got["hits"], base["hits"])
    assert np.array_equal(got["hit_hash"], base["hit_hash"])


@pytest.mark.parametrize("which,direction", [(0, -1), (1, +1), (2, -1), (3, +1)])
def test_year_loss_monotone_in_each_term(which, direction):
    yet, pool = _small(100)
    lt = list(oracle.calibrate_layer_terms(yet, pool))
    base = oracle.run_layer(yet, pool, lt, seed=2)["ylt"]
    bumped = list(lt)
    bumped[which] = lt[which] * 1.3 + 1.0
    moved = oracle.run_layer(yet, pool, bumped, seed=2)["ylt"]
    assert np.all(direction * (moved - base) >= -1e-9)
    assert np.any(moved != base)


def test_hit_counts_brute_force():
    yet, pool = _small(50)
    r = oracle.run_layer(yet, pool, (0.0, np.inf, 0.0, np.inf), seed=0)
    sets = [set(pool.event_ids[pool.rec_offsets[j]:pool.rec_offsets[j + 1]].tolist()) for j in range(pool.n_elts)]
    for t in range(yet.n_trials):
        ev = yet.event_ids[yet.offsets[t]:yet.offsets[t + 1]]
        assert r["hits"][t] == sum(int(e) in s for e in ev for s in sets)


def test_trial_list_matches_full_run():
    yet, pool = _small(120)
    lt = oracle.calibrate_layer_terms(yet, pool)
    full = oracle.run_layer(yet, pool, lt, seed=5)
    pick = np.array([0, 7, 33, 119, 64], np.int64)
    part = oracle.run_layer(yet, pool, lt, seed=5, trials=pick)
    for key in ("ylt", "gross", "hits", "hit_hash"):
        assert np.array_equal(part[key], full[key][pick])


# ------------------------------------------------------------------ PML / TVaR
def _brute_pml_tvar(y, rps):
    order = np.lexsort((np.arange(y.size), -y))  # descending value, ascending index
    pml, tvar = [], []
    for rp in rps:
        m = min(max(int(math.ceil(y.size / rp)), 1), y.size)
        pml.append(y[order[m - 1]])
        tvar.append(math.fsum(y[order[:m]]) / m)
    return order, np.array(pml), np.array(tvar)


@pytest.mark.parametrize("n", [1, 7, 1000, 4099])
def test_pml_tvar_brute_force(n):
    rng = np.random.default_rng(n)
    y = np.round(rng.lognormal(5, 2, n), 1)  # rounding makes ties
    y[rng.random(n) < 0.3] = 0.0
    rps = np.array([2.0, 100.0, 250.0, 1e9])
    order, pml, tvar = _brute_pml_tvar(y, rps)
    assert np.array_equal(oracle.sort_desc(y), order)
    got_pml, got_tvar = oracle.pml_tvar(y, rps)
    assert np.array_equal(got_pml, pml)
    assert np.allclose(got_tvar, tvar, rtol=1e-15, atol=0)


def test_percentile_calibration_is_nearest_rank():
    yet, pool = _small(200)
    occ_r, occ_l, agg_r, agg_l = oracle.calibrate_layer_terms(yet, pool)
    g = oracle.event_losses(yet, pool, primary_only=True)
    assert occ_r == np.percentile(g, 50, method="inverted_cdf")
    assert occ_l == np.percentile(g, 99, method="inverted_cdf")
    s = oracle.run_layer(yet, pool, (occ_r, occ_l, 0.0, np.inf), primary_only=True)["ylt"]
    assert agg_r == np.percentile(s, 10, method="inverted_cdf")
    assert agg_l == np.percentile(s, 99, method="inverted_cdf")
    assert 0 < occ_r < occ_l and 0 <= agg_r < agg_l
