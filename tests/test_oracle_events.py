"""Pins of the oracle's per-event output (the Algorithm 1 loop of Section 2.2
emitting, per event occurrence held by the layer, its occurrence loss O_k and
the increment inc_k = A_k - A_{k-1} of the loss after aggregate terms; and
each trial's largest O_k): hand-worked rows of the tiny golden YET, the row
set against a brute-force membership test, the increments adding up to the
year loss, the bounds 0 <= inc_k <= O_k, and inc_k = O_k without aggregate
terms."""

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


def _golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def _tiny(g, elt_terms):
    trials = g["yet"]
    offsets = np.zeros(len(trials) + 1, np.int64)
    offsets[1:] = np.cumsum([len(t) for t in trials])
    yet = synth.YET(offsets, np.array([e for t in trials for e in t], np.int32), g["catalogue"])
    pids = g["elts"]["pool_ids"]
    ev, mu, offs = [], [], [0]
    for pid in pids:
        for e, m in g["elts"]["records"][str(pid)]:
            ev.append(e)
            mu.append(m)
        offs.append(len(ev))
    mu = np.array(mu, np.float32)
    terms = np.array([[_f(v) for v in elt_terms[str(p)]] for p in pids], np.float32)
    pool = synth.ELTPool(np.array(pids, np.int32), np.array(offs, np.int64), np.array(ev, np.int32), mu,
                         np.zeros_like(mu), (2.0 * mu).astype(np.float32), terms)
    return yet, pool


@pytest.mark.parametrize("case", ["layer_terms", "elt_terms"])
def test_hand_worked_event_rows(case):
    g = _golden()
    c = next(c for c in g["cases"] if c["name"] == case)
    want = g["event_rows"][case]
    yet, pool = _tiny(g, c["elt_terms"])
    r = oracle.run_layer_events(yet, pool, [_f(v) for v in c["layer_terms"]], seed=5)
    got = [[int(r["trial"][i]), int(r["k"][i]), int(r["event"][i]), r["occ"][i], r["inc"][i]]
           for i in range(len(r["trial"]))]
    assert got == [[int(a), int(b), int(e), float(o), float(d)] for a, b, e, o, d in want["rows"]]
    assert np.array_equal(r["max_occ"], np.array(want["max_occ"]))


@pytest.fixture(scope="module")
def world():
    yet = synth.make_yet(400, 60.0, 3000, 71)
    pool = synth.make_elt_pool(4, 500, 3000, 72, correlated=0.4)
    terms = oracle.calibrate_layer_terms(yet, pool)
    return yet, pool, terms


def test_rows_are_the_held_occurrences(world):
    yet, pool, terms = world
    r = oracle.run_layer_events(yet, pool, terms, seed=3, t_begin=17, t_end=350)
    held = np.zeros(yet.catalogue_size, bool)
    held[pool.event_ids] = True
    want_t, want_k = [], []
    for t in range(17, 350):
        ids = yet.event_ids[yet.offsets[t]:yet.offsets[t + 1]]
        for k in np.flatnonzero(held[ids]):
            want_t.append(t)
            want_k.append(k)
    assert np.array_equal(r["trial"], np.array(want_t)) and np.array_equal(r["k"], np.array(want_k))
    assert np.array_equal(r["event"], yet.event_ids[yet.offsets[r["trial"]] + r["k"]])


def test_increments_add_up_to_the_year_loss(world):
    yet, pool, terms = world
    r = oracle.run_layer_events(yet, pool, terms, seed=3)
    y = oracle.run_layer(yet, pool, terms, seed=3)["ylt"]
    sums = np.zeros(yet.n_trials)
    np.add.at(sums, r["trial"], r["inc"])
    assert np.allclose(sums, y, rtol=1e-12, atol=1e-9)
    assert np.all(r["inc"] >= 0.0) and np.all(r["inc"] <= r["occ"] * (1 + 1e-12) + 1e-9)
    occ_max = np.zeros(yet.n_trials)
    np.maximum.at(occ_max, r["trial"], r["occ"])
    assert np.array_equal(occ_max, r["max_occ"])
    assert np.all(r["occ"] <= terms[1])  # occurrence limit


def test_without_aggregate_terms_the_increment_is_the_occurrence_loss(world):
    yet, pool, terms = world
    r = oracle.run_layer_events(yet, pool, (terms[0], terms[1], 0.0, math.inf), seed=3)
    assert np.allclose(r["inc"], r["occ"], rtol=1e-12, atol=1e-6)
