"""Seeded synthetic inputs for Aggregate Risk Analysis (ARA).

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's scripts.  It draws inputs only: it holds none of the method's
arithmetic (no lookup, no secondary uncertainty, no terms, no aggregation).

The proprietary industry YET/ELTs measured in the paper (Section 5: 800,000
trials x 1,000 events, one layer of 16 XELTs) are not available, so these
generators stand in for them with the shapes the paper describes:

* Year Event Table (Section 2.1 (i)): trials of ``Poisson(lambda)`` event
  occurrences, each event id uniform over a catalogue of ``C`` events, kept in
  time order.  Time stamps only fix the order of a trial's events (they enter
  the method nowhere else), and i.i.d. ids sorted by i.i.d. time stamps are
  again i.i.d., so the ids are stored directly in their (time) order and no
  time stamps are materialised.
* Event Loss Tables (Section 2.1 (ii), Section 3.1): each ELT holds
  ``entries`` distinct event ids drawn without replacement from the
  catalogue, sorted, with a mean loss ``mu ~ LogNormal(10, 2)``, an exposure
  (the maximum loss ``max_l``) ``mu * U(2, 20)`` and a standard deviation
  ``sigma = mu * U(0.1, 1.0)``.  ``sigma`` is clipped so that both shape
  parameters of the loss's Beta distribution stay >= ``shape_floor``; the
  clip uses only the textbook Beta moments (mean m, variance
  m (1 - m) / (a + b + 1)).
* The "stress" recipe draws the Beta shapes ``a, b`` log-uniform in
  ``[0.2, 50]`` and sets exposure and sigma from the same moments.

Every array is generated chunk-wise from ``numpy.random.SeedSequence([seed,
stream, chunk])`` so the result is independent of the thread count.
"""

from __future__ import annotations

import dataclasses
import math
from concurrent.futures import ThreadPoolExecutor
from typing import Optional

import numpy as np

_CHUNK = 1 << 24

# stream ids within one workload seed
_S_COUNTS, _S_IDS, _S_ELT, _S_LAYERS, _S_CORR = 1, 2, 3, 4, 5


@dataclasses.dataclass
class YET:
    """CSR Year Event Table: trial t owns ``event_ids[offsets[t]:offsets[t+1]]``."""

    offsets: np.ndarray  # int64 [N + 1]
    event_ids: np.ndarray  # int32 [E], time order within a trial
    catalogue_size: int

    @property
    def n_trials(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_events(self) -> int:
        return int(self.offsets[-1])


@dataclasses.dataclass
class ELTPool:
    """A pool of Event Loss Tables in CSR form.

    ELT ``i`` (pool id ``elt_ids[i]``) owns records
    ``rec_offsets[i]:rec_offsets[i+1]`` of ``event_ids/mean/sigma/exposure``;
    its event ids are strictly increasing.  ``terms`` holds the per-ELT
    financial terms (retention, limit, share) as float32 ``[n, 3]``.
    """

    elt_ids: np.ndarray  # int32 [n]
    rec_offsets: np.ndarray  # int64 [n + 1]
    event_ids: np.ndarray  # int32 [R]
    mean: np.ndarray  # float32 [R]
    sigma: np.ndarray  # float32 [R]
    exposure: np.ndarray  # float32 [R]
    terms: np.ndarray  # float32 [n, 3]: retention, limit, share
    sigma_c: Optional[np.ndarray] = None  # float32 [R]: correlated standard deviation (None: all zero)

    @property
    def n_elts(self) -> int:
        return int(self.elt_ids.shape[0])

    def subset(self, positions) -> "ELTPool":
        """The ELTs at the given pool positions, as a new pool (copies)."""
        positions = list(positions)
        ev, mu, sg, ex, sc, offs = [], [], [], [], [], [0]
        for p in positions:
            lo, hi = int(self.rec_offsets[p]), int(self.rec_offsets[p + 1])
            ev.append(self.event_ids[lo:hi])
            mu.append(self.mean[lo:hi])
            sg.append(self.sigma[lo:hi])
            ex.append(self.exposure[lo:hi])
            if self.sigma_c is not None:
                sc.append(self.sigma_c[lo:hi])
            offs.append(offs[-1] + hi - lo)
        cat = lambda xs, dt: (np.concatenate(xs) if xs else np.zeros(0, dt)).astype(dt)
        return ELTPool(
            elt_ids=self.elt_ids[positions].copy(),
            rec_offsets=np.asarray(offs, dtype=np.int64),
            event_ids=cat(ev, np.int32),
            mean=cat(mu, np.float32),
            sigma=cat(sg, np.float32),
            exposure=cat(ex, np.float32),
            terms=self.terms[positions].copy(),
            sigma_c=None if self.sigma_c is None else cat(sc, np.float32),
        )


def _rng(seed: int, stream: int, chunk: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream), int(chunk)]))


def _threads() -> int:
    import os

    return max(1, min(16, os.cpu_count() or 1))


def yet_offsets(n_trials: int, mean_events: float, seed: int) -> np.ndarray:
    """Trial offsets of a YET with Poisson(``mean_events``) events per trial."""
    counts = _rng(seed, _S_COUNTS).poisson(mean_events, size=n_trials).astype(np.int64)
    offsets = np.zeros(n_trials + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return offsets


def fill_yet_ids(out: np.ndarray, catalogue_size: int, seed: int) -> np.ndarray:
    """Fill ``out`` (int32, any length) with i.i.d. uniform event ids.

    ``out`` may be a numpy view of pinned host memory.  Chunk ``c`` of
    ``2**24`` ids always comes from the same sub-stream, so the content
    depends only on ``seed`` and the length.
    """
    n = int(out.shape[0])
    n_chunks = (n + _CHUNK - 1) // _CHUNK

    def fill(c: int) -> None:
        lo = c * _CHUNK
        hi = min(n, lo + _CHUNK)
        out[lo:hi] = _rng(seed, _S_IDS, c).integers(0, catalogue_size, size=hi - lo, dtype=np.int32)

    if n_chunks <= 1:
        for c in range(n_chunks):
            fill(c)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(fill, range(n_chunks)))
    return out


def make_yet(n_trials: int, mean_events: float, catalogue_size: int, seed: int) -> YET:
    offsets = yet_offsets(n_trials, mean_events, seed)
    ids = np.empty(int(offsets[-1]), dtype=np.int32)
    fill_yet_ids(ids, catalogue_size, seed)
    return YET(offsets=offsets, event_ids=ids, catalogue_size=int(catalogue_size))


def _clip_sigma_for_shape_floor(mean, exposure, sigma, shape_floor):
    """Largest sigma for which both Beta shapes stay >= shape_floor.

    With m = mean / exposure and s = sigma / exposure, the Beta with mean m
    and variance s^2 has a + b = m (1 - m) / s^2 - 1, a = m (a + b),
    b = (1 - m)(a + b).  Requiring min(a, b) >= f means
    a + b >= f / min(m, 1 - m), i.e. s^2 <= m (1 - m) / (1 + f / min(m, 1 - m)).
    """
    m = mean / exposure
    smax = exposure * np.sqrt(m * (1.0 - m) / (1.0 + shape_floor / np.minimum(m, 1.0 - m)))
    return np.minimum(sigma, smax * (1.0 - 1e-6))


def make_elt_pool(
    n_elts: int,
    entries: int,
    catalogue_size: int,
    seed: int,
    recipe: str = "plain",
    first_id: int = 0,
    shape_floor: float = 0.05,
    stress_range=(0.2, 50.0),
    correlated: float = 0.0,
) -> ELTPool:
    """A pool of ``n_elts`` ELTs with ``entries`` distinct events each.

    ``recipe="plain"``: mu ~ LogNormal(10, 2), exposure = mu * U(2, 20),
    sigma = mu * U(0.1, 1.0) clipped so that min(a, b) >= ``shape_floor``.
    ``recipe="stress"``: a, b ~ log-uniform over ``stress_range``; exposure
    and sigma follow from the Beta moments.  Pool ids are
    ``first_id .. first_id + n_elts - 1``; terms are the identity
    (retention 0, limit +inf, share 1).
    ``correlated > 0`` splits each record's sigma into an independent and a
    correlated part (Section 3.1): sigma_C = sigma * u, sigma_I = sigma - sigma_C
    with u ~ U(0, correlated) per record, so sigma_I + sigma_C (and the Beta
    shapes) are those of the recipe.
    """
    if entries > catalogue_size:
        raise ValueError("an ELT cannot hold more distinct events than the catalogue")
    ev_l, mu_l, sg_l, ex_l = [], [], [], []
    for j in range(n_elts):
        rng = _rng(seed, _S_ELT, j)
        ev = np.sort(rng.choice(catalogue_size, size=entries, replace=False)).astype(np.int32)
        mu = rng.lognormal(mean=10.0, sigma=2.0, size=entries)
        if recipe == "plain":
            ex = mu * rng.uniform(2.0, 20.0, size=entries)
            sg = mu * rng.uniform(0.1, 1.0, size=entries)
            sg = _clip_sigma_for_shape_floor(mu, ex, sg, shape_floor)
        elif recipe == "stress":
            lo, hi = math.log(stress_range[0]), math.log(stress_range[1])
            a = np.exp(rng.uniform(lo, hi, size=entries))
            b = np.exp(rng.uniform(lo, hi, size=entries))
            m = a / (a + b)
            ex = mu / m
            sg = ex * np.sqrt(m * (1.0 - m) / (a + b + 1.0))
        else:
            raise ValueError(f"unknown recipe {recipe!r}")
        ev_l.append(ev)
        mu_l.append(mu.astype(np.float32))
        sg_l.append(sg.astype(np.float32))
        ex_l.append(ex.astype(np.float32))
    offs = np.zeros(n_elts + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(e) for e in ev_l])
    terms = np.tile(np.array([0.0, np.inf, 1.0], dtype=np.float32), (n_elts, 1))
    sigma = np.concatenate(sg_l) if sg_l else np.zeros(0, np.float32)
    sigma_c = None
    if correlated > 0.0:
        u = _rng(seed, _S_CORR).uniform(0.0, correlated, size=sigma.shape[0])
        sigma_c = (sigma.astype(np.float64) * u).astype(np.float32)
        sigma = (sigma.astype(np.float64) - sigma_c).astype(np.float32)
    return ELTPool(
        elt_ids=np.arange(first_id, first_id + n_elts, dtype=np.int32),
        rec_offsets=offs,
        event_ids=np.concatenate(ev_l) if ev_l else np.zeros(0, np.int32),
        mean=np.concatenate(mu_l) if mu_l else np.zeros(0, np.float32),
        sigma=sigma,
        exposure=np.concatenate(ex_l) if ex_l else np.zeros(0, np.float32),
        terms=terms,
        sigma_c=sigma_c,
    )


def draw_layers(n_layers: int, pool_ids: np.ndarray, max_elts: int, seed: int):
    """Uneven layers: |J| ~ U{1..max_elts} distinct pool ids per layer."""
    rng = _rng(seed, _S_LAYERS)
    out = []
    for _ in range(n_layers):
        k = int(rng.integers(1, max_elts + 1))
        out.append(np.sort(rng.choice(pool_ids, size=k, replace=False)).astype(np.int32))
    return out


# Workloads (shapes of the paper's Section 5 workload and the stated configurations).
WORKLOADS = {
    "plain-1k": dict(
        n_trials=1_000, mean_events=100.0, catalogue=10_000, n_elts=3, entries=1_000,
        recipe="plain", seed=20150126, return_periods=(100.0, 250.0),
    ),
    "paper-1m": dict(
        n_trials=1_000_000, mean_events=1000.0, catalogue=2_000_000, n_elts=15, entries=10_000,
        recipe="plain", seed=20150127, return_periods=(100.0, 250.0),
    ),
    "stress-1m": dict(
        n_trials=1_000_000, mean_events=1000.0, catalogue=2_000_000, n_elts=15, entries=10_000,
        recipe="stress", seed=20150127, elt_seed=20150129, return_periods=(100.0, 250.0),
    ),
    # several layers over one YET (a portfolio's layers, Section 2.1 (iii)): the paper-1m
    # YET, a pool of 64 ELTs, 16 layers of 1..32 ELTs each (draw_layers)
    "batched-16": dict(
        n_trials=1_000_000, mean_events=1000.0, catalogue=2_000_000, n_elts=64, entries=10_000,
        recipe="plain", seed=20150127, elt_seed=20150130, layer_seed=20150131, n_layers=16,
        max_layer_elts=32, return_periods=(100.0, 250.0),
    ),
    # layer requests served against a resident YET and pool: the paper-1m YET, a pool of 200
    # ELTs, |J| ~ U{1..15}, trial prefixes log-uniform in [1e4, 1e6]
    "serving": dict(
        n_trials=1_000_000, mean_events=1000.0, catalogue=2_000_000, n_elts=200, entries=10_000,
        recipe="plain", seed=20150127, elt_seed=20150132, request_seed=20150133, max_layer_elts=15,
        min_prefix=10_000, max_prefix=1_000_000, return_periods=(100.0, 250.0),
    ),
}


def serving_requests(spec, n: int, seed: int):
    """Requests of a serving workload: per request the sorted pool ids of its layer
    (|J| ~ U{1..max_layer_elts} from the pool) and its trial prefix (log-uniform in
    [min_prefix, max_prefix]); inter-arrival gaps are drawn by the caller."""
    rng = _rng(seed, _S_LAYERS)
    out = []
    for _ in range(n):
        k = int(rng.integers(1, spec["max_layer_elts"] + 1))
        ids = np.sort(rng.choice(spec["n_elts"], size=k, replace=False)).astype(np.int32)
        lo, hi = math.log(spec["min_prefix"]), math.log(spec["max_prefix"])
        t_end = int(round(math.exp(rng.uniform(lo, hi))))
        out.append((ids, min(max(t_end, 1), spec["n_trials"])))
    return out


def workload_layers(spec, pool) -> list:
    """The layers (sorted pool-id arrays) of a batched workload."""
    return draw_layers(spec["n_layers"], pool.elt_ids, spec["max_layer_elts"], spec["layer_seed"])


def workload(name: str, n_trials: Optional[int] = None):
    """(yet, pool, spec) for a named workload; ``n_trials`` truncates the YET."""
    spec = dict(WORKLOADS[name])
    n = spec["n_trials"] if n_trials is None else int(n_trials)
    yet = make_yet(n, spec["mean_events"], spec["catalogue"], spec["seed"])
    pool = make_elt_pool(
        spec["n_elts"], spec["entries"], spec["catalogue"], spec.get("elt_seed", spec["seed"]),
        recipe=spec["recipe"],
    )
    return yet, pool, spec
