"""FP64 CPU oracle for ARA with secondary uncertainty -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  It wraps the plain C
implementation in ``ara_oracle.c`` (built with gcc into ``libara_oracle.so``)
and shares no code with the CUDA path.

Functions cite the paper's sections; every function here is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` against closed forms,
SciPy, cuRAND's Philox generator (run as a library), hand-summed tiny cases
and invariants.  The full-size workloads have no printed values in the paper
(parity of full configurations against the paper itself is unpinned); the
oracle is pinned function by function instead.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ara_oracle.c")
_LIB = os.path.join(_HERE, "libara_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``ara_oracle.c`` with gcc (OpenMP over trials)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            lib.or_philox4x32_10.argtypes = [P, P, P]
            lib.or_philox4x32_10.restype = None
            lib.or_uniform.argtypes = [u64, i64, i32, i32]
            lib.or_uniform.restype = dbl
            lib.or_betainc.argtypes = [dbl, dbl, dbl]
            lib.or_betainc.restype = dbl
            lib.or_betaincinv.argtypes = [dbl, dbl, dbl]
            lib.or_betaincinv.restype = dbl
            lib.or_beta_params.argtypes = [dbl, dbl, dbl, P, P]
            lib.or_beta_params.restype = ctypes.c_int
            lib.or_run_layer.argtypes = [
                i64, P, P, i32,  # yet
                i32, P, P, P, P, P, P, P, P,  # elts (ids, offsets, events, mean, sigma, sigma_c, exposure, terms)
                dbl, dbl, dbl, dbl,  # layer terms
                u64, ctypes.c_int,  # seed, primary_only
                i64, P,  # trial list
                P, P, P, P, ctypes.c_int,  # outputs, threads
            ]
            lib.or_run_layer.restype = ctypes.c_int
            lib.or_event_losses.argtypes = [
                P, P, i32, i32, P, P, P, P, P, P, P, P, u64, ctypes.c_int, i64, i64, P, i64
            ]
            lib.or_event_losses.restype = i64
            lib.or_run_layer_events.argtypes = [
                P, P, i32, i32, P, P, P, P, P, P, P, P, dbl, dbl, dbl, dbl, u64, ctypes.c_int, i64, i64,
                P, P, P, P, P, i64, P,
            ]
            lib.or_run_layer_events.restype = i64
            lib.or_uniform_batch.argtypes = [u64, i64, P, P, P, P]
            lib.or_uniform_batch.restype = None
            lib.or_combined_normal_batch.argtypes = [u64, i64, P, P, P, dbl, dbl, P, P]
            lib.or_combined_normal_batch.restype = None
            lib.or_normcdfinv_batch.argtypes = [i64, P, P]
            lib.or_normcdfinv_batch.restype = None
            lib.or_normcdf.argtypes = [dbl]
            lib.or_normcdf.restype = dbl
            lib.or_uniform_event.argtypes = [u64, i64, i32]
            lib.or_uniform_event.restype = dbl
            lib.or_betaincinv_batch.argtypes = [i64, P, P, P, P]
            lib.or_betaincinv_batch.restype = None
            lib.or_betainc_batch.argtypes = [i64, P, P, P, P]
            lib.or_betainc_batch.restype = None
            lib.or_betaincinv_complement.argtypes = [dbl, dbl, dbl]
            lib.or_betaincinv_complement.restype = dbl
            lib.or_betaincinv_upper.argtypes = [dbl, dbl, dbl]
            lib.or_betaincinv_upper.restype = dbl
            lib.or_sort_desc.argtypes = [P, i64, P]
            lib.or_sort_desc.restype = ctypes.c_int
            lib.or_pml_tvar.argtypes = [P, i64, P, i32, P, P]
            lib.or_pml_tvar.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------- Philox
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform(seed: int, trial: int, k: int, elt_id: int) -> float:
    """The uniform z of one (trial, event index, ELT) triple (Section 3.1 (i))."""
    return _load().or_uniform(int(seed), int(trial), int(k), int(elt_id))


# ---------------------------------------------------------------- Beta
def betainc(x: float, a: float, b: float) -> float:
    """Regularised incomplete Beta I_x(a, b) = B(x; a, b) / B(a, b) (Section 3.3)."""
    return _load().or_betainc(float(x), float(a), float(b))


def betaincinv(p: float, a: float, b: float) -> float:
    """InvCDF_beta(p; a, b) (Section 3.3): the x with I_x(a, b) = p."""
    return _load().or_betaincinv(float(p), float(a), float(b))


def betaincinv_complement(p: float, a: float, b: float) -> float:
    """1 - InvCDF_beta(p; a, b), accurate when the root is close to 1."""
    return _load().or_betaincinv_complement(float(p), float(a), float(b))


def betaincinv_upper(q: float, a: float, b: float) -> float:
    """InvCDF_beta(1 - q; a, b) from the upper-tail probability q."""
    return _load().or_betaincinv_upper(float(q), float(a), float(b))


def uniform_batch(seed: int, trials, ks, elts) -> np.ndarray:
    """Vectorised ``uniform`` over arrays of (trial, k, elt_id)."""
    t = _c(trials, np.int64)
    k = _c(ks, np.int32)
    e = _c(elts, np.int32)
    out = np.zeros(t.shape[0])
    _load().or_uniform_batch(int(seed), t.shape[0], _p(t), _p(k), _p(e), _p(out))
    return out


def betaincinv_batch(p, a, b) -> np.ndarray:
    """Vectorised ``betaincinv`` (OpenMP over elements)."""
    p, a, b = np.broadcast_arrays(np.asarray(p, np.float64), np.asarray(a, np.float64), np.asarray(b, np.float64))
    p, a, b = _c(p, np.float64), _c(a, np.float64), _c(b, np.float64)
    out = np.zeros(p.shape, np.float64)
    _load().or_betaincinv_batch(p.size, _p(p), _p(a), _p(b), _p(out))
    return out


def betainc_batch(x, a, b) -> np.ndarray:
    """Vectorised ``betainc``."""
    x, a, b = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(a, np.float64), np.asarray(b, np.float64))
    x, a, b = _c(x, np.float64), _c(a, np.float64), _c(b, np.float64)
    out = np.zeros(x.shape, np.float64)
    _load().or_betainc_batch(x.size, _p(x), _p(a), _p(b), _p(out))
    return out


def beta_params(mu: float, sigma: float, max_l: float):
    """(kind, alpha, beta) of one XELT record (Section 3.3).

    kind 0: secondary uncertainty with Beta(alpha, beta); 1: deterministic
    (mu == 0 or sigma == 0); -1: invalid record.
    """
    a = np.zeros(1)
    b = np.zeros(1)
    kind = _load().or_beta_params(float(mu), float(sigma), float(max_l), _p(a), _p(b))
    return kind, float(a[0]), float(b[0])


# ---------------------------------------------------------------- ARA
# The ELT word of the Philox counter that every ELT of an occurrence shares
# when z_(Prog,E) is one draw per YET entry (Section 3.1): 0xFFFFFFFE.
SHARED_Z_WORD = -2


def _elt_arrays(pool, shared_z: bool = False):
    """The pool's arrays in the oracle's argument order (sigma_c: None when the
    records carry no correlated standard deviation).  ``shared_z``: every ELT
    keys its uniforms (and the hit hash) by SHARED_Z_WORD instead of its pool id."""
    sc = getattr(pool, "sigma_c", None)
    ids = np.full(pool.n_elts, SHARED_Z_WORD, np.int32) if shared_z else _c(pool.elt_ids, np.int32)
    return [
        ids, _c(pool.rec_offsets, np.int64), _c(pool.event_ids, np.int32),
        _c(pool.mean, np.float32), _c(pool.sigma, np.float32), None if sc is None else _c(sc, np.float32),
        _c(pool.exposure, np.float32), _c(pool.terms, np.float32),
    ]


def uniform_event(seed: int, trial: int, k: int) -> float:
    """The event-occurrence uniform z_(E) (Section 3.1 (ii)): shared by all ELTs."""
    return _load().or_uniform_event(int(seed), int(trial), int(k))


def normcdf(v: float) -> float:
    """Standard normal CDF (Section 3.2 step v)."""
    return _load().or_normcdf(float(v))


def normcdfinv_batch(p) -> np.ndarray:
    """Standard normal quantile (Section 3.2 step ii)."""
    p = _c(p, np.float64)
    out = np.zeros(p.shape[0], np.float64)
    _load().or_normcdfinv_batch(p.shape[0], _p(p), _p(out))
    return out


def combined_normal_batch(seed: int, trials, ks, elts, sigma_i: float, sigma_c: float):
    """(v, z) of the five steps of Section 3.2 for each (trial, k, ELT pool id)."""
    t = _c(trials, np.int64)
    k = _c(ks, np.int32)
    e = _c(elts, np.int32)
    v = np.zeros(t.shape[0], np.float64)
    z = np.zeros(t.shape[0], np.float64)
    _load().or_combined_normal_batch(int(seed), t.shape[0], _p(t), _p(k), _p(e), float(sigma_i), float(sigma_c),
                                     _p(v), _p(z))
    return v, z


def run_layer(yet, pool, layer_terms, seed: int = 0, primary_only: bool = False,
              trials=None, threads: int = 0, shared_z: bool = False):
    """Algorithm 1 with secondary uncertainty over one layer (Sections 2.2, 3.3).

    ``pool`` holds exactly the layer's ELTs (an ``ELTPool``); ``layer_terms``
    is (OccR, OccL, AggR, AggL).  Returns a dict with ``ylt`` (year loss per
    evaluated trial), ``gross`` (sum of the trial's event losses before any
    terms), ``hits`` (number of (event, ELT) lookups that found a record)
    and ``hit_hash`` (order-free hash of the (k, elt_id) hit list).
    """
    lib = _load()
    offs = _c(yet.offsets, np.int64)
    ids = _c(yet.event_ids, np.int32)
    tl = None if trials is None else _c(trials, np.int64)
    n = yet.n_trials if tl is None else int(tl.shape[0])
    ylt = np.zeros(n, np.float64)
    gross = np.zeros(n, np.float64)
    hits = np.zeros(n, np.int64)
    hh = np.zeros(n, np.uint64)
    arrs = _elt_arrays(pool, shared_z)
    occ_r, occ_l, agg_r, agg_l = (float(v) for v in layer_terms)
    rc = lib.or_run_layer(
        yet.n_trials, _p(offs), _p(ids), int(yet.catalogue_size),
        pool.n_elts, *[_p(a) if a is not None else None for a in arrs],
        occ_r, occ_l, agg_r, agg_l, int(seed), int(bool(primary_only)),
        0 if tl is None else n, _p(tl) if tl is not None else None,
        _p(ylt), _p(gross), _p(hits), _p(hh), int(threads),
    )
    if rc != 0:
        raise ValueError(f"oracle run_layer failed with code {rc}")
    return {"ylt": ylt, "gross": gross, "hits": hits, "hit_hash": hh}


def event_losses(yet, pool, seed=0, primary_only=True, t_begin=0, t_end=None):
    """Nonzero combined event losses (after ELT terms, before occurrence terms)."""
    lib = _load()
    t_end = yet.n_trials if t_end is None else int(t_end)
    offs = _c(yet.offsets, np.int64)
    ids = _c(yet.event_ids, np.int32)
    cap = int(offs[t_end] - offs[t_begin]) + 1
    out = np.zeros(cap, np.float64)
    arrs = _elt_arrays(pool)
    n = lib.or_event_losses(
        _p(offs), _p(ids), int(yet.catalogue_size), pool.n_elts, *[_p(a) if a is not None else None for a in arrs],
        int(seed), int(bool(primary_only)), int(t_begin), int(t_end), _p(out), cap,
    )
    if n < 0:
        raise ValueError(f"oracle event_losses failed with code {n}")
    return out[:n]


def run_layer_events(yet, pool, layer_terms, seed=0, primary_only=False, t_begin=0, t_end=None, shared_z=False):
    """Per-event output of a layer over trials [t_begin, t_end): one row per event
    occurrence held by at least one of the layer's ELTs, in (trial, k) order, as a
    dict of arrays ``trial, k, event, occ`` (O_k after occurrence terms) and ``inc``
    (A_k - A_{k-1}), plus ``max_occ`` per trial."""
    lib = _load()
    t_end = yet.n_trials if t_end is None else int(t_end)
    offs = _c(yet.offsets, np.int64)
    ids = _c(yet.event_ids, np.int32)
    cap = int(offs[t_end] - offs[t_begin]) + 1
    rows = {"trial": np.zeros(cap, np.int64), "k": np.zeros(cap, np.int32), "event": np.zeros(cap, np.int32),
            "occ": np.zeros(cap, np.float64), "inc": np.zeros(cap, np.float64)}
    max_occ = np.zeros(max(t_end - t_begin, 1), np.float64)
    occ_r, occ_l, agg_r, agg_l = (float(v) for v in layer_terms)
    arrs = _elt_arrays(pool, shared_z)
    n = lib.or_run_layer_events(
        _p(offs), _p(ids), int(yet.catalogue_size), pool.n_elts, *[_p(a) if a is not None else None for a in arrs],
        occ_r, occ_l, agg_r, agg_l, int(seed), int(bool(primary_only)), int(t_begin), int(t_end),
        _p(rows["trial"]), _p(rows["k"]), _p(rows["event"]), _p(rows["occ"]), _p(rows["inc"]), cap, _p(max_occ),
    )
    if n < 0:
        raise ValueError(f"oracle run_layer_events failed with code {n}")
    out = {k: v[:n] for k, v in rows.items()}
    out["max_occ"] = max_occ[: t_end - t_begin]
    return out


# ---------------------------------------------------------------- PML / TVaR
def sort_desc(ylt) -> np.ndarray:
    """Trial indices ordered by year loss, largest first, ties by index."""
    y = _c(ylt, np.float64)
    order = np.zeros(y.shape[0], np.int64)
    _load().or_sort_desc(_p(y), y.shape[0], _p(order))
    return order


def pml_tvar(ylt, return_periods):
    """PML and TVaR at the given return periods (Section 2.3)."""
    y = _c(ylt, np.float64)
    rps = _c(return_periods, np.float64)
    pml = np.zeros(rps.shape[0])
    tvar = np.zeros(rps.shape[0])
    rc = _load().or_pml_tvar(_p(y), y.shape[0], _p(rps), rps.shape[0], _p(pml), _p(tvar))
    if rc != 0:
        raise ValueError(f"oracle pml_tvar failed with code {rc}")
    return pml, tvar


# ---------------------------------------------------------------- term calibration
def nearest_rank(values, pct: float) -> float:
    """Nearest-rank percentile: the ceil(pct/100 * n)-th smallest value."""
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return 0.0
    r = int(np.ceil(pct / 100.0 * v.size))
    return float(v[min(max(r, 1), v.size) - 1])


def calibrate_layer_terms(yet, pool, t_begin=0, t_end=None, occ_pct=(50.0, 99.0), agg_pct=(10.0, 99.0)):
    """Percentile-set layer terms, computed with primary uncertainty only.

    OccR / OccL are the 50th / 99th nearest-rank percentiles of the nonzero
    combined per-event layer losses over the trials; AggR / AggL are the
    10th / 99th percentiles of the trials' sums of occurrence losses (after
    the occurrence terms, zeros included).  OccL and AggL are used as the
    limits of the occurrence and aggregate terms (Section 2.2).
    """
    t_end = yet.n_trials if t_end is None else int(t_end)
    g = event_losses(yet, pool, primary_only=True, t_begin=t_begin, t_end=t_end)
    occ_r = nearest_rank(g, occ_pct[0])
    occ_l = nearest_rank(g, occ_pct[1])
    trials = np.arange(t_begin, t_end, dtype=np.int64)
    # trial sums of occurrence losses: the aggregate terms set to the identity
    r = run_layer(yet, pool, (occ_r, occ_l, 0.0, np.inf), primary_only=True, trials=trials)
    agg_r = nearest_rank(r["ylt"], agg_pct[0])
    agg_l = nearest_rank(r["ylt"], agg_pct[1])
    return (occ_r, occ_l, agg_r, agg_l)
