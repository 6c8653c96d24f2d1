"""Python binding of the ``libara`` C ABI (``include/ara.h``).

Argument marshalling only: every step of the ARA hot path runs in the CUDA
kernels of ``libara.so``.  The module-level functions mirror the C entry
points one to one (``ara_create``, ``ara_load_yet``, ``ara_load_elts``,
``ara_run_layer``, ``ara_run_layer_diag``, ``ara_run_layers``, ``ara_pml_tvar``, ``ara_sort_ylt``,
``ara_get_stats``, ``ara_last_error``, ``ara_destroy``); ``Ara`` wraps them
with error checking.  Arrays may be numpy arrays (host memory) or torch
tensors (host, pinned or CUDA): only their data pointers cross the boundary.

There is no fallback: if ``libara.so`` cannot be loaded (not built, or no
CUDA driver) every call raises.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libara.so")

ARA_OK, ARA_EINVAL, ARA_ENOMEM, ARA_ENOTLOADED, ARA_ECUDA, ARA_ETIMEOUT, ARA_EAGAIN = 0, -1, -2, -3, -4, -5, -6
ARA_PRIMARY_ONLY = 1
ARA_NEWTON_ONLY = 2
ARA_SHARED_Z = 4
ARA_AUTOTUNE = 16
ARA_MAX_LAYER_ELTS = 32
ARA_MAX_BATCH_LAYERS = 32
ARA_MAX_BATCH_ELTS = 64
ARA_SERVE_MAX_RP = 16
ARA_BATCH_AUTO, ARA_BATCH_ITEM_TILE, ARA_BATCH_ITEM_TRIAL, ARA_BATCH_ITEM_DENSE, ARA_BATCH_ITEM_INDEXED = -1, 0, 1, 2, 3
_ERR_NAMES = {
    ARA_EINVAL: "ARA_EINVAL", ARA_ENOMEM: "ARA_ENOMEM", ARA_ENOTLOADED: "ARA_ENOTLOADED",
    ARA_ECUDA: "ARA_ECUDA", ARA_ETIMEOUT: "ARA_ETIMEOUT", ARA_EAGAIN: "ARA_EAGAIN",
}

# Every function the header declares (checked by the tests against the .so).
EXPORTED = (
    "ara_create", "ara_set_stream", "ara_load_yet", "ara_load_elts", "ara_run_layer",
    "ara_run_layer_diag", "ara_pml_tvar", "ara_sort_ylt", "ara_debug_uniforms",
    "ara_debug_record_losses", "ara_get_stats", "ara_get_timing", "ara_last_error", "ara_destroy",
    "ara_pml_tvar_noalloc", "ara_run_layers", "ara_submit", "ara_serve_step", "ara_poll", "ara_load_xelts",
    "ara_run_layer_events", "ara_wait", "ara_load_yet_async", "ara_finish_yet", "ara_serve_stats",
    "ara_top_m", "ara_merge_top", "ara_set_batch_config", "ara_build_yet_index", "ara_yet_index_info",
)
ARA_NOALLOC_MAX_RP = 64


class AraError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {message}")
        self.code = code


class EltTerms(ctypes.Structure):
    _fields_ = [("retention", ctypes.c_float), ("limit", ctypes.c_float), ("share", ctypes.c_float)]


class Layer(ctypes.Structure):
    _fields_ = [
        ("n_elts", ctypes.c_int32),
        ("elt_ids", ctypes.POINTER(ctypes.c_int32)),
        ("occ_retention", ctypes.c_double),
        ("occ_limit", ctypes.c_double),
        ("agg_retention", ctypes.c_double),
        ("agg_limit", ctypes.c_double),
        ("flags", ctypes.c_uint32),
    ]


class Diag(ctypes.Structure):
    _fields_ = [("hits", ctypes.c_void_p), ("hit_hash", ctypes.c_void_p)]


class EventRows(ctypes.Structure):
    _fields_ = [
        ("capacity", ctypes.c_int64),
        ("trial", ctypes.c_void_p),
        ("event_index", ctypes.c_void_p),
        ("event_id", ctypes.c_void_p),
        ("occ_loss", ctypes.c_void_p),
        ("agg_inc", ctypes.c_void_p),
        ("max_occ", ctypes.c_void_p),
        ("n_rows", ctypes.c_int64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_events", ctypes.c_int64),
        ("n_evals", ctypes.c_int64),
        ("n_pairs_hit", ctypes.c_int64),
        ("n_nonconverged", ctypes.c_int64),
        ("n_newton", ctypes.c_int64),
        ("index_ms", ctypes.c_float),
        ("kernel_ms", ctypes.c_float),
        ("grid", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int32),
        ("filter_bits", ctypes.c_int32),
        ("batch_item", ctypes.c_int32),
        ("batch_blocks_per_sm", ctypes.c_int32),
        ("batch_tuned", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServeInfo(ctypes.Structure):
    _fields_ = [
        ("queued", ctypes.c_int64),
        ("active", ctypes.c_int64),
        ("rounds_in_flight", ctypes.c_int64),
        ("rounds_launched", ctypes.c_int64),
        ("passes_launched", ctypes.c_int64),
        ("requests_finished", ctypes.c_int64),
        ("chunk_trials", ctypes.c_int64),
        ("arena_bytes", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Timing(ctypes.Structure):
    _fields_ = [
        ("layer_calls", ctypes.c_int64),
        ("kernel_ms", ctypes.c_double),
        ("gather_ms", ctypes.c_double),
        ("losses_ms", ctypes.c_double),
        ("index_ms", ctypes.c_double),
        ("pml_calls", ctypes.c_int64),
        ("pml_ms", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``libara.so`` and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with paper_1501_06326_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    lib.ara_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t, P]
    lib.ara_set_stream.argtypes = [P, P]
    lib.ara_load_yet.argtypes = [P, i64, P, P, i32]
    lib.ara_load_yet_async.argtypes = [P, i64, P, P, i32]
    lib.ara_finish_yet.argtypes = [P]
    lib.ara_load_elts.argtypes = [P, i32, P, P, P, P, P, P, P]
    lib.ara_load_xelts.argtypes = [P, i32, P, P, P, P, P, P, P, P]
    lib.ara_run_layer.argtypes = [P, ctypes.POINTER(Layer), u64, i64, i64, P]
    lib.ara_run_layer_diag.argtypes = [P, ctypes.POINTER(Layer), u64, i64, i64, P, ctypes.POINTER(Diag)]
    lib.ara_run_layers.argtypes = [P, i32, ctypes.POINTER(Layer), u64, i64, i64, P]
    lib.ara_set_batch_config.argtypes = [P, i32, i32]
    lib.ara_build_yet_index.argtypes = [P]
    lib.ara_yet_index_info.argtypes = [P, P, P, P, P]
    lib.ara_run_layer_events.argtypes = [P, ctypes.POINTER(Layer), u64, i64, i64, P, ctypes.POINTER(EventRows)]
    lib.ara_submit.argtypes = [P, ctypes.POINTER(Layer), u64, i64, P, i32, P]
    lib.ara_serve_step.argtypes = [P, P]
    lib.ara_poll.argtypes = [P, i64, P, P]
    lib.ara_wait.argtypes = [P, i64, P, P, u64]
    lib.ara_serve_stats.argtypes = [P, ctypes.POINTER(ServeInfo)]
    lib.ara_top_m.argtypes = [P, P, i64, i64, i64, P, P]
    lib.ara_merge_top.argtypes = [P, P, i64, i64, P, i32, P, P]
    lib.ara_pml_tvar.argtypes = [P, P, i64, P, i32, P, P]
    lib.ara_sort_ylt.argtypes = [P, P, i64, P]
    lib.ara_debug_uniforms.argtypes = [P, u64, i64, P, P, P, P]
    lib.ara_debug_record_losses.argtypes = [P, i64, P, P, P, P, i32, P, P]
    lib.ara_pml_tvar_noalloc.argtypes = [P, i64, P, i32, P, P, P]
    lib.ara_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.ara_get_timing.argtypes = [P, ctypes.POINTER(Timing), ctypes.c_int]
    lib.ara_last_error.argtypes = [P]
    lib.ara_last_error.restype = ctypes.c_char_p
    lib.ara_destroy.argtypes = [P]
    lib.ara_destroy.restype = None
    for name in EXPORTED:
        if name not in ("ara_last_error", "ara_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


# ------------------------------------------------------------------ marshalling
def _ptr(a, dtype=None) -> Optional[int]:
    """Data pointer of a numpy array or torch tensor (C-contiguous, exact dtype)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if dtype is not None and a.dtype != np.dtype(dtype):
            raise TypeError(f"expected dtype {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if dtype is not None:
            import torch

            want = {np.int32: torch.int32, np.int64: torch.int64, np.float32: torch.float32,
                    np.float64: torch.float64, np.uint64: torch.uint64}[np.dtype(dtype).type]
            if a.dtype != want:
                raise TypeError(f"expected dtype {want}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _len(a) -> int:
    return int(a.shape[0])


# ------------------------------------------------------------------ C ABI mirror
def ara_create(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int = 0):
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.ara_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), ctypes.c_void_p(cuda_stream or None))
    return rc, h


def ara_set_stream(h, cuda_stream: int):
    return load_library().ara_set_stream(h, ctypes.c_void_p(cuda_stream or None))


def ara_load_yet(h, n_trials, offsets, event_ids, catalogue_size):
    return load_library().ara_load_yet(h, int(n_trials), _ptr(offsets, np.int64), _ptr(event_ids, np.int32),
                                       int(catalogue_size))


def ara_load_yet_async(h, n_trials, offsets, event_ids, catalogue_size):
    return load_library().ara_load_yet_async(h, int(n_trials), _ptr(offsets, np.int64), _ptr(event_ids, np.int32),
                                             int(catalogue_size))


def ara_finish_yet(h):
    return load_library().ara_finish_yet(h)


def ara_load_elts(h, n_elts, elt_ids, rec_offsets, event_ids, mean, sigma, exposure, terms=None):
    return load_library().ara_load_elts(
        h, int(n_elts), _ptr(elt_ids, np.int32), _ptr(rec_offsets, np.int64), _ptr(event_ids, np.int32),
        _ptr(mean, np.float32), _ptr(sigma, np.float32), _ptr(exposure, np.float32), _ptr(terms, np.float32),
    )


def ara_load_xelts(h, n_elts, elt_ids, rec_offsets, event_ids, mean, sigma_i, sigma_c, exposure, terms=None):
    return load_library().ara_load_xelts(
        h, int(n_elts), _ptr(elt_ids, np.int32), _ptr(rec_offsets, np.int64), _ptr(event_ids, np.int32),
        _ptr(mean, np.float32), _ptr(sigma_i, np.float32), _ptr(sigma_c, np.float32), _ptr(exposure, np.float32),
        _ptr(terms, np.float32),
    )


def ara_run_layer(h, layer: Layer, seed, trial_begin, trial_end, ylt_out):
    return load_library().ara_run_layer(h, ctypes.byref(layer), int(seed), int(trial_begin), int(trial_end),
                                        _ptr(ylt_out, np.float64))


def ara_run_layer_diag(h, layer: Layer, seed, trial_begin, trial_end, ylt_out, diag: Diag):
    return load_library().ara_run_layer_diag(h, ctypes.byref(layer), int(seed), int(trial_begin),
                                             int(trial_end), _ptr(ylt_out, np.float64), ctypes.byref(diag))


def ara_run_layer_events(h, layer: Layer, seed, trial_begin, trial_end, ylt_out, rows: EventRows):
    return load_library().ara_run_layer_events(h, ctypes.byref(layer), int(seed), int(trial_begin),
                                               int(trial_end), _ptr(ylt_out, np.float64), ctypes.byref(rows))


def ara_run_layers(h, n_layers, layers, seed, trial_begin, trial_end, ylt_out):
    """``layers``: a ctypes array of ``Layer``; ``ylt_out``: n_layers x (trial_end - trial_begin), layer-major."""
    return load_library().ara_run_layers(h, int(n_layers), layers, int(seed), int(trial_begin), int(trial_end),
                                         _ptr(ylt_out, np.float64))


def ara_submit(h, layer: Layer, seed, trial_end, return_periods, n_rp, ticket_out):
    return load_library().ara_submit(h, ctypes.byref(layer), int(seed), int(trial_end),
                                     _ptr(return_periods, np.float64), int(n_rp), _ptr(ticket_out, np.int64))


def ara_serve_step(h, n_done_out):
    return load_library().ara_serve_step(h, _ptr(n_done_out, np.int32))


def ara_set_batch_config(h, item, blocks_per_sm):
    return load_library().ara_set_batch_config(h, item, blocks_per_sm)


def ara_build_yet_index(h):
    return load_library().ara_build_yet_index(h)


def ara_yet_index_info(h, built, nbytes, build_ms, method):
    return load_library().ara_yet_index_info(h, built, nbytes, build_ms, method)


def ara_serve_stats(h, out):
    return load_library().ara_serve_stats(h, ctypes.byref(out))


def ara_top_m(h, ylt, n, m, trial_offset, values_out, trials_out):
    return load_library().ara_top_m(h, _ptr(ylt, np.float64), n, m, trial_offset, _ptr(values_out, np.float64),
                                    _ptr(trials_out, np.int64))


def ara_merge_top(values, trials, count, n_total, rps, n_rp, pml_out, tvar_out):
    return load_library().ara_merge_top(_ptr(values, np.float64), _ptr(trials, np.int64), count, n_total,
                                        _ptr(rps, np.float64), n_rp, _ptr(pml_out, np.float64),
                                        _ptr(tvar_out, np.float64))


def merge_top(values, trials, n_total: int, return_periods):
    """PML and TVaR of a trial-sharded YLT from the ranks' ara_top_m lists
    (concatenated host arrays): ara_merge_top, which needs no GPU."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    t = np.ascontiguousarray(trials, dtype=np.int64)
    rps = np.ascontiguousarray(return_periods, dtype=np.float64)
    pml, tvar = np.zeros(rps.shape[0]), np.zeros(rps.shape[0])
    rc = ara_merge_top(v, t, v.shape[0], int(n_total), rps, rps.shape[0], pml, tvar)
    if rc != ARA_OK:
        raise AraError(rc, "ara_merge_top: bad arguments or fewer than m finite values")
    return pml, tvar


def ara_poll(h, ticket, pml_out, tvar_out):
    return load_library().ara_poll(h, int(ticket), _ptr(pml_out, np.float64), _ptr(tvar_out, np.float64))


def ara_wait(h, ticket, pml_out, tvar_out, timeout_ns=0):
    return load_library().ara_wait(h, int(ticket), _ptr(pml_out, np.float64), _ptr(tvar_out, np.float64),
                                   int(timeout_ns))


def ara_pml_tvar(h, ylt, n, return_periods, n_rp, pml_out, tvar_out):
    return load_library().ara_pml_tvar(h, _ptr(ylt, np.float64), int(n), _ptr(return_periods, np.float64),
                                       int(n_rp), _ptr(pml_out, np.float64), _ptr(tvar_out, np.float64))


def ara_sort_ylt(h, ylt, n, order_out):
    return load_library().ara_sort_ylt(h, _ptr(ylt, np.float64), int(n), _ptr(order_out, np.int64))


def ara_debug_uniforms(h, seed, n, trials, ks, elts, out):
    return load_library().ara_debug_uniforms(h, int(seed), int(n), _ptr(trials, np.int64), _ptr(ks, np.int32),
                                             _ptr(elts, np.int32), _ptr(out, np.float32))


def ara_debug_record_losses(h, n, mean, sigma, exposure, z, newton_only, out, iters_out=None):
    return load_library().ara_debug_record_losses(h, int(n), _ptr(mean, np.float32), _ptr(sigma, np.float32),
                                                  _ptr(exposure, np.float32), _ptr(z, np.float32),
                                                  int(newton_only), _ptr(out, np.float32),
                                                  _ptr(iters_out, np.int32))


def ara_pml_tvar_noalloc(ylt, n, return_periods, n_rp, pml_out, tvar_out, cuda_stream: int = 0):
    """PML / TVaR without device allocation (no context; ylt must be device memory)."""
    return load_library().ara_pml_tvar_noalloc(_ptr(ylt, np.float64), int(n), _ptr(return_periods, np.float64),
                                               int(n_rp), _ptr(pml_out, np.float64), _ptr(tvar_out, np.float64),
                                               ctypes.c_void_p(cuda_stream or None))


def ara_get_stats(h, out: Stats):
    return load_library().ara_get_stats(h, ctypes.byref(out))


def ara_get_timing(h, out: Timing, reset: int):
    return load_library().ara_get_timing(h, ctypes.byref(out), int(reset))


def ara_last_error(h) -> str:
    msg = load_library().ara_last_error(h)
    return msg.decode() if msg else ""


def ara_destroy(h) -> None:
    load_library().ara_destroy(h)


# ------------------------------------------------------------------ wrapper
class Ara:
    """One engine context on one CUDA device (see ``include/ara.h``)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int = 0):
        rc, h = ara_create(device, hbm_budget_bytes, cuda_stream)
        if rc != ARA_OK:
            raise AraError(rc, f"ara_create(device={device}) failed")
        self._h = h
        self._yet_refs = None  # the arrays of an upload in flight (load_yet_async)

    # -- lifecycle
    def close(self) -> None:
        if getattr(self, "_h", None):
            ara_destroy(self._h)
            self._h = None
        self._yet_refs = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int) -> None:
        if rc != ARA_OK:
            raise AraError(rc, ara_last_error(self._h))

    # -- calls
    def set_stream(self, cuda_stream: int) -> None:
        self._check(ara_set_stream(self._h, cuda_stream))

    def load_yet(self, offsets, event_ids, catalogue_size: int) -> None:
        # the call waits for an upload in flight before its arrays are let go
        rc = ara_load_yet(self._h, _len(offsets) - 1, offsets, event_ids, catalogue_size)
        self._yet_refs = None
        self._check(rc)

    def load_yet_async(self, offsets, event_ids, catalogue_size: int) -> None:
        """``ara_load_yet_async``: returns while the ids are copied; the arrays
        are kept referenced until the next YET load or ``close``."""
        rc = ara_load_yet_async(self._h, _len(offsets) - 1, offsets, event_ids, catalogue_size)
        self._yet_refs = (offsets, event_ids)
        self._check(rc)

    def finish_yet(self) -> None:
        self._check(ara_finish_yet(self._h))

    def load_elts(self, elt_ids, rec_offsets, event_ids, mean, sigma, exposure, terms=None) -> None:
        if terms is not None and isinstance(terms, np.ndarray):
            terms = np.ascontiguousarray(terms, dtype=np.float32)
        self._check(ara_load_elts(self._h, _len(elt_ids), elt_ids, rec_offsets, event_ids, mean, sigma, exposure,
                                  terms))

    def load_xelts(self, elt_ids, rec_offsets, event_ids, mean, sigma_i, sigma_c, exposure, terms=None) -> None:
        if terms is not None and isinstance(terms, np.ndarray):
            terms = np.ascontiguousarray(terms, dtype=np.float32)
        self._check(ara_load_xelts(self._h, _len(elt_ids), elt_ids, rec_offsets, event_ids, mean, sigma_i, sigma_c,
                                   exposure, terms))

    def load_pool(self, pool) -> None:
        """Load an ``ELTPool`` (see ``synth``); a pool with a correlated part
        ``sigma_c`` goes through ``ara_load_xelts``."""
        if getattr(pool, "sigma_c", None) is not None:
            self.load_xelts(pool.elt_ids, pool.rec_offsets, pool.event_ids, pool.mean, pool.sigma, pool.sigma_c,
                            pool.exposure, pool.terms)
        else:
            self.load_elts(pool.elt_ids, pool.rec_offsets, pool.event_ids, pool.mean, pool.sigma, pool.exposure,
                           pool.terms)

    @staticmethod
    def make_layer(elt_ids: Sequence[int], layer_terms, primary_only: bool = False, newton_only: bool = False,
                   shared_z: bool = False, autotune: bool = False):
        ids = (ctypes.c_int32 * len(elt_ids))(*[int(i) for i in elt_ids])
        occ_r, occ_l, agg_r, agg_l = (float(v) for v in layer_terms)
        flags = ((ARA_PRIMARY_ONLY if primary_only else 0) | (ARA_NEWTON_ONLY if newton_only else 0)
                 | (ARA_SHARED_Z if shared_z else 0) | (ARA_AUTOTUNE if autotune else 0))
        lay = Layer(len(elt_ids), ids, occ_r, occ_l, agg_r, agg_l, flags)
        lay._ids = ids  # keep the id array alive with the struct
        return lay

    def run_layer(self, elt_ids, layer_terms, seed: int, trial_begin: int, trial_end: int, ylt_out,
                  primary_only: bool = False, hits_out=None, hash_out=None, newton_only: bool = False,
                  shared_z: bool = False) -> None:
        lay = self.make_layer(elt_ids, layer_terms, primary_only, newton_only, shared_z)
        if hits_out is None and hash_out is None:
            self._check(ara_run_layer(self._h, lay, seed, trial_begin, trial_end, ylt_out))
        else:
            d = Diag(_ptr(hits_out, np.int64), _ptr(hash_out, np.uint64))
            self._check(ara_run_layer_diag(self._h, lay, seed, trial_begin, trial_end, ylt_out, d))

    def run_layer_events(self, elt_ids, layer_terms, seed: int, trial_begin: int, trial_end: int, ylt_out,
                         trial=None, event_index=None, event_id=None, occ_loss=None, agg_inc=None, max_occ=None,
                         capacity: Optional[int] = None, primary_only: bool = False,
                         newton_only: bool = False, shared_z: bool = False) -> int:
        """ara_run_layer plus the per-event rows (any array may be None); returns
        the number of rows of the trial range (rows beyond ``capacity`` -- by
        default the length of the given row arrays -- are not written)."""
        lay = self.make_layer(elt_ids, layer_terms, primary_only, newton_only, shared_z)
        arrs = [(trial, np.int64), (event_index, np.int32), (event_id, np.int32), (occ_loss, np.float64),
                (agg_inc, np.float64)]
        if capacity is None:
            lens = [len(a) for a, _ in arrs if a is not None]
            capacity = min(lens) if lens else 0
        rows = EventRows(int(capacity), *[_ptr(a, dt) for a, dt in arrs], _ptr(max_occ, np.float64), 0)
        self._check(ara_run_layer_events(self._h, lay, seed, trial_begin, trial_end, ylt_out, rows))
        return int(rows.n_rows)

    def run_layers(self, layers, seed: int, trial_begin: int, trial_end: int, ylt_out,
                   primary_only: bool = False, newton_only: bool = False, shared_z: bool = False,
                   autotune: bool = False) -> None:
        """Several layers in one pass.  ``layers``: a sequence of (elt_ids, layer_terms);
        ``ylt_out``: (n_layers, trial_end - trial_begin) float64, C order.  ``autotune``:
        ARA_AUTOTUNE (measure the losses kernel's configurations on a new shape)."""
        made = [self.make_layer(ids, terms, primary_only, newton_only, shared_z, autotune) for ids, terms in layers]
        arr = (Layer * len(made))(*made)
        self._check(ara_run_layers(self._h, len(made), arr, seed, trial_begin, trial_end, ylt_out))

    def set_batch_config(self, item: int = ARA_BATCH_AUTO, blocks_per_sm: int = 0) -> None:
        """Pin the batched losses kernel's work item (ARA_BATCH_ITEM_*) and CTAs per
        SM (0: as many as an SM holds); ARA_BATCH_AUTO returns to the autotuner's
        cached choice or the default rule."""
        self._check(ara_set_batch_config(self._h, int(item), int(blocks_per_sm)))

    def build_yet_index(self) -> None:
        """Build the loaded YET's event-major index (ara_build_yet_index)."""
        self._check(ara_build_yet_index(self._h))

    def yet_index_info(self) -> dict:
        """Whether the YET's index is built, its bytes, its build's device time and
        how it was built ("buckets", "radix sort", or None when not built)."""
        built = np.zeros(1, np.int32)
        nbytes = np.zeros(1, np.int64)
        ms = np.zeros(1, np.float32)
        method = np.zeros(1, np.int32)
        self._check(ara_yet_index_info(self._h, built.ctypes.data, nbytes.ctypes.data, ms.ctypes.data,
                                       method.ctypes.data))
        return {"built": bool(built[0]), "bytes": int(nbytes[0]), "build_ms": float(ms[0]),
                "method": {0: "buckets", 1: "radix sort"}.get(int(method[0]))}

    def submit(self, elt_ids, layer_terms, seed: int, trial_end: int, return_periods,
               primary_only: bool = False, shared_z: bool = False) -> int:
        """Queue a serving request; returns its ticket."""
        lay = self.make_layer(elt_ids, layer_terms, primary_only, shared_z=shared_z)
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        tk = np.zeros(1, np.int64)
        self._check(ara_submit(self._h, lay, seed, trial_end, rps, rps.shape[0], tk))
        return int(tk[0])

    def serve_step(self) -> int:
        """Finish what the device has completed, admit queued requests and launch
        the next round without waiting for it; returns how many requests
        finished in this call."""
        n = np.zeros(1, np.int32)
        self._check(ara_serve_step(self._h, n))
        return int(n[0])

    def top_m(self, ylt, m: int, trial_offset: int = 0, values_out=None, trials_out=None):
        """The m largest year losses (descending, ties by trial) and their global
        trial indices (ara_top_m); host arrays unless outputs are given."""
        vals = np.zeros(m) if values_out is None else values_out
        trials = np.zeros(m, np.int64) if trials_out is None else trials_out
        self._check(ara_top_m(self._h, ylt, _len(ylt), int(m), int(trial_offset), vals, trials))
        return vals, trials

    def serve_stats(self) -> dict:
        """Queue state and totals of the serving loop (ara_serve_stats)."""
        info = ServeInfo()
        self._check(ara_serve_stats(self._h, info))
        return info.as_dict()

    def poll(self, ticket: int, n_rp: int):
        """(pml, tvar) of a finished request, or None while it is queued."""
        pml, tvar = np.zeros(n_rp), np.zeros(n_rp)
        rc = ara_poll(self._h, ticket, pml, tvar)
        if rc == ARA_EAGAIN:
            return None
        self._check(rc)
        return pml, tvar

    def wait(self, ticket: int, n_rp: int, timeout_ns: int = 0):
        """Serve until the request is finished; its (pml, tvar).  Raises AraError
        (code ARA_ETIMEOUT) when timeout_ns passes first."""
        pml, tvar = np.zeros(n_rp), np.zeros(n_rp)
        self._check(ara_wait(self._h, ticket, pml, tvar, timeout_ns))
        return pml, tvar

    def pml_tvar(self, ylt, return_periods, pml_out=None, tvar_out=None):
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        pml = np.zeros(rps.shape[0]) if pml_out is None else pml_out
        tvar = np.zeros(rps.shape[0]) if tvar_out is None else tvar_out
        self._check(ara_pml_tvar(self._h, ylt, _len(ylt), rps, rps.shape[0], pml, tvar))
        return pml, tvar

    def sort_ylt(self, ylt, order_out=None):
        order = np.zeros(_len(ylt), np.int64) if order_out is None else order_out
        self._check(ara_sort_ylt(self._h, ylt, _len(ylt), order))
        return order

    def debug_uniforms(self, seed, trials, ks, elts) -> np.ndarray:
        t = np.ascontiguousarray(trials, np.int64)
        k = np.ascontiguousarray(ks, np.int32)
        e = np.ascontiguousarray(elts, np.int32)
        out = np.zeros(t.shape[0], np.float32)
        self._check(ara_debug_uniforms(self._h, seed, t.shape[0], t, k, e, out))
        return out

    def debug_record_losses(self, mean, sigma, exposure, z, newton_only: bool = False):
        mu = np.ascontiguousarray(mean, np.float32)
        sg = np.ascontiguousarray(sigma, np.float32)
        ex = np.ascontiguousarray(exposure, np.float32)
        zz = np.ascontiguousarray(z, np.float32)
        out = np.zeros(mu.shape[0], np.float32)
        iters = np.zeros(mu.shape[0], np.int32)
        self._check(ara_debug_record_losses(self._h, mu.shape[0], mu, sg, ex, zz, int(newton_only), out, iters))
        return out, iters

    def stats(self) -> dict:
        s = Stats()
        self._check(ara_get_stats(self._h, s))
        return s.as_dict()

    def timing(self, reset: bool = False) -> dict:
        t = Timing()
        self._check(ara_get_timing(self._h, t, 1 if reset else 0))
        return t.as_dict()
