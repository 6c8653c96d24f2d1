"""Trial-sharded ARA across ranks: the host-side merge of PML / TVaR.

Trials are independent (Algorithm 1 loops over them with no exchange), so
each rank runs the layer on its own contiguous trial range and keeps its YLT
slice.  PML(RP) and TVaR(RP) of the whole YLT need only the m = ceil(N / RP)
largest year losses overall, and these are contained in the union of every
rank's own m largest.  So one all-gather of each rank's top m values
(descending) is the only exchange, and the merge below is exact.
"""

from __future__ import annotations

import math
from typing import Iterable, Sequence

import numpy as np


def local_top(ylt: np.ndarray, m: int) -> np.ndarray:
    """The m largest values of one rank's YLT slice, descending, padded with -inf."""
    y = np.asarray(ylt, dtype=np.float64)
    k = min(m, y.size)
    out = np.full(m, -np.inf)
    if k:
        part = np.partition(y, y.size - k)[y.size - k:]
        out[:k] = np.sort(part)[::-1]
    return out


def global_pml_tvar(tops: Iterable[np.ndarray], n_total: int, return_periods: Sequence[float]):
    """Exact PML / TVaR of the concatenated YLT from every rank's ``local_top``."""
    allv = np.sort(np.concatenate([np.asarray(t, np.float64) for t in tops]))[::-1]
    pml, tvar = [], []
    for rp in return_periods:
        m = min(max(int(math.ceil(n_total / rp)), 1), n_total)
        if m > allv.size or not np.isfinite(allv[m - 1]):
            raise ValueError("each rank must contribute at least m values")
        pml.append(float(allv[m - 1]))
        tvar.append(float(math.fsum(allv[:m]) / m))
    return np.array(pml), np.array(tvar)
