"""Sparse semantic representation (Sec. 3.1 "Sparse Semantic
Representation") -- TEST INFRASTRUCTURE (same rules as the rest of
``oracle``).

A Gaussian keeps the k classes of highest probability of its first observed
distribution; later observations update the k probabilities with the ids
fixed.  Written as a per-row sort of (probability, class id) pairs.

Readings where the paper is silent: equal
probabilities are ranked by the lower class id; NaN ranks below every
number; the kept probabilities are stored as observed (no renormalisation,
the renderer blends them as given).

Parity: pinned by hand-written examples (ties, NaN, k = m) and a
pure-Python selection on small random rows (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np


def topk_init(probs: np.ndarray, k: int, rows=None):
    """probs [*, m]; rows: row index per Gaussian (None: every row).  Returns
    (ids int32 [n, k], w float32 [n, k])."""
    p = np.asarray(probs, np.float32).reshape(-1, np.asarray(probs).shape[-1])
    r = np.arange(p.shape[0]) if rows is None else np.asarray(rows, np.int64)
    sel = p[r].astype(np.float64)
    key = np.where(np.isnan(sel), -np.inf, sel)
    m = p.shape[1]
    # lexsort: last key primary -> sort by (-value, id)
    order = np.lexsort((np.broadcast_to(np.arange(m), key.shape), -key), axis=1)[:, :k]
    ids = order.astype(np.int32)
    w = np.take_along_axis(p[r], order, axis=1).astype(np.float32)
    return ids, w


def topk_gather(probs: np.ndarray, ids: np.ndarray, w: np.ndarray, rows=None) -> np.ndarray:
    """w with the entries of valid ids replaced by the observed probabilities."""
    p = np.asarray(probs, np.float32).reshape(-1, np.asarray(probs).shape[-1])
    r = np.arange(ids.shape[0]) if rows is None else np.asarray(rows, np.int64)
    out = np.array(w, np.float32, copy=True)
    m = p.shape[1]
    for i in range(ids.shape[0]):
        for l in range(ids.shape[1]):
            if 0 <= ids[i, l] < m:
                out[i, l] = p[r[i], ids[i, l]]
    return out
