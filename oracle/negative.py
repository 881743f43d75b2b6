"""CPU oracle of negative tables (forbidden tuples): TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the library never does.

A negative table lists the forbidden tuples (the extension of Compact-Table the
paper cites, Sec. 1, but does not evaluate). Written from the definition, in
integer arithmetic:
  * retained: the tuples whose components are all in the initial domains,
    each distinct tuple once (first occurrence, input order kept);
  * valid under domains D: every component in its domain;
  * one filtering pass: value a of the k-th scope variable survives iff some
    assignment of the other scope variables within their (input) domains,
    together with a, is not forbidden, i.e. iff the valid forbidden tuples with
    component a at k are fewer than the product of the other domain sizes;
    the table fails when a domain empties. Unlike a positive table's, one pass
    is not a fixpoint (a removal shrinks the other variables' products); a
    network repeats it until nothing changes;
  * currTable: bit j set iff retained tuple j is valid (ct_oracle packing).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import ct_oracle as O


def retained_negative(tuples, dom_lo, dom_size) -> np.ndarray:
    tup = O.retained_tuples(tuples, dom_lo, dom_size)
    seen, keep = set(), []
    for j, row in enumerate(tup):
        key = tuple(int(v) for v in row)
        if key not in seen:
            seen.add(key)
            keep.append(j)
    return tup[keep]


def gac_table_negative(tup: np.ndarray, dom_lo, masks):
    """(status, new masks, valid) of one negative table under `masks`."""
    masks = [np.asarray(m, dtype=bool) for m in masks]
    if any(not m.any() for m in masks):
        return O.INFEASIBLE, [np.zeros_like(m) for m in masks], np.zeros(len(tup), dtype=bool)
    valid = O.valid_mask(tup, dom_lo, masks)
    vt = tup[valid]
    sizes = [int(m.sum()) for m in masks]
    out = []
    for k, (lo, m) in enumerate(zip(dom_lo, masks)):
        other = math.prod(sizes[:k] + sizes[k + 1:])
        cnt = np.bincount(vt[:, k] - lo, minlength=len(m)) if len(vt) else np.zeros(len(m), dtype=np.int64)
        out.append(m & (cnt < other))
    st = O.INFEASIBLE if any(not o.any() for o in out) else O.OK
    return st, out, valid


def complement(tup: np.ndarray, dom_lo, dom_size) -> np.ndarray:
    """The allowed tuples of a negative table (every combination of the initial
    domains that is not forbidden)."""
    import itertools
    forb = {tuple(int(v) for v in row) for row in tup}
    rows = [c for c in itertools.product(*[range(l, l + s) for l, s in zip(dom_lo, dom_size)]) if c not in forb]
    return np.asarray(rows, dtype=np.int64).reshape(-1, len(dom_lo))
