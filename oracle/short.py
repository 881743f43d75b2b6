"""CPU oracle of short tables (tuples with wildcards): TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the library never does.

Short tables are the extension of Compact-Table to tuples with wildcard
components that the paper cites (Sec. 1) but does not evaluate. A component
equal to STAR stands for any value of its variable: the short tuple denotes
every ground tuple obtained by replacing its wildcards with values. Written
from that definition, in float-free integer arithmetic:
  * retained: every non-wildcard component inside its initial domain (input
    order kept), like ct_oracle.retained_tuples for ground tuples;
  * valid under domains D (none empty: propagation fails before): every
    non-wildcard component in its domain;
  * GAC: value a of the k-th scope variable survives iff some valid tuple has
    component a or a wildcard at position k; the table fails when no tuple is
    valid or a domain empties;
  * currTable: bit j set iff retained tuple j is valid, packed as in ct_oracle.
"""
from __future__ import annotations

import itertools

import numpy as np

from oracle import ct_oracle as O

STAR = -2 ** 31


def retained_short(tuples, dom_lo, dom_size) -> np.ndarray:
    tuples = np.asarray(tuples, dtype=np.int64).reshape(-1, len(dom_lo))
    lo = np.asarray(dom_lo, dtype=np.int64)
    hi = lo + np.asarray(dom_size, dtype=np.int64)
    star = tuples == STAR
    keep = np.all(star | ((tuples >= lo) & (tuples < hi)), axis=1)
    return tuples[keep]


def valid_short(tup: np.ndarray, dom_lo, masks) -> np.ndarray:
    ok = np.ones(tup.shape[0], dtype=bool)
    for k, (lo, m) in enumerate(zip(dom_lo, masks)):
        col = tup[:, k]
        star = col == STAR
        idx = np.where(star, 0, col - lo)
        ok &= star | m[idx]
    return ok


def gac_table_short(tup: np.ndarray, dom_lo, masks):
    """(status, new masks, valid) of one short table under `masks`."""
    masks = [np.asarray(m, dtype=bool) for m in masks]
    valid = valid_short(tup, dom_lo, masks)
    if not valid.any():
        return O.INFEASIBLE, [np.zeros_like(m) for m in masks], valid
    vt = tup[valid]
    out = []
    for k, (lo, m) in enumerate(zip(dom_lo, masks)):
        col = vt[:, k]
        if (col == STAR).any():
            keep = m.copy()
        else:
            keep = np.zeros_like(m)
            keep[col - lo] = True
            keep &= m
        out.append(keep)
    st = O.INFEASIBLE if any(not o.any() for o in out) else O.OK
    return st, out, valid


def expand(tup: np.ndarray, dom_lo, dom_size) -> np.ndarray:
    """The ground tuples a short table stands for (wildcards over the initial
    domains), duplicates kept."""
    rows = []
    for t in tup:
        choices = [range(dom_lo[k], dom_lo[k] + dom_size[k]) if t[k] == STAR else [int(t[k])]
                   for k in range(len(t))]
        rows.extend(itertools.product(*choices))
    return np.asarray(rows, dtype=np.int64).reshape(-1, len(dom_lo))
