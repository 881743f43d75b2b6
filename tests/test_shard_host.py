"""The word-range split of one table (host side, no GPU): ct_shard_bounds
against its definition, and the decomposition it relies on, pinned on the
oracle: the GAC domains of a table are the union of the values each part of
its tuple list supports, its currTable the concatenation of the parts'
validity, and it fails iff every part has no valid tuple (Sec. 2: a value is
supported iff some valid tuple carries it)."""
import os
import shutil

import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import build as B
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")):
        if not os.path.exists(B.LIB):
            pytest.skip("no nvcc and no prebuilt libct.so")
    else:
        B.build()
    return C.load()


@pytest.mark.parametrize("t", [1, 127, 128, 129, 1000, 40_000, 100_001])
def test_shard_bounds_definition(lib, t):
    chunks = (t + 127) // 128
    for K in sorted({1, 2, 3, 7, chunks}):
        if K > chunks:
            continue
        st, b = C.ct_shard_bounds(t, K)
        assert st == C.CT_OK
        assert b[0] == 0 and b[-1] == t
        assert all(b[k] < b[k + 1] for k in range(K)), "every shard non-empty"
        assert all(b[k] % 128 == 0 for k in range(K)), "whole 128-tuple chunks"
        sizes = np.diff(b[:-1]) // 128 if K > 1 else np.array([])
        if len(sizes):
            assert sizes.max() - sizes.min() <= 1, "chunks spread evenly"
    assert C.ct_shard_bounds(t, chunks + 1)[0] == C.CT_ERR_ARG
    assert C.ct_shard_bounds(0, 1)[0] == C.CT_ERR_ARG


def _supported(tup, lo, masks):
    """Values carried by the valid tuples of one part (empty when none)."""
    st, out, valid = O.gac_table(tup, lo, masks) if len(tup) else (O.INFEASIBLE, None, np.zeros(0, bool))
    if st != O.OK:
        return [np.zeros_like(m) for m in masks], valid
    return out, valid


@pytest.mark.parametrize("seed", range(6))
def test_gac_is_the_union_over_tuple_ranges(seed):
    rng = G.Rng(6500 + seed)
    arity, d = 3 + seed % 3, 5 + seed
    lo, size = [0] * arity, [d] * arity
    tup = G.distinct_uniform_tuples(6500 + seed, lo, size, G.cap_distinct(size, 300 + 150 * seed))
    ret = O.retained_tuples(tup, lo, size)
    for trial in range(20):
        masks = [np.ones(d, bool) for _ in range(arity)]
        masks, _ = G.remove_random_values(rng, masks, int(rng.int(arity * (d - 1))) + 1)
        cuts = np.sort(rng.below(4, len(ret) + 1)) if trial % 2 else np.array([len(ret) // 3, 2 * len(ret) // 3])
        parts = np.split(ret, cuts)
        st, want, valid = O.gac_table(ret, lo, masks)
        union = [np.zeros(d, bool) for _ in range(arity)]
        vparts = []
        for p in parts:
            sup, v = _supported(p, lo, masks)
            union = [u | s for u, s in zip(union, sup)]
            vparts.append(v if len(v) == len(p) else np.zeros(len(p), bool))
        assert np.array_equal(np.concatenate(vparts), valid)
        if st == O.OK:
            assert all(np.array_equal(u, w) for u, w in zip(union, want))
        else:
            assert not any(u.any() for u in union)
