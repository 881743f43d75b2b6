"""The serial CPU bitset CT baseline (Algorithms 1-3) agrees with the oracle.

Third opinion beside the oracle and the GPU library: same domains, status and
currTable words on delta/reset streams with save/restore."""
import numpy as np
import pytest

from oracle import ct_oracle as O
from oracle.serial_ct import SerialCT
from paper_2507_18413_gb300 import inputs as G


def _pack(masks):
    out = []
    for m in masks:
        nw = (len(m) + 31) // 32
        w = np.zeros(nw, dtype=np.uint64)
        for a in np.flatnonzero(m):
            w[a // 32] |= np.uint64(1) << np.uint64(a % 32)
        out.append(w.astype(np.uint32))
    return np.concatenate(out)


def _unpack(words, sizes):
    masks, off = [], 0
    for d in sizes:
        nw = (d + 31) // 32
        m = np.zeros(d, dtype=bool)
        for a in range(d):
            m[a] = (int(words[off + a // 32]) >> (a % 32)) & 1
        masks.append(m)
        off += nw
    return masks


def _stream(dom_lo, dom_size, tup, calls, seed, edit, depth=8):
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    ct = SerialCT(dom_lo, dom_size, tup)
    rng = G.Rng(seed)
    full = [np.ones(d, bool) for d in dom_size]
    w = _pack(full)
    st = ct.propagate(w)
    st_o, root, valid = O.gac_table(tup_ret, dom_lo, full)
    assert st == st_o == O.OK
    ct.save()
    masks, d, seen = root, 0, {"ok": 0, "fail": 0}
    for k in range(calls):
        ct.save()
        new = edit(rng, masks)
        w = _pack(new)
        st = ct.propagate(w)
        st_o, out_o, valid = O.gac_table(tup_ret, dom_lo, new)
        assert st == st_o, k
        d += 1
        if st == O.OK:
            got = _unpack(w, dom_size)
            for i in range(len(dom_size)):
                assert np.array_equal(got[i], out_o[i]), (k, i)
            words_o = O.currtable_words(valid)
            assert np.array_equal(ct.currtable(len(words_o)), words_o), k
            seen["ok"] += 1
        else:
            seen["fail"] += 1
        if st != O.OK or d >= depth:
            assert ct.restore(1) == 0
            ct.save()
            masks, d = root, 0
        else:
            masks = out_o
    ct.close()
    return seen


def test_tiny_stream_matches_oracle():
    dom_lo, dom_size, tup = G.tiny_table(seed=1)
    seen = _stream(dom_lo, dom_size, tup, 600, 3,
                   lambda rng, m: G.remove_random_values(rng, m, 1 + rng.int(4))[0], depth=12)
    assert seen["ok"] > 0 and seen["fail"] > 0


@pytest.mark.parametrize("t", [1000, 20000])
def test_delta_reset_stream_matches_oracle(t):
    dom_lo, dom_size, tup = G.large_table(5 + t, t)

    def edit(rng, m):
        new, i = (G.delta_step if rng.int(2) == 0 else G.reset_step)(rng, m)
        return new if i is not None else G.remove_random_values(rng, m, 1)[0]

    _stream(dom_lo, dom_size, tup, 120, 7, edit)


def test_empty_and_grown_domains():
    ct = SerialCT([0, 0], [3, 3], np.zeros((0, 2), np.int32))
    assert ct.create_status == 1
    assert ct.propagate(_pack([np.ones(3, bool), np.ones(3, bool)])) == 1
    dom_lo, dom_size, tup = G.tiny_table(seed=2)
    ct = SerialCT(dom_lo, dom_size, tup)
    m = [np.ones(8, bool) for _ in range(3)]
    m[0][:3] = False
    assert ct.propagate(_pack(m)) in (0, 1)
    assert ct.propagate(_pack([np.ones(8, bool) for _ in range(3)])) in (-4, -1)
