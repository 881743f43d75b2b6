"""Pins of the CPU oracle to things other than itself (no GPU needed).

* values the paper prints for its worked examples (Table 1; the Sec. 4.2 launch
  example) stored under tests/golden/ with their citations;
* brute force on tiny inputs written as different code (per-value search over
  the tuple list, full enumeration of assignments);
* closed-form solution counts and a search tree traced by hand;
* invariants of the GAC fixpoint.

The mutation tests at the end plant plausible mistakes in copies of oracle
functions and check that one of these pins catches each of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import inputs as G


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def _bits_str(row):
    return "".join("1" if b else "0" for b in row)


# --------------------------------------------------------------------------
# Table 1 (Sec. 2)
# --------------------------------------------------------------------------

def test_table1_supports_rows(golden_dir):
    g = _load(golden_dir, "table1.json")
    tup = g["tuples"]["rows"]
    lo, sz = g["scope_dom_lo"], g["scope_dom_size"]
    m = O.supports_matrix(tup, lo, sz)
    assert m.shape == (12, 5)
    for key, want in g["supports_rows"]["rows"].items():
        var, val = key.split(",")
        i = int(var[1:]) - 1
        assert _bits_str(m[O.support_row(i, int(val), lo, sz)]) == want, key


def _table1_masks(lo, sz, doms):
    masks = []
    for i in range(3):
        m = np.zeros(sz[i], dtype=bool)
        m[np.array(doms[i]) - lo[i]] = True
        masks.append(m)
    return masks


def test_table1_currtable_and_filter(golden_dir):
    """The printed currTable 01010 holds exactly tau_2 = (1,2,3) and tau_4 = (1,4,1), the two
    tuples with x1 = 1; with dom(x1) = {1} they are the valid ones, and projecting them
    leaves dom(x2) = {2,4} and dom(x3) = {1,3}."""
    g = _load(golden_dir, "table1.json")
    lo, sz = g["scope_dom_lo"], g["scope_dom_size"]
    tup = O.retained_tuples(g["tuples"]["rows"], lo, sz)
    ex = g["currtable_example"]
    masks = _table1_masks(lo, sz, [[1], [1, 2, 3, 4], [1, 2, 3, 4]])
    st, out, valid = O.gac_table(tup, lo, masks)
    assert st == O.OK
    assert _bits_str(valid) == ex["currtable"]
    # packed words: tau_j at bit j-1 of word 0
    words = O.currtable_words(valid)
    want = sum(1 << j for j, c in enumerate(ex["currtable"]) if c == "1")
    assert words.tolist() == [want]
    for i, want_vals in enumerate([[1], [2, 4], [1, 3]]):
        assert (np.flatnonzero(out[i]) + lo[i]).tolist() == want_vals


def test_table1_root_gac(golden_dir):
    """Full domains: every tuple is valid; the columns of Table 1(a) carry x1 in {3,1,2},
    x2 in {1,2,3,4} and x3 in {1,3}, so 4 leaves dom(x1) and 2, 4 leave dom(x3)."""
    g = _load(golden_dir, "table1.json")
    lo, sz = g["scope_dom_lo"], g["scope_dom_size"]
    tup = O.retained_tuples(g["tuples"]["rows"], lo, sz)
    st, out, valid = O.gac_table(tup, lo, [np.ones(4, dtype=bool)] * 3)
    assert st == O.OK and valid.all()
    for i, want_vals in enumerate([[1, 2, 3], [1, 2, 3, 4], [1, 3]]):
        assert (np.flatnonzero(out[i]) + lo[i]).tolist() == want_vals


def test_table1_search_tree(golden_dir):
    """Tree traced by hand on the CSP made of Table 1(a) alone (first-fail, min value):
    root -> x3 is smallest {1,3};
      x3=1 -> {tau_1, tau_4}: x1 {1,3}, x2 {1,4}; pick x1 -> x1=1 (sol (1,4,1)), x1!=1 (sol);
      x3!=1 -> {tau_2, tau_3, tau_5}: x1 {1,2,3}, x2 {2,3,4}; pick x1 -> x1=1 (sol);
        x1!=1 -> x1 {2,3}, x2 {3,4}; pick x1 -> x1=2 (sol), x1!=2 (sol).
    9 nodes, 0 fails, 5 solutions; the first solution is (1,4,1)."""
    g = _load(golden_dir, "table1.json")
    csp = O.Csp(g["scope_dom_lo"], g["scope_dom_size"])
    csp.add_table([0, 1, 2], g["tuples"]["rows"])
    st = O.dfs(csp, count_all=True)
    assert (st.nodes, st.fails, st.solutions) == (9, 0, 5)
    assert st.first_solution == [1, 4, 1]
    first = O.dfs(csp, count_all=False)
    assert (first.nodes, first.solutions, first.first_solution) == (3, 1, [1, 4, 1])


def test_hand_traced_tree_with_failures():
    """x0, x1, x2 in {0,1}; tables x0 = x1, x1 != x2, x0 = x2 (each GAC on full domains,
    jointly unsatisfiable). Root keeps all values; first-fail takes x0:
    x0=0 forces x1=0, x2=1, and x0 = x2 fails; x0!=0 forces x1=1, x2=0 and fails again.
    3 nodes, 2 fails, 0 solutions."""
    csp = O.Csp([0, 0, 0], [2, 2, 2])
    csp.add_table([0, 1], [[0, 0], [1, 1]])
    csp.add_table([1, 2], [[0, 1], [1, 0]])
    csp.add_table([0, 2], [[0, 0], [1, 1]])
    st, masks, _ = O.gac_network(csp, csp.full_masks())
    assert st == O.OK and all(m.all() for m in masks)
    res = O.dfs(csp, count_all=True)
    assert (res.nodes, res.fails, res.solutions) == (3, 2, 0)


# --------------------------------------------------------------------------
# Sec. 4.2 launch-arithmetic example: concatenated value-bit indexing
# --------------------------------------------------------------------------

def test_launch_example_value_indexing(golden_dir):
    g = _load(golden_dir, "launch_example.json")
    lo, sz = g["dom_lo"], g["dom_size"]
    nbits = sum(sz)
    assert nbits == g["domain_bits"]
    assert (nbits + 31) // 32 == g["words"]
    a, b = g["word1_values"]
    var = g["word1_var"]
    for v in range(lo[var], lo[var] + sz[var]):
        in_word1 = O.support_row(var, v, lo, sz) // 32 == 1
        assert in_word1 == (a <= v <= b), v
    # x2's first value follows x1's last one
    assert O.support_row(1, lo[1], lo, sz) == sz[0]


# --------------------------------------------------------------------------
# brute force on tiny inputs
# --------------------------------------------------------------------------

def _brute_supported(tuples, lo, masks):
    """Per-value search: is there a tuple carrying (x_i, a) whose every entry is in its domain?"""
    out = []
    for i in range(len(masks)):
        m = np.zeros_like(masks[i])
        for a in range(len(masks[i])):
            if not masks[i][a]:
                continue
            for tu in tuples:
                if tu[i] - lo[i] != a:
                    continue
                if all(masks[k][tu[k] - lo[k]] for k in range(len(masks))):
                    m[a] = True
                    break
        out.append(m)
    return out


def _random_masks(rng, sizes, p_keep=0.6):
    masks = []
    for d in sizes:
        m = rng.uniform(d) < p_keep
        if not m.any():
            m[rng.int(d)] = True
        masks.append(m)
    return masks


@pytest.mark.parametrize("seed", range(40))
def test_gac_table_matches_per_value_brute_force(seed):
    rng = G.Rng(1000 + seed)
    arity = 2 + rng.int(3)
    sizes = [2 + rng.int(5) for _ in range(arity)]
    lo = [rng.int(5) - 2 for _ in range(arity)]
    t = 1 + rng.int(30)
    # duplicates and out-of-range values on purpose
    cols = [rng.below(t, sizes[i] + 2).astype(np.int64) + lo[i] - 1 for i in range(arity)]
    raw = np.stack(cols, axis=1)
    tup = O.retained_tuples(raw, lo, sizes)
    masks = _random_masks(rng, sizes)
    st, out, valid = O.gac_table(tup, lo, masks)
    bf = _brute_supported(tup.tolist(), lo, masks)
    feasible = any(m.any() for m in bf) and all(m.any() for m in bf)
    if not feasible:
        assert st == O.INFEASIBLE
        return
    assert st == O.OK
    for i in range(arity):
        assert np.array_equal(out[i], bf[i])
    assert len(O.currtable_words(valid)) == (len(tup) + 31) // 32
    assert sum(bin(int(w)).count("1") for w in O.currtable_words(valid)) == int(valid.sum())


def _enumerate_solutions(csp):
    sols = []
    for assign in itertools.product(*[range(csp.dom_lo[v], csp.dom_lo[v] + csp.dom_size[v])
                                      for v in range(csp.nvars)]):
        ok = True
        for scope, tup in csp.tables:
            row = [assign[v] for v in scope]
            if not any(list(t) == row for t in tup.tolist()):
                ok = False
                break
        if ok:
            sols.append(assign)
    return sols


def _tiny_csp(seed, nvars, ntables, arity, d, t):
    rng = G.Rng(seed)
    csp = O.Csp([0] * nvars, [d] * nvars)
    for k in range(ntables):
        scope = G.random_scope(rng, nvars, arity)
        tt = G.cap_distinct([d] * arity, t)
        csp.add_table(scope, G.distinct_uniform_tuples(G.derive_seed(seed, k), [0] * arity, [d] * arity, tt))
    return csp


@pytest.mark.parametrize("seed", range(12))
def test_network_and_search_match_enumeration(seed):
    csp = _tiny_csp(77 + seed, nvars=5, ntables=3, arity=3, d=4, t=20 + 3 * seed)
    sols = _enumerate_solutions(csp)
    st, masks, _ = O.gac_network(csp, csp.full_masks())
    if st == O.OK:
        # soundness: no value of any solution is pruned
        for s in sols:
            for v in range(csp.nvars):
                assert masks[v][s[v] - csp.dom_lo[v]]
        # fixpoint: every table is GAC on the result
        for scope, tup in csp.tables:
            st2, out, _ = O.gac_table(tup, [csp.dom_lo[v] for v in scope], [masks[v] for v in scope])
            assert st2 == O.OK
            for k, v in enumerate(scope):
                assert np.array_equal(out[k], masks[v])
    else:
        assert sols == []
    res = O.dfs(csp, count_all=True)
    assert res.solutions == len(sols)
    assert res.complete
    if sols:
        first = O.dfs(csp, count_all=False)
        assert tuple(first.first_solution) in set(sols)
        assert first.solutions == 1


def test_one_table_closed_form_count_tiny_config():
    dom_lo, dom_size, tup = G.tiny_table(seed=1)
    assert len({tuple(r) for r in tup.tolist()}) == 200
    csp = O.Csp(dom_lo, dom_size)
    csp.add_table([0, 1, 2], tup)
    st = O.dfs(csp, count_all=True)
    assert st.solutions == 200 and st.complete


@pytest.mark.parametrize("seed", range(8))
def test_search_tree_identity_single_table(seed):
    """On a CSP of one table, GAC domains equal the projections of the solutions left in
    the domains, so a search whose propagator projects brute-force solution sets must
    visit the identical tree: same nodes, fails and solutions."""
    rng = G.Rng(500 + seed)
    arity, d = 3, 4
    t = 6 + rng.int(30)
    tup = G.distinct_uniform_tuples(G.derive_seed(seed, 9), [0] * arity, [d] * arity, t)
    csp = O.Csp([0] * arity, [d] * arity)
    csp.add_table(list(range(arity)), tup)
    rows = [tuple(r) for r in tup.tolist()]

    def project(masks):
        live = [r for r in rows if all(masks[i][r[i]] for i in range(arity))]
        if not live:
            return O.INFEASIBLE, masks
        out = [np.zeros(d, dtype=bool) for _ in range(arity)]
        for r in live:
            for i in range(arity):
                out[i][r[i]] = True
        return O.OK, out

    a = O.dfs(csp, count_all=True)
    b = O.dfs(csp, count_all=True, propagate=project)
    assert (a.nodes, a.fails, a.solutions) == (b.nodes, b.fails, b.solutions)
    assert a.solutions == len(set(rows))


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_idempotence_and_monotonicity(seed):
    dom_lo, dom_size, tup = G.tiny_table(seed=seed + 3)
    tup = O.retained_tuples(tup, dom_lo, dom_size)
    rng = G.Rng(seed)
    masks = _random_masks(rng, dom_size, p_keep=0.7)
    st, out, valid = O.gac_table(tup, dom_lo, masks)
    if st == O.INFEASIBLE:
        return
    for i in range(3):
        assert not (out[i] & ~masks[i]).any()
    st2, out2, valid2 = O.gac_table(tup, dom_lo, out)
    assert st2 == O.OK
    assert np.array_equal(valid, valid2)
    for i in range(3):
        assert np.array_equal(out[i], out2[i])


def test_empty_and_out_of_range_inputs():
    lo, sz = [0, 0], [3, 3]
    assert O.retained_tuples(np.zeros((0, 2), dtype=np.int32), lo, sz).shape == (0, 2)
    tup = O.retained_tuples([[0, 0], [3, 0], [-1, 2], [2, 2], [2, 2]], lo, sz)
    assert tup.tolist() == [[0, 0], [2, 2], [2, 2]]
    st, out, valid = O.gac_table(tup, lo, [np.ones(3, bool), np.ones(3, bool)])
    assert st == O.OK and valid.tolist() == [True, True, True]
    assert out[0].tolist() == [True, False, True]
    st, _, _ = O.gac_table(tup[:0], lo, [np.ones(3, bool), np.ones(3, bool)])
    assert st == O.INFEASIBLE
    st, _, _ = O.gac_table(tup, lo, [np.zeros(3, bool), np.ones(3, bool)])
    assert st == O.INFEASIBLE


# --------------------------------------------------------------------------
# planted mistakes: each one must be caught by a pin above
# --------------------------------------------------------------------------

def _valid_drop_last_column(tup, dom_lo, masks):
    valid = np.ones(tup.shape[0], dtype=bool)
    for i in range(tup.shape[1] - 1):
        valid &= masks[i][tup[:, i] - int(dom_lo[i])]
    return valid


def _valid_transposed(tup, dom_lo, masks):
    valid = np.ones(tup.shape[0], dtype=bool)
    n = tup.shape[1]
    for i in range(n):
        j = (i + 1) % n
        valid &= masks[j][np.minimum(tup[:, i] - int(dom_lo[i]), len(masks[j]) - 1)]
    return valid


@pytest.mark.parametrize("mutant", [_valid_drop_last_column, _valid_transposed])
def test_pins_catch_planted_validity_mistakes(monkeypatch, mutant):
    monkeypatch.setattr(O, "valid_mask", mutant)
    caught = False
    for seed in range(40):
        try:
            test_gac_table_matches_per_value_brute_force(seed)
        except AssertionError:
            caught = True
            break
    assert caught


def test_pins_catch_planted_bit_order_mistake(monkeypatch, golden_dir):
    def msb_first(bits):
        bits = np.asarray(bits, dtype=bool)
        nw = (bits.shape[0] + 31) // 32
        w = np.zeros(nw, dtype=np.uint64)
        for j in np.flatnonzero(bits):
            w[j // 32] |= np.uint64(1) << np.uint64(31 - j % 32)
        return w.astype(np.uint32)
    monkeypatch.setattr(O, "pack_words", msb_first)
    with pytest.raises(AssertionError):
        test_table1_currtable_and_filter(golden_dir)


def test_pins_catch_planted_row_offset_mistake(monkeypatch, golden_dir):
    def off_by_one(i, v, dom_lo, dom_size):
        return sum(int(d) for d in dom_size[:i]) + int(v) - int(dom_lo[i]) + (1 if i > 0 else 0)
    monkeypatch.setattr(O, "support_row", off_by_one)
    with pytest.raises((AssertionError, IndexError)):
        test_table1_supports_rows(golden_dir)
        test_launch_example_value_indexing(golden_dir)


def test_pins_catch_planted_branching_mistake(monkeypatch, golden_dir):
    def max_first(masks):
        best, bs = None, None
        for v, m in enumerate(masks):
            s = int(m.sum())
            if s > 1 and (bs is None or s >= bs):
                best, bs = v, s
        return best
    monkeypatch.setattr(O, "select_first_fail", max_first)
    with pytest.raises(AssertionError):
        test_table1_search_tree(golden_dir)


# --------------------------------------------------------------------------
# currTable packing beyond word 0 (Sec. 3: 32-bit words)
# --------------------------------------------------------------------------

def test_pack_words_multiword_hand_computed():
    """Tuple j sits at word j // 32, bit j % 32 (Sec. 3 fixes 32-bit words; the bit
    order is the reading pinned by Table 1(c)). Worked by hand: 70 tuples with
    validity bits at 0, 31, 32, 33 and 69 give word 0 = bits 0 and 31 =
    0x80000001, word 1 = bits 0 and 1 = 0x3, word 2 = bit 5 (69 - 64) = 0x20."""
    bits = np.zeros(70, dtype=bool)
    bits[[0, 31, 32, 33, 69]] = True
    assert O.pack_words(bits).tolist() == [0x80000001, 0x3, 0x20]
    # word count: ceil(t / 32); a 97th tuple opens a fourth word
    assert O.pack_words(np.zeros(96, dtype=bool)).tolist() == [0, 0, 0]
    b97 = np.zeros(97, dtype=bool)
    b97[96] = True
    assert O.pack_words(b97).tolist() == [0, 0, 0, 1]
    # currTable of a table is the packed validity vector: tuples 32..63 valid
    # (value 1 of a unary table) fill word 1 and nothing else
    tup = np.array([[0]] * 32 + [[1]] * 32 + [[0]] * 6, dtype=np.int64)
    st, _, valid = O.gac_table(tup, [0], [np.array([False, True])])
    assert st == O.OK
    assert O.currtable_words(valid).tolist() == [0, 0xFFFFFFFF, 0]


def _pack_reversed_words(bits):
    bits = np.asarray(bits, dtype=bool)
    nw = (bits.shape[0] + 31) // 32
    w = np.zeros(nw, dtype=np.uint64)
    for j in np.flatnonzero(bits):
        w[nw - 1 - j // 32] |= np.uint64(1) << np.uint64(j % 32)
    return w.astype(np.uint32)


def _pack_split_off_by_one(bits):
    bits = np.asarray(bits, dtype=bool)
    nw = (bits.shape[0] + 31) // 32
    w = np.zeros(nw, dtype=np.uint64)
    for j in np.flatnonzero(bits):
        w[min(j // 31, nw - 1)] |= np.uint64(1) << np.uint64(j % 32)
    return w.astype(np.uint32)


@pytest.mark.parametrize("mutant", [_pack_reversed_words, _pack_split_off_by_one])
def test_pins_catch_planted_word_index_mistakes(monkeypatch, mutant, golden_dir):
    """Both mutants pass the Table 1 pins (5 tuples, one word) but not the multi-word pin."""
    monkeypatch.setattr(O, "pack_words", mutant)
    test_table1_currtable_and_filter(golden_dir)
    with pytest.raises(AssertionError):
        test_pack_words_multiword_hand_computed()
