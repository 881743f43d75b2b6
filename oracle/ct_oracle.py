"""CPU oracle for Compact-Table propagation: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The library (``paper_2507_18413_gb300``)
never imports it and has no CPU fallback.

What it computes is the plain definition that Compact-Table reaches exactly
(Sec. 2): a table constraint is GAC when every value left in a domain appears
in some *valid* tuple, i.e. a tuple whose every component lies in the current
domain of its variable. The oracle scans the tuple list for validity (an
STR-style linear scan) and projects the valid tuples onto each variable. It
shares no code with the bitset path: it never builds a supports matrix to
propagate, never keeps a currTable between calls and has no delta/reset
choice. One pass is a fixpoint for a single table, because removing a value
that no valid tuple carries does not invalidate any valid tuple.

Representation. A domain is a numpy bool mask over the variable's initial
range ``[dom_lo, dom_lo + dom_size)``. Tuples are int32 rows of actual values.

Readings of points the paper leaves open (each is listed with its reason in
the design notes):
  * tuples with a component outside the initial domain are dropped when a
    table is built; duplicates are kept; tuple j is the j-th retained tuple
    in input order;
  * currTable is packed into 32-bit words (Sec. 3, ``_currTable``), tuple j at
    word j >> 5, bit j & 31 (least significant bit first);
  * the support row of value v of the i-th scope variable is
    ``jmp[i] + v - dom_lo[i]`` with ``jmp`` the exclusive prefix sum of the
    initial domain sizes (Sec. 3, ``_supportJmp`` and ``_variablesOffsets``);
  * search is depth-first with first-fail binary branching (smallest domain
    among unfixed variables, ties to the lowest index; left branch x = min D,
    right branch x != min D); a node is every fixpoint computed on a search
    node, including the root and failed nodes.

Parity: every function here is pinned by tests in ``tests/test_oracle_pins.py``
against the paper's worked example (Table 1), the launch-arithmetic example of
Sec. 4.2, brute force on tiny inputs, closed-form solution counts and
invariants.
"""
from __future__ import annotations

import numpy as np

OK = 0
INFEASIBLE = 1


# --------------------------------------------------------------------------
# table construction (Sec. 2 definitions; Sec. 3 constructor)
# --------------------------------------------------------------------------

def retained_tuples(tuples, dom_lo, dom_size) -> np.ndarray:
    """Tuples whose every component lies in the initial domain, in input order."""
    tuples = np.asarray(tuples, dtype=np.int64).reshape(-1, len(dom_lo))
    lo = np.asarray(dom_lo, dtype=np.int64)
    hi = lo + np.asarray(dom_size, dtype=np.int64)
    keep = np.all((tuples >= lo) & (tuples < hi), axis=1)
    return tuples[keep]


def support_row(i: int, v: int, dom_lo, dom_size) -> int:
    """Row of the supports matrix for value v of scope position i (Sec. 3, _supportJmp)."""
    jmp = 0
    for k in range(i):
        jmp += int(dom_size[k])
    return jmp + int(v) - int(dom_lo[i])


def supports_matrix(tuples, dom_lo, dom_size) -> np.ndarray:
    """The static supports matrix of Sec. 2: bool [sum(dom_size), t].

    Cell (row of [x_i, v], j) is set iff the j-th tuple has value v at position i.
    """
    tup = retained_tuples(tuples, dom_lo, dom_size)
    rows = int(sum(int(d) for d in dom_size))
    m = np.zeros((rows, tup.shape[0]), dtype=bool)
    for i in range(len(dom_lo)):
        for v in range(int(dom_lo[i]), int(dom_lo[i]) + int(dom_size[i])):
            m[support_row(i, v, dom_lo, dom_size)] = tup[:, i] == v
    return m


def pack_words(bits: np.ndarray) -> np.ndarray:
    """Pack a bool vector into uint32 words, bit j at word j // 32, position j % 32."""
    bits = np.asarray(bits, dtype=bool)
    nw = (bits.shape[0] + 31) // 32
    words = np.zeros(nw, dtype=np.uint64)
    for j in np.flatnonzero(bits):
        words[j // 32] |= np.uint64(1) << np.uint64(j % 32)
    return words.astype(np.uint32)


# --------------------------------------------------------------------------
# single-table GAC (Sec. 2 definition; the fixed point Algorithms 1-3 reach)
# --------------------------------------------------------------------------

def valid_mask(tup: np.ndarray, dom_lo, masks) -> np.ndarray:
    """Tuple j is valid iff tup[j, i] is in the current domain of x_i for every i (Sec. 2)."""
    valid = np.ones(tup.shape[0], dtype=bool)
    for i in range(tup.shape[1]):
        valid &= masks[i][tup[:, i] - int(dom_lo[i])]
    return valid


def gac_table(tup: np.ndarray, dom_lo, masks):
    """GAC filtering of one table on the given domains.

    ``tup`` holds the retained tuples (see :func:`retained_tuples`). Returns
    ``(status, new_masks, valid)``: status INFEASIBLE when no tuple is valid or a
    domain is empty (Alg. 1 fails when currTable is all zero); otherwise each new
    domain is the set of values carried by valid tuples, and ``valid`` is the
    validity vector whose packed words are currTable.
    """
    masks = [np.asarray(m, dtype=bool) for m in masks]
    if any(not m.any() for m in masks):
        return INFEASIBLE, masks, np.zeros(tup.shape[0], dtype=bool)
    valid = valid_mask(tup, dom_lo, masks)
    if not valid.any():
        return INFEASIBLE, masks, valid
    out = []
    for i in range(tup.shape[1]):
        m = np.zeros_like(masks[i])
        m[tup[valid, i] - int(dom_lo[i])] = True
        out.append(m)
    return OK, out, valid


def currtable_words(valid: np.ndarray) -> np.ndarray:
    """currTable (Sec. 2) as 32-bit words (Sec. 3)."""
    return pack_words(valid)


# --------------------------------------------------------------------------
# networks of tables and search (Sec. 4: MiniCP alternates search and propagation)
# --------------------------------------------------------------------------

class Csp:
    """Variables with initial ranges and table constraints over them."""

    def __init__(self, dom_lo, dom_size):
        self.dom_lo = [int(v) for v in dom_lo]
        self.dom_size = [int(v) for v in dom_size]
        self.tables = []  # list of (scope, retained tuples)

    @property
    def nvars(self):
        return len(self.dom_lo)

    def add_table(self, scope, tuples):
        scope = [int(v) for v in scope]
        lo = [self.dom_lo[v] for v in scope]
        sz = [self.dom_size[v] for v in scope]
        self.tables.append((scope, retained_tuples(tuples, lo, sz)))

    def full_masks(self):
        return [np.ones(d, dtype=bool) for d in self.dom_size]


def gac_network(csp: Csp, masks):
    """Greatest common fixpoint of single-table GAC over all tables.

    Repeats passes over the tables until no domain changes or a table fails.
    The GAC closure is unique, so the order of the passes does not matter.
    Returns ``(status, masks, table_calls)``.
    """
    masks = [np.asarray(m, dtype=bool).copy() for m in masks]
    if any(not m.any() for m in masks):
        return INFEASIBLE, masks, 0
    calls = 0
    changed = True
    while changed:
        changed = False
        for scope, tup in csp.tables:
            lo = [csp.dom_lo[v] for v in scope]
            st, out, _ = gac_table(tup, lo, [masks[v] for v in scope])
            calls += 1
            if st == INFEASIBLE:
                return INFEASIBLE, masks, calls
            for k, v in enumerate(scope):
                if not np.array_equal(out[k], masks[v]):
                    masks[v] = out[k]
                    changed = True
    return OK, masks, calls


class SearchStats:
    def __init__(self):
        self.nodes = 0
        self.fails = 0
        self.solutions = 0
        self.complete = True
        self.first_solution = None
        self.max_depth = 0

    def as_dict(self):
        return dict(nodes=self.nodes, fails=self.fails, solutions=self.solutions,
                    complete=self.complete, max_depth=self.max_depth)


def select_first_fail(masks):
    """Unfixed variable with the smallest domain, ties to the lowest index; None if all fixed."""
    best, best_size = None, None
    for v, m in enumerate(masks):
        s = int(m.sum())
        if s > 1 and (best_size is None or s < best_size):
            best, best_size = v, s
    return best


def dfs(csp: Csp, masks=None, node_limit: int = 1 << 62, count_all: bool = True,
        propagate=None, select=None, value=None) -> SearchStats:
    """Depth-first search with binary branching.

    Defaults: first-fail variable choice and the minimum value; the left branch fixes
    x to the value, the right branch removes it. ``propagate(masks) -> (status, masks)``
    defaults to :func:`gac_network`. The search stops at the node limit (stats marked
    incomplete) or, unless ``count_all``, at the first solution.
    """
    if masks is None:
        masks = csp.full_masks()
    if propagate is None:
        def propagate(m):
            st, out, _ = gac_network(csp, m)
            return st, out
    if select is None:
        select = select_first_fail
    if value is None:
        def value(m):
            return int(np.flatnonzero(m)[0])
    st = SearchStats()

    def node(m, depth):
        if st.nodes >= node_limit:
            st.complete = False
            return True
        st.nodes += 1
        st.max_depth = max(st.max_depth, depth)
        s, m = propagate(m)
        if s == INFEASIBLE:
            st.fails += 1
            return False
        x = select(m)
        if x is None:
            st.solutions += 1
            if st.first_solution is None:
                st.first_solution = [csp.dom_lo[v] + int(np.flatnonzero(mm)[0])
                                     for v, mm in enumerate(m)]
            return not count_all
        a = value(m[x])
        left = [mm.copy() for mm in m]
        left[x][:] = False
        left[x][a] = True
        if node(left, depth + 1):
            return True
        right = [mm.copy() for mm in m]
        right[x][a] = False
        return node(right, depth + 1)

    node([np.asarray(mm, dtype=bool).copy() for mm in masks], 0)
    return st
