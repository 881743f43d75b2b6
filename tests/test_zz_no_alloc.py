"""ct_propagate_noalloc, the propagation entry point that allocates nothing.

Callers whose device memory belongs to someone else at propagation time (a
framework's memory pool, a service that allocates only at start-up, code that
must not trigger the implicit synchronisation of cudaMalloc/cudaFree) hand the
library every buffer: supports, currTable, domains and last domains. The
library keeps its scratch in one static device array and calls no allocator.
Here that entry point must give exactly what ct_propagate gives (domains,
currTable words, changed variables, status) on two calls in a row, match the
oracle along a stream (a reset, a delta, a call with no change, a wipe-out,
a grown domain), serve a larger and then a smaller table from the same
scratch, leave device memory untouched after its first call, and report a
barrier wait that ran out. The file is collected last so that a run stopping
at the first failure has run every other test before it; it also passes when
run alone in a fresh process.
"""
import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


class CallerBuffers:
    """The buffers a caller of ct_propagate_noalloc owns (allocated here by torch,
    up front): supports rows, currTable, domains, last domains."""

    def __init__(self, torch, h, dom_size):
        info = C.ct_get_info(h)[1]
        self.torch = torch
        self.size = list(dom_size)
        self.W, W4, R = info["words"], info["chunks"], info["rows"]
        self.t = info["tuples"]
        Wp = 4 * W4
        sup = np.zeros((R, Wp), np.uint32)
        for r in range(R):
            st, row = C.ct_get_support_row(h, r, self.W)
            assert st == C.CT_OK
            sup[r, : self.W] = row
        self.sup = torch.from_numpy(sup.view(np.int32)).cuda()
        curr = np.zeros(Wp, np.uint32)
        curr[: self.t // 32] = 0xFFFFFFFF
        if self.t % 32:
            curr[self.t // 32] = (1 << (self.t % 32)) - 1
        self.curr0 = torch.from_numpy(curr.view(np.int32).copy())
        self.full = torch.from_numpy(C.masks_to_words([np.ones(d, bool) for d in dom_size]).view(np.int32).copy())
        self.curr = self.curr0.cuda()
        self.last = self.full.cuda()
        self.dom = torch.zeros(self.full.shape[0], dtype=torch.int32, device="cuda")
        self.host = torch.zeros(self.full.shape[0], dtype=torch.int32).pin_memory()

    def reset(self):
        """Back to the table's initial state (the caller's own backtracking)."""
        self.curr.copy_(self.curr0)
        self.last.copy_(self.full)

    def call(self, masks, stream):
        self.host.copy_(self.torch.from_numpy(C.masks_to_words(masks).view(np.int32).copy()))
        self.dom.copy_(self.host)
        return C.ct_propagate_noalloc(self.size, self.t, self.sup, self.curr, self.dom, self.last, stream=stream)

    def masks(self):
        return C.words_to_masks(self.dom.cpu().numpy().view(np.uint32), self.size)

    def words(self):
        return self.curr.cpu().numpy().view(np.uint32)


def test_noalloc_matches_ct_propagate_on_two_calls_in_a_row():
    torch = torch_cuda()
    C.load()
    stream = torch.cuda.current_stream()
    # ragged sizes: 50,000 tuples -> 1,563 words -> 391 chunks (a partial last segment)
    dom_lo, dom_size, tup = G.large_table(seed=17, t=50_000, arity=5, d=20)
    st, h = C.ct_create(5, dom_lo, dom_size, tup, stream=stream)
    assert st == C.CT_OK, C.last_error()
    buf = CallerBuffers(torch, h, dom_size)
    W = buf.W
    dom_ref = torch.zeros_like(buf.dom)
    rng = G.Rng(5)
    masks = [np.ones(d, bool) for d in dom_size]
    for k in range(2):
        new, _ = G.reset_step(rng, masks) if k == 0 else G.delta_step(rng, masks)
        dom_ref.copy_(torch.from_numpy(C.masks_to_words(new).view(np.int32).copy()))
        st_ref, ch_ref = C.ct_propagate(h, dom_ref, 1)
        st_na, ch_na = buf.call(new, stream)
        assert st_ref == C.CT_OK, C.last_error()
        assert st_na == st_ref, C.last_error()
        assert torch.equal(buf.dom, dom_ref), f"call {k}: domains differ"
        st, ref_words, _ = C.ct_get_currtable(h, W)
        got = buf.words()
        assert np.array_equal(got[:W], ref_words), f"call {k}: currTable differs"
        assert not got[W:].any()
        assert ch_na == int(ch_ref[0]), f"call {k}: changed variables differ"
        assert torch.equal(buf.last, dom_ref), f"call {k}: last domains are not the output"
        masks = C.words_to_masks(dom_ref.cpu().numpy().view(np.uint32), dom_size)
    C.ct_destroy(h)


def _oracle_check(buf, tup_ret, dom_lo, new, st_na):
    st_o, out_o, valid = O.gac_table(tup_ret, dom_lo, new)
    assert st_na == st_o, (st_na, st_o, C.last_error())
    if st_o == O.OK:
        got = buf.masks()
        for i in range(len(new)):
            assert np.array_equal(got[i], out_o[i]), f"domain of x{i} differs"
        w = buf.words()
        assert np.array_equal(w[: buf.W], O.currtable_words(valid)), "currTable differs"
        assert not w[buf.W:].any()
    return st_o, out_o


def _no_tuple_assignment(tup_ret, dom_lo, masks):
    """Singleton domains inside `masks` whose values no retained tuple holds together."""
    import itertools
    used = {tuple(r) for r in (tup_ret - np.asarray(dom_lo)).tolist()}
    firsts = [np.flatnonzero(m)[:2].tolist() for m in masks]
    for combo in itertools.product(*firsts):
        if combo not in used:
            new = [np.zeros(len(m), bool) for m in masks]
            for i, a in enumerate(combo):
                new[i][a] = True
            return new
    raise AssertionError("every small combination is a tuple")


def test_noalloc_stream_matches_the_oracle_and_shares_the_scratch_between_tables():
    """A larger table and then a smaller one (different rows, chunks and
    segments) through the same static scratch, each along a stream checked
    against the oracle: reset and delta steps, a call with no domain change,
    a wipe-out (CT_INFEASIBLE, the caller then starts over from its own copy)
    and a grown domain (CT_ERR_STATE, the same as ct_propagate)."""
    torch = torch_cuda()
    C.load()
    stream = torch.cuda.current_stream()
    for seed, t, arity, d in ((23, 300_000, 6, 24), (29, 9_001, 3, 40)):
        dom_lo, dom_size, tup = G.large_table(seed, t, arity=arity, d=d)
        tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
        st, h = C.ct_create(arity, dom_lo, dom_size, tup, stream=stream)
        assert st == C.CT_OK
        buf = CallerBuffers(torch, h, dom_size)
        rng = G.Rng(G.derive_seed(seed, 1))
        root = [np.ones(x, bool) for x in dom_size]
        st, masks = _oracle_check(buf, tup_ret, dom_lo, root, buf.call(root, stream)[0])
        assert st == O.OK
        kinds = {"ok": 0, "same": 0, "fail": 0}
        for k in range(14):
            if k == 5:
                new = [m.copy() for m in masks]  # no change since the last call
                kinds["same"] += 1
            elif k == 9:
                # every variable fixed to one of its present values, together held
                # by no tuple: a wipe-out
                new = _no_tuple_assignment(tup_ret, dom_lo, masks)
            else:
                new, _ = (G.delta_step if k % 2 else G.reset_step)(rng, masks)
            st_na, ch = buf.call(new, stream)
            st, out = _oracle_check(buf, tup_ret, dom_lo, new, st_na)
            if st == O.INFEASIBLE:
                kinds["fail"] += 1
                buf.reset()
                st, masks = _oracle_check(buf, tup_ret, dom_lo, root, buf.call(root, stream)[0])
                continue
            kinds["ok"] += 1
            masks = out
        assert kinds["fail"] >= 1 and kinds["same"] == 1 and kinds["ok"] >= 8, kinds
        # a domain that grew since the last call: CT_ERR_STATE, as from ct_propagate
        grown = [m.copy() for m in masks]
        i = next(i for i, m in enumerate(grown) if not m.all())
        grown[i][np.flatnonzero(~grown[i])[0]] = True
        st_na, _ = buf.call(grown, stream)
        assert st_na == C.CT_ERR_STATE, (st_na, C.last_error())
        ref = torch.zeros_like(buf.dom)
        C.ct_propagate(h, ref.copy_(torch.from_numpy(C.masks_to_words(root).view(np.int32).copy())), 0)
        st_ref, _ = C.ct_propagate(h, ref.copy_(torch.from_numpy(C.masks_to_words(masks).view(np.int32).copy())), 0)
        st_ref, _ = C.ct_propagate(h, ref.copy_(torch.from_numpy(C.masks_to_words(grown).view(np.int32).copy())), 0)
        assert st_ref == C.CT_ERR_STATE
        C.ct_destroy(h)


def test_noalloc_allocates_nothing_after_its_first_call():
    """After the first call (which looks the scratch array up), further calls
    leave torch's allocator and the device's free memory unchanged."""
    torch = torch_cuda()
    C.load()
    stream = torch.cuda.current_stream()
    dom_lo, dom_size, tup = G.large_table(31, 120_000, arity=5, d=16)
    st, h = C.ct_create(5, dom_lo, dom_size, tup, stream=stream)
    assert st == C.CT_OK
    buf = CallerBuffers(torch, h, dom_size)
    rng = G.Rng(8)
    root = [np.ones(x, bool) for x in dom_size]
    assert buf.call(root, stream)[0] == C.CT_OK
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    masks = root
    for k in range(8):
        new, _ = (G.delta_step if k % 2 else G.reset_step)(rng, masks)
        st, _ = buf.call(new, stream)
        assert st >= 0, C.last_error()
        if st == C.CT_INFEASIBLE:
            buf.reset()
            masks = root
        else:
            masks = buf.masks()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    C.ct_destroy(h)


def test_noalloc_reports_a_barrier_wait_that_ran_out():
    """The test hook makes every barrier wait of the next call run out (no
    fault, no hang): the kernel returns without publishing and the call
    returns CT_ERR_TIMEOUT; the next call starts afresh and matches the oracle."""
    torch = torch_cuda()
    C.load()
    stream = torch.cuda.current_stream()
    dom_lo, dom_size, tup = G.large_table(37, 40_000, arity=4, d=18)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    st, h = C.ct_create(4, dom_lo, dom_size, tup, stream=stream)
    assert st == C.CT_OK
    buf = CallerBuffers(torch, h, dom_size)
    root = [np.ones(x, bool) for x in dom_size]
    assert C.ct_arm_wait_timeout(None, 1500) == C.CT_OK
    st, _ = buf.call(root, stream)
    assert st == C.CT_ERR_TIMEOUT, (st, C.last_error())
    buf.reset()  # the timed-out call may have left the caller's buffers half-updated
    st, masks = _oracle_check(buf, tup_ret, dom_lo, root, buf.call(root, stream)[0])
    assert st == O.OK
    new, _ = G.reset_step(G.Rng(2), masks)
    _oracle_check(buf, tup_ret, dom_lo, new, buf.call(new, stream)[0])
    C.ct_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch_cuda()
    C.load()
    fake = 1 << 20  # never dereferenced: the sizes are refused first
    st, _ = C.ct_propagate_noalloc([4] * 17, 10, fake, fake, fake, fake)
    assert st == C.CT_ERR_ARG and "arity" in C.last_error()
    st, _ = C.ct_propagate_noalloc([1000, 100], 10, fake, fake, fake, fake)
    assert st == C.CT_ERR_ARG and "limits" in C.last_error()
    st, _ = C.ct_propagate_noalloc([4, 4], 9_000_000, fake, fake, fake, fake)
    assert st == C.CT_ERR_ARG and "limits" in C.last_error()
