"""Python binding of libct.so (ctypes): argument marshalling only.

Every function keeps the name of the C entry point it wraps (include/ct.h)
and returns the C status code together with any outputs. Device buffers are
passed as torch CUDA tensors (or raw device addresses); PyTorch provides the
device memory and the stream, all propagation work runs in the library's
CUDA kernels. There is no CPU fallback: if libct.so has not been built the
first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CT_STAR = -2**31  # wildcard component of a short tuple
CT_OK = 0
CT_INFEASIBLE = 1
CT_ERR_ARG = -1
CT_ERR_OOM = -2
CT_ERR_CUDA = -3
CT_ERR_STATE = -4
CT_ERR_TIMEOUT = -5
CT_ERR_LEVEL = -6


class CtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class ct_options(ctypes.Structure):
    _fields_ = [("reserved0", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("no_residues", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("host_fixpoint", ctypes.c_int32), ("autotune", ctypes.c_int32), ("copy_state", ctypes.c_int32),
                ("shard", ctypes.c_int32), ("no_split", ctypes.c_int32), ("no_early_filter", ctypes.c_int32)]


class ct_table_info(ctypes.Structure):
    _fields_ = [("arity", ctypes.c_int32), ("rows", ctypes.c_int32), ("tuples", ctypes.c_int64),
                ("words", ctypes.c_int64), ("chunks", ctypes.c_int64), ("segments", ctypes.c_int32),
                ("seg_capacity", ctypes.c_int32), ("live_chunks", ctypes.c_int64),
                ("trail_size", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("local_plan", ctypes.c_int32), ("grid_blocks", ctypes.c_int32), ("short_tuples", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("loads_in_flight", ctypes.c_int32), ("autotuned", ctypes.c_int32)]


class ct_call_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("changed_vars", ctypes.c_int32),
                ("delta_vars", ctypes.c_int32), ("reset_vars", ctypes.c_int32),
                ("rows_ored", ctypes.c_int32), ("sup_vars", ctypes.c_int32),
                ("residue_hits", ctypes.c_int32), ("local_found", ctypes.c_int32),
                ("hard", ctypes.c_int32), ("windows", ctypes.c_int32),
                ("pruned", ctypes.c_int32), ("trail_added", ctypes.c_int32),
                ("live_chunks_in", ctypes.c_int64), ("live_chunks_out", ctypes.c_int64),
                ("live_words_in", ctypes.c_int64), ("update_bytes", ctypes.c_int64),
                ("filter_bytes", ctypes.c_int64), ("phase_ns", ctypes.c_int32 * 4),
                ("early_filter", ctypes.c_int32)]


class ct_profile(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("kernel_ms", ctypes.c_double), ("update_bytes", ctypes.c_int64),
                ("filter_bytes", ctypes.c_int64), ("device_ms", ctypes.c_double), ("host_ms", ctypes.c_double),
                ("launch_ms", ctypes.c_double), ("wait_ms", ctypes.c_double)]


class ct_search_stats(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_int64), ("fails", ctypes.c_int64), ("solutions", ctypes.c_int64),
                ("propagations", ctypes.c_int64), ("max_depth", ctypes.c_int32),
                ("complete", ctypes.c_int32), ("seconds", ctypes.c_double)]


class ct_model_stats(ctypes.Structure):
    _fields_ = [("fixpoints", ctypes.c_int64), ("rounds", ctypes.c_int64), ("propagations", ctypes.c_int64),
                ("residue_hits", ctypes.c_int64), ("window_hits", ctypes.c_int64), ("hard_values", ctypes.c_int64),
                ("update_bytes", ctypes.c_int64), ("filter_bytes", ctypes.c_int64), ("wait_seconds", ctypes.c_double),
                ("phase_seconds", ctypes.c_double * 8)]


class ct_batch_info(ctypes.Structure):
    _fields_ = [("open_nodes", ctypes.c_int64), ("split_nodes", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("steals", ctypes.c_int64), ("slot_nodes", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("residue_hits", ctypes.c_int64), ("window_hits", ctypes.c_int64), ("hard_values", ctypes.c_int64),
                ("update_bytes", ctypes.c_int64), ("filter_bytes", ctypes.c_int64),
                ("slots", ctypes.c_int32), ("split_depth", ctypes.c_int32), ("setup_seconds", ctypes.c_double),
                ("wait_seconds", ctypes.c_double), ("slot_seconds", ctypes.c_double),
                ("phase_seconds", ctypes.c_double * 8)]


def _as_dict(s):
    out = {}
    for k, _ in s._fields_:
        v = getattr(s, k)
        out[k] = list(v) if isinstance(v, ctypes.Array) else v
    return out


_P = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_F32P = ctypes.POINTER(ctypes.c_float)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_I64P = ctypes.POINTER(ctypes.c_int64)

_SIGS = {
    "ct_create": (ctypes.c_int, [ctypes.c_int, _I32P, _I32P, _I32P, ctypes.c_int64,
                                 ctypes.POINTER(ct_options), _P, ctypes.POINTER(_P)]),
    "ct_propagate": (ctypes.c_int, [_P, _P, _U32P]),
    "ct_propagate_host": (ctypes.c_int, [_P, _U32P, _U32P]),
    "ct_save": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "ct_restore": (ctypes.c_int, [_P, ctypes.c_int]),
    "ct_get_currtable": (ctypes.c_int, [_P, _U32P, _I64P]),
    "ct_get_support_row": (ctypes.c_int, [_P, ctypes.c_int, _U32P]),
    "ct_get_index": (ctypes.c_int, [_P, _I32P, _I64P]),
    "ct_get_info": (ctypes.c_int, [_P, ctypes.POINTER(ct_table_info)]),
    "ct_get_call_stats": (ctypes.c_int, [_P, ctypes.POINTER(ct_call_stats)]),
    "ct_get_profile": (ctypes.c_int, [_P, ctypes.POINTER(ct_profile)]),
    "ct_reset_profile": (ctypes.c_int, [_P]),
    "ct_set_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "ct_destroy": (ctypes.c_int, [_P]),
    "ct_propagate_noalloc": (ctypes.c_int, [ctypes.c_int, _I32P, ctypes.c_int64, _P, _P, _P, _P, _U32P, _P]),
    "ct_arm_wait_timeout": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "ct_read_ceiling": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_float)]),
    "ct_debug_guard_buffers": (ctypes.c_int, [ctypes.c_int]),
    "ct_debug_check_guards": (ctypes.c_int, [_P, ctypes.c_int, _I64P]),
    "ct_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int]),
    "ct_debug_device_bytes": (ctypes.c_int, [_I64P]),
    "ct_shard_bounds": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _I64P]),
    "ct_sharded_create": (ctypes.c_int, [ctypes.c_int, _I32P, _I32P, _I32P, ctypes.c_int64, ctypes.c_int,
                                         _P, _P, ctypes.POINTER(_P)]),
    "ct_sharded_propagate": (ctypes.c_int, [_P, _P, _U32P]),
    "ct_sharded_save": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "ct_sharded_restore": (ctypes.c_int, [_P, ctypes.c_int]),
    "ct_sharded_get_currtable": (ctypes.c_int, [_P, _U32P, _I64P]),
    "ct_sharded_get_shard": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "ct_sharded_destroy": (ctypes.c_int, [_P]),
    "ct_model_create": (ctypes.c_int, [ctypes.c_int, _I32P, _I32P, ctypes.POINTER(ct_options), _P,
                                       ctypes.POINTER(_P)]),
    "ct_model_add_table": (ctypes.c_int, [_P, _I32P, ctypes.c_int, _I32P, ctypes.c_int64]),
    "ct_model_propagate": (ctypes.c_int, [_P]),
    "ct_model_get_domains": (ctypes.c_int, [_P, _U32P]),
    "ct_model_set_domains": (ctypes.c_int, [_P, _U32P]),
    "ct_model_save": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "ct_model_restore": (ctypes.c_int, [_P, ctypes.c_int]),
    "ct_search_dfs": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ct_search_stats), _I32P]),
    "ct_search_batch": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                       ctypes.POINTER(ct_search_stats), _I32P, ctypes.POINTER(ct_batch_info)]),
    "ct_search_batch_assign": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                              ctypes.POINTER(ct_search_stats), _I32P, ctypes.POINTER(ct_batch_info)]),
    "ct_search_batch_device": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                              ctypes.POINTER(ct_search_stats), _I32P, ctypes.POINTER(ct_batch_info)]),
    "ct_model_destroy": (ctypes.c_int, [_P]),
    "ct_create_negative": (ctypes.c_int, [ctypes.c_int, _I32P, _I32P, _I32P, ctypes.c_int64, ctypes.POINTER(ct_options),
                                          _P, ctypes.POINTER(_P)]),
    "ct_model_add_negative_table": (ctypes.c_int, [_P, _I32P, ctypes.c_int, _I32P, ctypes.c_int64]),
    "ct_model_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ct_model_stats)]),
    "ct_model_reset_stats": (ctypes.c_int, [_P]),
    "ct_mlp_create": (ctypes.c_int, [_F32P, _P, ctypes.POINTER(_P)]),
    "ct_mlp_set_weights": (ctypes.c_int, [_P, _F32P]),
    "ct_mlp_get_weights": (ctypes.c_int, [_P, _F32P]),
    "ct_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "ct_mlp_grad": (ctypes.c_int, [_P, _F32P, _F32P, ctypes.c_int, _F32P, _F32P]),
    "ct_mlp_train": (ctypes.c_int, [_P, _F32P, _F32P, ctypes.c_int64, _I32P, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_float, _F32P]),
    "ct_mlp_destroy": (ctypes.c_int, [_P]),
    "ct_model_features": (ctypes.c_int, [_P, _F32P]),
    "ct_model_set_policy": (ctypes.c_int, [_P, _P]),
    "ct_model_set_trace": (ctypes.c_int, [_P, _I32P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "ct_model_lookahead": (ctypes.c_int, [_P, ctypes.c_int, _F32P]),
    "ct_search_collect": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, _F32P, _F32P,
                                         ctypes.POINTER(ctypes.c_int64)]),
    "ct_last_error": (ctypes.c_char_p, []),
    "ct_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ct_version": (ctypes.c_int, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libct.so (built by paper_2507_18413_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libct.so not found at {p}; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def exported_names():
    return list(_SIGS)


def last_error() -> str:
    return load().ct_last_error().decode()


def status_string(st: int) -> str:
    try:
        return load().ct_status_string(int(st)).decode()
    except RuntimeError:
        return str(st)


def check(st: int) -> int:
    if st < 0:
        raise CtError(st, last_error())
    return st


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def _i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(_I32P)


def _u32_out(n):
    a = np.zeros(max(int(n), 1), dtype=np.uint32)
    return a, a.ctypes.data_as(_U32P)


def _dev_ptr(x) -> int:
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


_CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream as an explicit handle


def _stream_ptr(stream):
    """A torch stream (or raw handle) as a cudaStream_t. Torch's default stream has
    handle 0, which the C API reads as "no stream given"; it is passed as
    cudaStreamLegacy instead so that the library runs in order with torch."""
    if stream is None:
        return None
    h = stream if isinstance(stream, int) else int(stream.cuda_stream)
    return h if h != 0 else _CUDA_STREAM_LEGACY


def make_options(grid_blocks=0, no_residues=0, profile=0, host_fixpoint=0, copy_state=0, autotune=0, shard=0,
                 no_split=0, no_early_filter=0):
    o = ct_options()
    o.no_early_filter = no_early_filter
    o.no_split = no_split
    o.shard = shard
    o.autotune = autotune
    o.host_fixpoint = host_fixpoint
    o.copy_state = copy_state
    o.grid_blocks = grid_blocks
    o.no_residues = no_residues
    o.profile = profile
    return o


def dom_layout(dom_size):
    """Word offsets and word counts of domains stored back to back."""
    nw = [(int(d) + 31) // 32 for d in dom_size]
    off = np.concatenate([[0], np.cumsum(nw)]).astype(np.int64)
    return off, nw


def masks_to_words(masks) -> np.ndarray:
    """Domains as bool masks -> packed uint32 words (bit a of word a // 32 = value dom_lo + a)."""
    out = []
    for m in masks:
        m = np.asarray(m, dtype=bool)
        nw = (m.shape[0] + 31) // 32
        padded = np.zeros(nw * 32, dtype=bool)
        padded[: m.shape[0]] = m
        by = np.packbits(padded.reshape(-1, 8), axis=1, bitorder="little").reshape(-1)
        out.append(by.view("<u4").astype(np.uint32))
    return np.concatenate(out) if out else np.zeros(0, dtype=np.uint32)


def words_to_masks(words, dom_size):
    words = np.asarray(words, dtype=np.uint32)
    off, nw = dom_layout(dom_size)
    masks = []
    for i, d in enumerate(dom_size):
        w = words[off[i]: off[i] + nw[i]].astype("<u4")
        bits = np.unpackbits(w.view(np.uint8), bitorder="little")[: int(d)]
        masks.append(bits.astype(bool))
    return masks


# --------------------------------------------------------------------------
# table
# --------------------------------------------------------------------------

def ct_create(arity, dom_lo, dom_size, tuples, opt=None, stream=None, negative=False):
    """Returns (status, handle). tuples: int32 [t, arity] (host); negative=True
    makes them the forbidden tuples (ct_create_negative)."""
    L = load()
    lo, plo = _i32(dom_lo)
    sz, psz = _i32(dom_size)
    tup = np.ascontiguousarray(np.asarray(tuples, dtype=np.int32).reshape(-1, arity))
    t = tup.shape[0]
    ptup = tup.ctypes.data_as(_I32P) if t else None
    h = _P()
    fn = L.ct_create_negative if negative else L.ct_create
    st = fn(int(arity), plo, psz, ptup, int(t), ctypes.byref(opt) if opt is not None else None,
            _stream_ptr(stream), ctypes.byref(h))
    return st, h


def ct_shard_bounds(t, K):
    """Returns (status, int64 bounds[K + 1]) of the split of t retained tuples."""
    b = np.zeros(int(K) + 1, dtype=np.int64)
    st = load().ct_shard_bounds(int(t), int(K), b.ctypes.data_as(_I64P))
    return st, b


def ct_sharded_create(arity, dom_lo, dom_size, tuples, K, opt=None, stream=None):
    """Returns (status, handle) of the table split into K word-range shards."""
    lo, plo = _i32(dom_lo)
    sz, psz = _i32(dom_size)
    tup = np.ascontiguousarray(np.asarray(tuples, dtype=np.int32).reshape(-1, arity))
    t = tup.shape[0]
    h = _P()
    st = load().ct_sharded_create(int(arity), plo, psz, tup.ctypes.data_as(_I32P) if t else None, int(t), int(K),
                                  ctypes.byref(opt) if opt is not None else None, _stream_ptr(stream),
                                  ctypes.byref(h))
    return st, h


def ct_sharded_propagate(h, dom_bits, changed_words: int = 0):
    ch, pch = _u32_out(changed_words)
    st = load().ct_sharded_propagate(h, _dev_ptr(dom_bits), pch if changed_words else None)
    return st, ch[:changed_words]


def ct_sharded_save(h):
    lv = ctypes.c_int(-1)
    st = load().ct_sharded_save(h, ctypes.byref(lv))
    return st, lv.value


def ct_sharded_restore(h, level):
    return load().ct_sharded_restore(h, int(level))


def ct_sharded_get_currtable(h, nwords):
    w, pw = _u32_out(nwords)
    nz = ctypes.c_int64(0)
    st = load().ct_sharded_get_currtable(h, pw, ctypes.byref(nz))
    return st, w[:nwords], nz.value


def ct_sharded_get_shard(h, k):
    t = _P()
    st = load().ct_sharded_get_shard(h, int(k), ctypes.byref(t))
    return st, t


def ct_sharded_destroy(h):
    return load().ct_sharded_destroy(h)


def ct_propagate(h, dom_bits, changed_words: int = 0):
    """dom_bits: device buffer (torch tensor or address). Returns (status, changed uint32 words)."""
    ch, pch = _u32_out(changed_words)
    st = load().ct_propagate(h, _dev_ptr(dom_bits), pch if changed_words else None)
    return st, ch[:changed_words]


def ct_debug_guard_buffers(on):
    """Test hook: tables created from now on guard their device buffers (on=1) or not."""
    return load().ct_debug_guard_buffers(int(bool(on)))


def ct_debug_check_guards(h, poke=0):
    """Changed guard bytes of table h's buffers (poke > 0: corrupt that many first)."""
    n = ctypes.c_int64(0)
    st = load().ct_debug_check_guards(h, int(poke), ctypes.byref(n))
    return st, int(n.value)


def ct_debug_fail_alloc(n):
    """Test hook: the table-buffer allocation after the next n fails (n < 0: disarm)."""
    return load().ct_debug_fail_alloc(int(n))


def ct_debug_device_bytes():
    n = ctypes.c_int64(0)
    st = load().ct_debug_device_bytes(ctypes.byref(n))
    return st, int(n.value)


def ct_read_ceiling(buf, nbytes, stream=None, timed=False):
    """One streaming read of nbytes of the device buffer (a torch tensor or a raw
    device pointer), launched on stream. Returns the status, and with timed the
    CUDA-event interval around the launch in ms (the call then waits for it)."""
    if not timed:
        return load().ct_read_ceiling(_dev_ptr(buf), int(nbytes), _stream_ptr(stream), None)
    ms = ctypes.c_float(0.0)
    st = load().ct_read_ceiling(_dev_ptr(buf), int(nbytes), _stream_ptr(stream), ctypes.byref(ms))
    return st, float(ms.value)


def ct_arm_wait_timeout(h, polls):
    """Test hook: the next ct_propagate on h (None: the next ct_propagate_noalloc) runs
    its barrier waits out after `polls` polls and returns CT_ERR_TIMEOUT."""
    return load().ct_arm_wait_timeout(h, int(polls))


def ct_propagate_host(h, dom_words: np.ndarray, changed_words: int = 0):
    """dom_words: host uint32 array, filtered in place on CT_OK."""
    assert dom_words.dtype == np.uint32 and dom_words.flags["C_CONTIGUOUS"]
    ch, pch = _u32_out(changed_words)
    st = load().ct_propagate_host(h, dom_words.ctypes.data_as(_U32P), pch if changed_words else None)
    return st, ch[:changed_words]


def ct_save(h):
    lv = ctypes.c_int(-1)
    st = load().ct_save(h, ctypes.byref(lv))
    return st, lv.value


def ct_restore(h, level):
    return load().ct_restore(h, int(level))


def ct_get_currtable(h, nwords):
    w, pw = _u32_out(nwords)
    nz = ctypes.c_int64(0)
    st = load().ct_get_currtable(h, pw, ctypes.byref(nz))
    return st, w[:nwords], nz.value


def ct_get_support_row(h, row, nwords):
    w, pw = _u32_out(nwords)
    st = load().ct_get_support_row(h, int(row), pw)
    return st, w[:nwords]


def ct_get_index(h):
    n = ctypes.c_int64(0)
    L = load()
    st = L.ct_get_index(h, None, ctypes.byref(n))
    if st != CT_OK:
        return st, None
    a = np.zeros(max(n.value, 1), dtype=np.int32)
    st = L.ct_get_index(h, a.ctypes.data_as(_I32P), ctypes.byref(n))
    return st, a[: n.value]


def ct_get_info(h):
    i = ct_table_info()
    st = load().ct_get_info(h, ctypes.byref(i))
    return st, _as_dict(i)


def ct_get_call_stats(h):
    s = ct_call_stats()
    st = load().ct_get_call_stats(h, ctypes.byref(s))
    return st, _as_dict(s)


def ct_get_profile(h):
    p = ct_profile()
    st = load().ct_get_profile(h, ctypes.byref(p))
    return st, _as_dict(p)


def ct_reset_profile(h):
    return load().ct_reset_profile(h)


def ct_set_profile(h, on):
    return load().ct_set_profile(h, 1 if on else 0)


def ct_destroy(h):
    return load().ct_destroy(h)


def ct_propagate_noalloc(dom_size, t, supports, curr_table, dom_bits, last_dom_bits, stream=None):
    """Device buffers as torch tensors or addresses. Returns (status, changed mask word)."""
    sz, psz = _i32(dom_size)
    ch, pch = _u32_out(1)
    st = load().ct_propagate_noalloc(len(sz), psz, int(t), _dev_ptr(supports), _dev_ptr(curr_table),
                                     _dev_ptr(dom_bits), _dev_ptr(last_dom_bits), pch, _stream_ptr(stream))
    return st, int(ch[0])


# --------------------------------------------------------------------------
# model
# --------------------------------------------------------------------------

def ct_model_create(dom_lo, dom_size, opt=None, stream=None):
    L = load()
    lo, plo = _i32(dom_lo)
    sz, psz = _i32(dom_size)
    h = _P()
    st = L.ct_model_create(len(lo), plo, psz, ctypes.byref(opt) if opt is not None else None,
                           _stream_ptr(stream), ctypes.byref(h))
    return st, h


def ct_model_add_table(m, scope, tuples, negative=False):
    sc, psc = _i32(scope)
    tup = np.ascontiguousarray(np.asarray(tuples, dtype=np.int32).reshape(-1, len(sc)))
    ptup = tup.ctypes.data_as(_I32P) if tup.shape[0] else None
    fn = load().ct_model_add_negative_table if negative else load().ct_model_add_table
    return fn(m, psc, len(sc), ptup, int(tup.shape[0]))


def ct_model_propagate(m):
    return load().ct_model_propagate(m)


def ct_model_get_domains(m, nwords):
    w, pw = _u32_out(nwords)
    st = load().ct_model_get_domains(m, pw)
    return st, w[:nwords]


def ct_model_set_domains(m, words):
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    return load().ct_model_set_domains(m, w.ctypes.data_as(_U32P))


def ct_model_save(m):
    lv = ctypes.c_int(-1)
    st = load().ct_model_save(m, ctypes.byref(lv))
    return st, lv.value


def ct_model_restore(m, level):
    return load().ct_model_restore(m, int(level))


def ct_search_dfs(m, nvars, node_limit=0, count_all=True):
    s = ct_search_stats()
    sol = np.zeros(nvars, dtype=np.int32)
    st = load().ct_search_dfs(m, int(node_limit), 1 if count_all else 0, ctypes.byref(s),
                              sol.ctypes.data_as(_I32P))
    d = _as_dict(s)
    d["first_solution"] = sol.tolist() if d["solutions"] > 0 else None
    return st, d


def ct_search_batch_device(m, nvars, slots, split_depth, node_limit=0):
    """The batched search with the slots' search run on the device (count all
    solutions, first-fail): returns (status, stats dict with first_solution, batch info dict)."""
    s = ct_search_stats()
    info = ct_batch_info()
    sol = np.zeros(nvars, dtype=np.int32)
    st = load().ct_search_batch_device(m, int(slots), int(split_depth), int(node_limit), ctypes.byref(s),
                                       sol.ctypes.data_as(_I32P), ctypes.byref(info))
    d = _as_dict(s)
    d["first_solution"] = sol.tolist() if d["solutions"] > 0 else None
    return st, d, _as_dict(info)


def ct_search_batch(m, nvars, slots, split_depth, node_limit=0, count_all=True, split_assignments=False):
    """Batched search: returns (status, stats dict with first_solution, batch info dict).
    count_all: True/1 all solutions, False/0 the depth-first first solution,
    2 (or "any") the first solution any slot finds. split_assignments: the
    split depth counts assignments on a node's path (ct_search_batch_assign)."""
    s = ct_search_stats()
    info = ct_batch_info()
    sol = np.zeros(nvars, dtype=np.int32)
    mode = 2 if count_all == "any" else int(count_all)
    fn = load().ct_search_batch_assign if split_assignments else load().ct_search_batch
    st = fn(m, int(slots), int(split_depth), int(node_limit), mode,
            ctypes.byref(s), sol.ctypes.data_as(_I32P), ctypes.byref(info))
    d = _as_dict(s)
    d["first_solution"] = sol.tolist() if d["solutions"] > 0 else None
    return st, d, _as_dict(info)


# --------------------------------------------------------------------------
# learned branching order
# --------------------------------------------------------------------------
MLP_FEATURES, MLP_HIDDEN, MLP_WEIGHTS, MLP_MAX_BATCH = 8, 64, 4801, 128


def _f32(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} floats, got {a.size}")
    return a


def ct_mlp_create(weights, stream=None):
    w = _f32(weights, MLP_WEIGHTS)
    h = _P()
    st = load().ct_mlp_create(w.ctypes.data_as(_F32P), _stream_ptr(stream), ctypes.byref(h))
    return st, h.value


def ct_mlp_set_weights(m, weights):
    w = _f32(weights, MLP_WEIGHTS)
    return load().ct_mlp_set_weights(m, w.ctypes.data_as(_F32P))


def ct_mlp_get_weights(m):
    w = np.zeros(MLP_WEIGHTS, dtype=np.float32)
    st = load().ct_mlp_get_weights(m, w.ctypes.data_as(_F32P))
    return st, w


def ct_mlp_forward(m, x_dev, n, scores_dev):
    """x_dev / scores_dev: device pointers (int) or tensors with data_ptr()."""
    xp = x_dev.data_ptr() if hasattr(x_dev, "data_ptr") else int(x_dev)
    sp = scores_dev.data_ptr() if hasattr(scores_dev, "data_ptr") else int(scores_dev)
    return load().ct_mlp_forward(m, xp, int(n), sp)


def ct_mlp_grad(m, X, y):
    X = _f32(X)
    y = _f32(y)
    n = y.size
    loss = ctypes.c_float()
    g = np.zeros(MLP_WEIGHTS, dtype=np.float32)
    st = load().ct_mlp_grad(m, X.ctypes.data_as(_F32P), y.ctypes.data_as(_F32P), int(n), ctypes.byref(loss),
                            g.ctypes.data_as(_F32P))
    return st, float(loss.value), g


def ct_mlp_train(m, X, y, orders, batch, lr):
    """orders: int32 [epochs, n] permutations. Returns (status, epoch losses)."""
    X = _f32(X)
    y = _f32(y)
    orders = np.ascontiguousarray(np.asarray(orders, dtype=np.int32))
    epochs = orders.shape[0]
    losses = np.zeros(epochs, dtype=np.float32)
    st = load().ct_mlp_train(m, X.ctypes.data_as(_F32P), y.ctypes.data_as(_F32P), int(y.size),
                             orders.ctypes.data_as(_I32P), int(epochs), int(batch), float(lr),
                             losses.ctypes.data_as(_F32P))
    return st, losses


def ct_mlp_destroy(m):
    return load().ct_mlp_destroy(m)


def ct_model_features(m, nvars):
    F = np.zeros((nvars, MLP_FEATURES), dtype=np.float32)
    st = load().ct_model_features(m, F.ctypes.data_as(_F32P))
    return st, F


def ct_model_set_policy(m, mlp):
    return load().ct_model_set_policy(m, mlp)


class Trace:
    """Host buffers of ct_model_set_trace (keep the object alive while searching)."""

    def __init__(self, capacity):
        self.buf = np.zeros(int(capacity), dtype=np.int32)
        self.count = ctypes.c_int64(0)

    def decisions(self):
        return self.buf[: int(self.count.value)].tolist()


def ct_model_set_trace(m, trace):
    if trace is None:
        return load().ct_model_set_trace(m, None, 0, None)
    return load().ct_model_set_trace(m, trace.buf.ctypes.data_as(_I32P), int(trace.buf.size),
                                     ctypes.byref(trace.count))


def ct_model_lookahead(m, nvars, slots):
    lab = np.zeros(nvars, dtype=np.float32)
    st = load().ct_model_lookahead(m, int(slots), lab.ctypes.data_as(_F32P))
    return st, lab


def ct_search_collect(m, node_limit, slots, max_samples):
    X = np.zeros((int(max_samples), MLP_FEATURES), dtype=np.float32)
    y = np.zeros(int(max_samples), dtype=np.float32)
    n = ctypes.c_int64(0)
    st = load().ct_search_collect(m, int(node_limit), int(slots), int(max_samples), X.ctypes.data_as(_F32P),
                                  y.ctypes.data_as(_F32P), ctypes.byref(n))
    return st, X[: n.value], y[: n.value]


def ct_model_get_stats(m):
    s = ct_model_stats()
    st = load().ct_model_get_stats(m, ctypes.byref(s))
    return st, _as_dict(s)


def ct_model_reset_stats(m):
    return load().ct_model_reset_stats(m)


def ct_model_destroy(m):
    return load().ct_model_destroy(m)
