"""ctypes wrapper of the serial CPU Compact-Table baseline (test and benchmark infrastructure)."""
import ctypes

import numpy as np

from . import build as _build

_lib = None
_I32P = ctypes.POINTER(ctypes.c_int32)
_U32P = ctypes.POINTER(ctypes.c_uint32)


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        lib.sct_create.restype = ctypes.c_void_p
        lib.sct_create.argtypes = [ctypes.c_int, _I32P, _I32P, _I32P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
        lib.sct_propagate.restype = ctypes.c_int
        lib.sct_propagate.argtypes = [ctypes.c_void_p, _U32P]
        lib.sct_save.restype = ctypes.c_int
        lib.sct_save.argtypes = [ctypes.c_void_p]
        lib.sct_restore.restype = ctypes.c_int
        lib.sct_restore.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.sct_currtable32.restype = None
        lib.sct_currtable32.argtypes = [ctypes.c_void_p, _U32P]
        lib.sct_destroy.restype = None
        lib.sct_destroy.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


class SerialCT:
    """One table; domains are packed uint32 words (value lo+a at bit a%32 of word a/32)."""

    def __init__(self, dom_lo, dom_size, tuples):
        L = load()
        lo = np.ascontiguousarray(dom_lo, dtype=np.int32)
        sz = np.ascontiguousarray(dom_size, dtype=np.int32)
        tup = np.ascontiguousarray(tuples, dtype=np.int32).reshape(-1, len(lo))
        st = ctypes.c_int(0)
        self.h = L.sct_create(len(lo), lo.ctypes.data_as(_I32P), sz.ctypes.data_as(_I32P),
                              tup.ctypes.data_as(_I32P) if tup.shape[0] else None, tup.shape[0], ctypes.byref(st))
        if not self.h:
            raise MemoryError("sct_create failed")
        self.create_status = st.value
        self.t = None
        self.nwords32 = None

    def propagate(self, words):
        """words: uint32 array, filtered in place. Returns 0 (ok), 1 (fail) or a negative error."""
        assert words.dtype == np.uint32 and words.flags["C_CONTIGUOUS"]
        return load().sct_propagate(self.h, words.ctypes.data_as(_U32P))

    def save(self):
        return load().sct_save(self.h)

    def restore(self, level):
        return load().sct_restore(self.h, level)

    def currtable(self, nwords):
        out = np.zeros(max(nwords, 1), dtype=np.uint32)
        load().sct_currtable32(self.h, out.ctypes.data_as(_U32P))
        return out[:nwords]

    def close(self):
        if self.h:
            load().sct_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
