"""The C-ABI library builds, loads and exports every symbol include/ct.h declares.

No compute call is made here (no GPU needed): only entry points that touch no
device (status strings, version, last error) are called.
"""
import os
import re
import shutil

import numpy as np
import pytest

from paper_2507_18413_gb300 import build as B
from paper_2507_18413_gb300 import ct as C

HEADER = os.path.join(B.ROOT, "include", "ct.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const\s+char\s*\*)\s*(ct_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")):
        if not os.path.exists(B.LIB):
            pytest.skip("no nvcc and no prebuilt libct.so")
    else:
        B.build()
    return C.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["ct_create", "ct_propagate", "ct_save", "ct_restore", "ct_get_currtable", "ct_destroy",
              "ct_model_create", "ct_model_add_table", "ct_model_propagate", "ct_search_dfs",
              "ct_model_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert sorted(C.exported_names()) == _declared()


def test_host_only_entry_points(lib):
    assert C.status_string(C.CT_OK) == "CT_OK"
    assert C.status_string(C.CT_INFEASIBLE) == "CT_INFEASIBLE"
    assert C.status_string(C.CT_ERR_LEVEL) == "CT_ERR_LEVEL"
    assert lib.ct_version() >= 10000
    assert isinstance(C.last_error(), str)


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.ct_create(3, None, None, None, 0, None, None, None) == C.CT_ERR_ARG
    assert lib.ct_propagate(None, None, None) == C.CT_ERR_ARG
    assert lib.ct_restore(None, 0) == C.CT_ERR_ARG
    assert lib.ct_destroy(None) == C.CT_OK
    assert lib.ct_model_destroy(None) == C.CT_OK
    assert lib.ct_search_batch(None, 4, 1, 0, 1, None, None, None) == C.CT_ERR_ARG


def test_domain_word_marshalling_round_trip():
    rng = np.random.default_rng(0)
    sizes = [1, 7, 32, 33, 64, 100]
    masks = [rng.random(d) < 0.5 for d in sizes]
    words = C.masks_to_words(masks)
    off, nw = C.dom_layout(sizes)
    assert words.shape[0] == off[-1] == sum(nw)
    back = C.words_to_masks(words, sizes)
    for a, b in zip(masks, back):
        assert np.array_equal(a, b)
    # value a of variable i is bit a % 32 of word off[i] + a // 32
    for i, m in enumerate(masks):
        for a in range(sizes[i]):
            assert bool((int(words[off[i] + a // 32]) >> (a % 32)) & 1) == bool(m[a])


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror has the size and field offsets the C compiler gives the header."""
    import ctypes
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [C.ct_options, C.ct_table_info, C.ct_call_stats, C.ct_profile, C.ct_search_stats, C.ct_batch_info,
               C.ct_model_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ct.h"', "int main(void){"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(B.ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for st in structs:
        n = st.__name__
        assert int(out[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(out[f"{n}.{f}"]) == getattr(st, f).offset, f"{n}.{f}"


def test_host_side_test_hooks_without_a_device(lib):
    """The test hooks' settings and argument checks touch no device: they run
    (and reject bad arguments) on a host without a GPU."""
    assert C.ct_debug_guard_buffers(1) == C.CT_OK
    assert C.ct_debug_guard_buffers(0) == C.CT_OK
    assert C.ct_debug_fail_alloc(3) == C.CT_OK
    assert C.ct_debug_fail_alloc(-1) == C.CT_OK
    st, n = C.ct_debug_device_bytes()
    assert st == C.CT_OK and n >= 0
    assert lib.ct_debug_device_bytes(None) == C.CT_ERR_ARG
    assert lib.ct_debug_check_guards(None, 0, None) == C.CT_ERR_ARG
    # the read ceiling checks its buffer and size before launching
    assert C.ct_read_ceiling(0, 16) == C.CT_ERR_ARG
    assert C.ct_read_ceiling(4096 + 4, 16) == C.CT_ERR_ARG
    assert C.ct_read_ceiling(4096, 0) == C.CT_ERR_ARG
    assert C.ct_read_ceiling(4096, 24) == C.CT_ERR_ARG
    assert "16-byte" in C.last_error()


def test_options_fields_reach_the_struct():
    o = C.make_options(grid_blocks=7, no_residues=1, profile=1, host_fixpoint=1, copy_state=1, autotune=1, shard=1,
                       no_split=1, no_early_filter=1)
    assert (o.reserved0, o.grid_blocks, o.no_residues, o.profile, o.host_fixpoint, o.copy_state, o.autotune,
            o.shard, o.no_split, o.no_early_filter) == (0, 7, 1, 1, 1, 1, 1, 1, 1, 1)
    d = C.make_options()
    assert all(getattr(d, f) == 0 for f, _ in d._fields_)
