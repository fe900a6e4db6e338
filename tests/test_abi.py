"""CPU-only checks of the C ABI: the library builds for sm_103a, loads without
a GPU, exports every entry point include/pcpm.h declares, and rejects invalid
arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

import paper_1709_07122_gb300 as pcpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if fname.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fname)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pcpm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    pcpm.build()
    return pcpm.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pcpm_build", "pcpm_pagerank", "pcpm_free", "pcpm_png_export", "pcpm_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_is_host_only(L):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, 99):
        assert isinstance(L.pcpm_strerror(code), bytes)
    assert b"invalid" in L.pcpm_strerror(-1)


def test_invalid_arguments_rejected_before_any_launch(L):
    h = ctypes.c_void_p()
    assert L.pcpm_build(None, None, 10, 0, 4, None, ctypes.byref(h)) == -1
    assert L.pcpm_build(ctypes.c_void_p(16), None, 0, 0, 4, None, ctypes.byref(h)) == -1  # n = 0
    assert L.pcpm_build(ctypes.c_void_p(16), None, 10, 0, 0, None, ctypes.byref(h)) == -1  # q = 0
    assert L.pcpm_build(ctypes.c_void_p(16), None, 10, 0, 40000, None, ctypes.byref(h)) == -1  # q too large
    assert L.pcpm_build(ctypes.c_void_p(16), None, 1 << 31, 0, 4, None, ctypes.byref(h)) == -1  # n >= 2^31
    assert L.pcpm_build(ctypes.c_void_p(16), None, 10_000_000, 0, 1, None, ctypes.byref(h)) == -1  # k too large
    assert L.pcpm_build(ctypes.c_void_p(16), None, 10, 0, 4, None, None) == -1
    assert L.pcpm_png_get_info(None, None) == -1
    assert L.pcpm_reset(None, None, None) == -1
    assert L.pcpm_iterate(None, 0.85, 1, 0.0, 0, None, None, None) == -1
    assert L.pcpm_pagerank(None, 0.85, 1, 0.0, 0, None, None, None, None, None) == -1
    assert L.pcpm_residual_history(None, None, 0) == -1
    assert L.pcpm_scatter_only(None, None) == -1
    assert L.pcpm_export_state(None, None, None, None, None) == -1
    L.pcpm_free(None)  # null-safe
    out = (ctypes.c_float * 4)()
    # host entry: bad damping factor and null pointers fail on the host
    rp = (ctypes.c_uint32 * 5)(0, 1, 2, 3, 4)
    col = (ctypes.c_uint32 * 4)(1, 2, 3, 0)
    assert L.pcpm_pagerank_host(rp, col, 4, 4, 2, 1.0, 5, 0.0, 0, out, None, None) == -1
    assert L.pcpm_pagerank_host(None, col, 4, 4, 2, 0.85, 5, 0.0, 0, out, None, None) == -1
    assert L.pcpm_pagerank_host(rp, col, 4, 4, 2, 0.85, -1, 0.0, 0, out, None, None) == -1
    assert L.pcpm_pagerank_host(rp, col, 4, 4, 2, 0.85, 5, 0.0, 0x80, out, None, None) == -1


def test_ppr_autotune_and_pool_entries_check_arguments_on_the_host(L):
    h = ctypes.c_void_p()
    ptr = (ctypes.c_uint32 * 65)(*range(65))
    idx = (ctypes.c_uint32 * 64)(*range(64))
    assert L.pcpm_ppr_create(None, ptr, idx, None, ctypes.byref(h)) == -1
    assert L.pcpm_ppr_run(None, 0.85, 1, None) == -1
    assert L.pcpm_ppr_residuals(None, None, 0) == -1
    assert L.pcpm_ppr_ranks(None, None, None) == -1
    assert L.pcpm_ppr_info(None, None, None) == -1
    L.pcpm_ppr_free(None)  # null-safe
    sizes = (ctypes.c_uint32 * 2)(1024, 4096)
    best = ctypes.c_uint32(0)
    dev = ctypes.c_void_p(16)
    assert L.pcpm_autotune(dev, dev, 10, 0, sizes, 0, 0.85, 1, 1, 0, None, ctypes.byref(best), None) == -1  # no candidates
    assert L.pcpm_autotune(dev, dev, 10, 0, sizes, 2, 0.85, 1, 0, 0, None, ctypes.byref(best), None) == -1  # iters = 0
    assert L.pcpm_autotune(dev, dev, 10, 0, sizes, 2, 1.5, 1, 1, 0, None, ctypes.byref(best), None) == -1  # bad d
    assert L.pcpm_autotune(dev, dev, 10, 0, sizes, 2, 0.85, 1, 1, 0x80, None, ctypes.byref(best), None) == -1  # flags
    assert L.pcpm_autotune(dev, dev, 10, 0, None, 2, 0.85, 1, 1, 0, None, ctypes.byref(best), None) == -1
    assert L.pcpm_release_cached_memory() == 0  # no pool was created in this process


def test_shard_entries_check_arguments_on_the_host(L):
    h = ctypes.c_void_p()
    dev = ctypes.c_void_p(16)
    cuts = (ctypes.c_uint32 * 3)()
    ids = (ctypes.c_uint64 * 4)(5, 0, 7, 1)
    assert L.pcpm_build_shard(dev, dev, 40, 0, 10, 2, 2, None, None, ctypes.byref(h)) == -1  # empty range
    assert L.pcpm_build_shard(dev, dev, 40, 0, 10, 0, 5, None, None, ctypes.byref(h)) == -1  # past k = 4
    assert L.pcpm_build_shard(dev, dev, 40, 0, 10, 0, 2, None, None, None) == -1
    assert L.pcpm_shard_init(None, None, dev, dev, None) == -1
    assert L.pcpm_shard_step(None, 0.85, 0, dev, dev, dev, None) == -1
    assert L.pcpm_sync_status(None) == -1
    assert L.pcpm_dest_partition_counts(dev, 0, 0, 10, ids, None) == -1  # n = 0
    assert L.pcpm_dest_partition_counts(dev, 0, 40, 10, None, None) == -1
    assert L.pcpm_shard_split(None, 40, 10, 2, cuts) == -1
    assert L.pcpm_shard_split(ids, 40, 10, 5, cuts) == -1  # more ranks than partitions
    assert L.pcpm_shard_split(ids, 40, 10, 2, cuts) == 0  # host only: works without a GPU
    assert list(cuts) == [0, 2, 4]


def test_binding_fails_loudly_without_library(tmp_path):
    saved = pcpm._lib
    try:
        pcpm._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            pcpm.lib(str(tmp_path / "missing.so"))
    finally:
        pcpm._lib = saved
