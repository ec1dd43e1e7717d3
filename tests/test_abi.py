"""The C-ABI library builds for sm_103a, loads, and exports every symbol
include/glop.h declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1704_02278_gb300 as glop
from paper_1704_02278_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "glop.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(glop_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return _build.build_lib()


def test_header_declarations_match_binding():
    assert declared_symbols() == sorted(glop.SYMBOLS)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (glop_[a-z_]+)\b", out))
    assert set(declared_symbols()) <= exported


def test_built_for_sm_103a_only(libpath):
    # every CUDA object of the library was compiled with exactly one target: sm_103a
    for src in _build.CUDA_SOURCES:
        log = os.path.join(_build.BUILD, src + ".o.log")
        if not os.path.exists(log):
            pytest.skip("objects built elsewhere")
        cmd = open(log).readline()
        assert re.findall(r"-gencode\s+(\S+)", cmd) == ["arch=compute_103a,code=sm_103a"], (src, cmd)
    link = open(os.path.join(_build.BUILD, "link.log")).readline()
    assert re.findall(r"-gencode\s+(\S+)", link) == ["arch=compute_103a,code=sm_103a"], link


def test_status_strings(libpath):
    lib = glop.lib()
    assert lib.glop_status_str(0) == b"ok"
    assert lib.glop_status_str(3) == b"match capacity exceeded"
    assert lib.glop_status_str(99) == b"unknown status"


def test_no_device_means_error_not_fallback(libpath):
    """Without a usable GPU the library reports GLOP_ECUDA (or refuses) instead of computing on the CPU."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    with pytest.raises(glop.GlopError) as e:
        glop.Automaton([b"abcd"])
    assert e.value.code in (glop.ECUDA, glop.ENOMEM)


def test_kernels_fit_register_budget(libpath):
    rep = _build.ptxas_report()
    regs = [int(x) for x in re.findall(r"Used (\d+) registers", rep)]
    assert regs and max(regs) <= 64  # 1024-thread blocks, one per SM
    assert "spill stores" in rep and not re.search(r"[1-9]\d* bytes spill stores", rep)


def test_new_entry_points_reject_bad_arguments_before_any_device_work(libpath):
    lib = glop.lib()
    u64 = ctypes.c_uint64()
    assert lib.glop_count_workspace_size(None, 0, ctypes.byref(u64)) == glop.EINVAL
    assert lib.glop_scan_count(None, None, 0, None, None, None, 0, None) == glop.EINVAL
    # batch split: NULL count / runs, and a segment count whose runs array would not be indexable
    assert lib.glop_batch_split(None, None, 0, 1, None, None, None) == glop.EINVAL
    dummy = ctypes.c_uint64(0)
    p = ctypes.addressof(dummy)
    assert lib.glop_batch_split(None, p, 0, 0xFFFFFFFF, None, p, None) == glop.EINVAL
    assert lib.glop_batch_split(None, p, 5, 1, None, p, None) == glop.EINVAL  # capacity without arrays
    # count and status words: NULL workspace or words
    assert lib.glop_scan_words(None, p, None) == glop.EINVAL
    assert lib.glop_scan_words(p, None, None) == glop.EINVAL
    # streaming ingestion: NULL handle or output, depth out of range, NULL object
    h = ctypes.c_void_p()
    assert lib.glop_ingest_create(None, 1 << 20, 0, 2, ctypes.byref(h)) == glop.EINVAL and not h.value
    assert lib.glop_ingest_create(p, 1 << 20, 0, 2, None) == glop.EINVAL
    assert lib.glop_ingest_create(p, 1 << 20, 0, 0, ctypes.byref(h)) == glop.EINVAL
    assert lib.glop_ingest_create(p, 1 << 20, 0, 9, ctypes.byref(h)) == glop.EINVAL
    assert lib.glop_ingest_create(p, 0, 0, 2, ctypes.byref(h)) == glop.EINVAL
    res = glop.IngestResult()
    n = ctypes.c_uint32()
    assert lib.glop_ingest_feed(None, None, 0, ctypes.byref(res)) == glop.EINVAL
    assert lib.glop_ingest_flush(None, None, 0, ctypes.byref(n)) == glop.EINVAL
    assert lib.glop_ingest_reset(None) == glop.EINVAL
    assert lib.glop_ingest_info(None, None, None) == glop.EINVAL
    assert lib.glop_ingest_destroy(None) == glop.EINVAL
    # several automata in one batch: no handles, too many groups
    assert lib.glop_scan_batch_multi(None, 1, p, None, 0, p, 0, None, 0, p, p, 0, None) == glop.EINVAL
    assert lib.glop_scan_batch_multi(p, 9, p, None, 0, p, 0, None, 0, p, p, 0, None) == glop.EINVAL
    assert lib.glop_batch_multi_kind(None, None) == glop.EINVAL
    # the native server: NULL sets, options or object; bad options
    srv = ctypes.c_void_p()
    opts = glop.ServerOpts(1 << 20, 2, 16, 1 << 20, 0, 0, 0, 0)
    assert lib.glop_server_create(None, 1, ctypes.byref(opts), ctypes.byref(srv)) == glop.EINVAL and not srv.value
    assert lib.glop_server_create(p, 0, ctypes.byref(opts), ctypes.byref(srv)) == glop.EINVAL
    bad = glop.ServerOpts(1 << 20, 0, 16, 1 << 20, 0, 0, 0, 0)  # no stream slots
    assert lib.glop_server_create(p, 1, ctypes.byref(bad), ctypes.byref(srv)) == glop.EINVAL
    assert lib.glop_server_submit(None, 0, 0, None, 0) == glop.EINVAL
    assert lib.glop_server_poll(None, None, 0, ctypes.byref(n), 0) == glop.EINVAL
    assert lib.glop_server_release(None, 0) == glop.EINVAL
    assert lib.glop_server_stats_get(None, None) == glop.EINVAL
    assert lib.glop_server_destroy(None) == glop.OK
