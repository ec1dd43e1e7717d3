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
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert arches == {"103a"}, arches


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
