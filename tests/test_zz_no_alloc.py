"""glop_scan_noalloc: the scan for callers that cannot allocate device memory
at scan time (their memory belongs to another allocator, or their loop must
not pay for an allocation's synchronisation).  It keeps its scratch in a
fixed device array inside the library, so it must give exactly what the
workspace-taking glop_scan gives, and what the CPU oracle gives -- also on a
second call, which finds the first call's leftovers in that array -- and its
callers read the outcome of their last call with glop_scan_status(NULL, ...)."""
import ctypes
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402

MAX_LEN = 16 << 20


def _noalloc(a, text, cap, stream, expect=glop.OK):
    lib = glop.lib()
    out = torch.full((max(cap, 1), 2), -1, dtype=torch.int32, device=text.device)
    cnt = torch.full((1,), -1, dtype=torch.int64, device=text.device)
    rc = lib.glop_scan_noalloc(a.handle, text.data_ptr(), text.numel(), out.data_ptr(), cap, cnt.data_ptr(),
                               stream.cuda_stream)
    assert rc == glop.OK, glop.STATUS.get(rc)
    total = ctypes.c_uint64()
    st = lib.glop_scan_status(None, stream.cuda_stream, ctypes.byref(total))
    assert st == expect, glop.STATUS.get(st)
    stream.synchronize()
    assert int(cnt.item()) == total.value
    return out, int(cnt.item())


def test_noalloc_equals_workspace_scan_on_two_calls():
    stream = torch.cuda.current_stream()
    w = W.config2(8 * W.MiB + 777)
    a = glop.Automaton(w.patterns)
    text = torch.from_numpy(w.text.copy()).cuda()
    ref, n = a.scan(text, stream=stream)
    ref = ref.cpu().numpy()
    assert n > 0
    assert np.array_equal(ref.view(np.uint32), oracle.ac_mt(w.text, w.patterns.csr()))
    # a smaller text in between leaves a different pattern of leftovers
    small = text[: 3 * 4096 + 5]
    ref_small, n_small = a.scan(small, stream=stream)
    assert np.array_equal(ref_small.cpu().numpy().view(np.uint32),
                          oracle.ac(w.text[: 3 * 4096 + 5], w.patterns.csr()))
    for call in range(2):
        got, cnt = _noalloc(a, text, n + 64, stream)
        assert cnt == n
        assert np.array_equal(got[:n].cpu().numpy(), ref)
        got_s, cnt_s = _noalloc(a, small, n_small + 8, stream)
        assert cnt_s == n_small
        assert np.array_equal(got_s[:n_small].cpu().numpy(), ref_small.cpu().numpy())
    a.close()


def test_noalloc_at_its_maximum_length():
    stream = torch.cuda.current_stream()
    w = W.config2(MAX_LEN)
    assert w.nbytes == MAX_LEN
    a = glop.Automaton(w.patterns)
    text = torch.from_numpy(w.text.copy()).cuda()
    ref, n = a.scan(text, stream=stream)
    exp = oracle.ac_mt(w.text, w.patterns.csr())
    assert n == len(exp)
    for call in range(2):
        got, cnt = _noalloc(a, text, n, stream)
        assert cnt == n
        got = got[:n].cpu().numpy()
        assert np.array_equal(got, ref.cpu().numpy())
        assert np.array_equal(got.view(np.uint32), exp)
    a.close()


def test_noalloc_status_overflow_and_timeout_read_back():
    stream = torch.cuda.current_stream()
    w = W.config2(2 * W.MiB + 13)
    a = glop.Automaton(w.patterns)
    text = torch.from_numpy(w.text.copy()).cuda()
    exp = oracle.ac_mt(w.text, w.patterns.csr())
    n = len(exp)
    # overflow: the true total comes back with the status, the first cap matches are the sorted prefix
    got, cnt = _noalloc(a, text, n // 3, stream, expect=glop.EOVERFLOW)
    assert cnt == n
    assert np.array_equal(got[: n // 3].cpu().numpy().view(np.uint32), exp[: n // 3])
    # a bounded wait that runs out (a grid barrier waits for a block that does not exist): the no-alloc
    # caller sees GLOP_ETIMEOUT through the status of the fixed array
    os.environ["GLOP_TEST_BARRIER_EXTRA"] = "1"
    os.environ["GLOP_TEST_SPIN_BUDGET"] = "20000000"  # ~10 ms per wait
    try:
        _noalloc(a, text[:65536], 4096, stream, expect=glop.ETIMEOUT)
    finally:
        del os.environ["GLOP_TEST_BARRIER_EXTRA"]
        del os.environ["GLOP_TEST_SPIN_BUDGET"]
    # the next call starts from a clean header and is exact again
    got, cnt = _noalloc(a, text, n, stream)
    assert cnt == n and np.array_equal(got[:n].cpu().numpy().view(np.uint32), exp)
    a.close()


def test_noalloc_rejects_texts_beyond_its_maximum():
    a = glop.Automaton([b"abcd"])
    text = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    out = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    # the length check comes before any use of the (short) buffer
    rc = glop.lib().glop_scan_noalloc(a.handle, text.data_ptr(), MAX_LEN + 1, out.data_ptr(), 4, cnt.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == glop.EINVAL
    a.close()
