"""Failure detection without a GPU fault: a bounded wait that nothing will
satisfy runs out, the kernel sets GLOP_ETIMEOUT in its status word and
returns, and the context stays usable for the next scan."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def test_grid_barrier_timeout_reports_and_recovers():
    text = (b"abcdefgh" * 512) + b"xyz"
    pats = [b"abcd", b"cdefgh"]
    a = glop.Automaton(pats)
    d = torch.from_numpy(np.frombuffer(text, np.uint8).copy()).cuda()
    m = torch.zeros((4096, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    os.environ["GLOP_TEST_BARRIER_EXTRA"] = "1"      # wait for a block that does not exist
    os.environ["GLOP_TEST_SPIN_BUDGET"] = "20000000"  # ~10 ms per wait
    try:
        a.scan_into(d, m, cnt)
        assert a.status(d.device) == glop.ETIMEOUT
    finally:
        del os.environ["GLOP_TEST_BARRIER_EXTRA"]
        del os.environ["GLOP_TEST_SPIN_BUDGET"]
    # the context is still usable and the next scan is exact
    got, n = a.scan(d)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), oracle.naive(text, pats))


def test_ring_wait_timeout_reports_and_recovers():
    """A chunk the producer never stages (a test hook withholds its bulk copy): every consumer's bounded wait
    on that ring slot runs out, the producer's wait for the slot to be released runs out too, the kernel
    waits for its other copies in flight, reports GLOP_ETIMEOUT and returns; the next scan is exact."""
    import workloads as W
    w = W.config2(300 * 1024 + 77)  # ten 31 KiB chunks on a tiny grid of ten blocks
    a = glop.Automaton(w.patterns)
    d = torch.from_numpy(w.text.copy()).cuda()
    exp = oracle.ac(w.text, w.patterns.csr())
    m = torch.zeros((len(exp) + 16, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for chunk in ("0", "7"):
        os.environ["GLOP_TEST_WITHHOLD_CHUNK"] = chunk
        os.environ["GLOP_TEST_SPIN_BUDGET"] = "20000000"  # ~10 ms per wait
        try:
            a.scan_into(d, m, cnt)
            assert a.status(d.device) == glop.ETIMEOUT
        finally:
            del os.environ["GLOP_TEST_WITHHOLD_CHUNK"]
            del os.environ["GLOP_TEST_SPIN_BUDGET"]
        got, n = a.scan(d)
        assert n == len(exp)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), exp)
