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
