"""CUDA-graph plans: a captured scan replayed with one graph launch gives the
same result as the direct call, on every replay."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def test_batch_plan_replays():
    p = W.config4_patterns()
    sizes = W.config4_sizes(120)
    seg = np.zeros(121, np.uint64)
    seg[1:] = np.cumsum(sizes)
    t = W.syslog_files(W.seed(4, 0), W.seed(4, 2), seg, 0.02, p)
    exp = oracle.batch(t, seg, p.csr())
    a = glop.Automaton(p)
    d = torch.from_numpy(t).cuda()
    s = torch.from_numpy(seg.view(np.int64).copy()).cuda()
    m = torch.empty((len(exp) + 5, 3), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan = glop.Plan(a, d, m, cnt, seg_offsets=s)
    for rep in range(3):
        m.fill_(-1)
        plan.launch()
        assert plan.status() == glop.OK
        assert int(cnt.item()) == len(exp)
        assert np.array_equal(m[: len(exp)].cpu().numpy().view(np.uint32), exp)
    plan.close()
    a.close()


def test_single_plan_replays():
    w = W.config2(3 * W.MiB + 11)
    exp = oracle.ac_mt(w.text, w.patterns.csr())
    a = glop.Automaton(w.patterns)
    d = torch.from_numpy(w.text).cuda()
    m = torch.empty((len(exp), 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan = glop.Plan(a, d, m, cnt)
    for rep in range(2):
        plan.launch()
        assert plan.status() == glop.OK
        assert np.array_equal(m.cpu().numpy().view(np.uint32), exp)
    plan.close()
    a.close()
