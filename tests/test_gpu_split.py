"""glop_batch_split: a batch scan's matches as (offset, pattern_id) pairs plus each segment's run."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def _expect(m, n_seg):
    seg = m[:, 0].astype(np.int64)
    return m[:, 1:], np.searchsorted(seg, np.arange(n_seg + 1), side="left")


def _split(m_dev, count, n_seg, cap=None):
    cap = m_dev.shape[0] if cap is None else cap
    pairs = torch.full((max(cap, 1), 2), -1, dtype=torch.int32, device="cuda")
    first = torch.full((n_seg + 1,), -1, dtype=torch.int64, device="cuda")
    glop.batch_split(m_dev[:max(cap, 1)], count, n_seg, pairs, first)
    torch.cuda.synchronize()
    return pairs.cpu().numpy().view(np.uint32), first.cpu().numpy()


@pytest.mark.parametrize("n_seg", [1, 7, 300])
def test_split_of_a_batch_scan(n_seg):
    w = W.config1()
    rng = np.random.default_rng(n_seg)
    cuts = np.sort(rng.choice(np.arange(1, w.text.size), n_seg - 1, replace=False)) if n_seg > 1 else []
    seg = np.concatenate([[0], cuts, [w.text.size]]).astype(np.int64)
    a = glop.Automaton(w.patterns)
    m, n = a.scan_batch(torch.from_numpy(w.text).cuda(), torch.from_numpy(seg).cuda())
    count = torch.tensor([n], dtype=torch.int64, device="cuda")
    pairs, first = _split(m.contiguous(), count, n_seg)
    exp_pairs, exp_first = _expect(m.cpu().numpy().view(np.uint32), n_seg)
    assert np.array_equal(pairs[:n], exp_pairs)
    assert np.array_equal(first, exp_first)


def test_split_empty_segments_and_no_matches():
    # segments 0, 3, 4 have matches; 1, 2, 5, 6 are empty
    m = np.array([[0, 5, 1], [0, 9, 2], [3, 1, 0], [4, 2, 2], [4, 2, 3]], np.uint32)
    dev = torch.from_numpy(m.view(np.int32)).cuda()
    pairs, first = _split(dev, torch.tensor([5], dtype=torch.int64, device="cuda"), 7)
    assert np.array_equal(pairs[:5], m[:, 1:])
    assert first.tolist() == [0, 2, 2, 2, 3, 5, 5, 5]
    pairs, first = _split(dev, torch.tensor([0], dtype=torch.int64, device="cuda"), 7)
    assert first.tolist() == [0] * 8


def test_split_reads_only_capacity_entries_on_overflow():
    m = np.array([[0, 5, 1], [1, 9, 2], [2, 1, 0], [2, 2, 2]], np.uint32)
    dev = torch.from_numpy(m.view(np.int32)).cuda()
    pairs, first = _split(dev, torch.tensor([10], dtype=torch.int64, device="cuda"), 3, cap=3)
    assert np.array_equal(pairs[:3], m[:3, 1:])
    assert first.tolist() == [0, 1, 2, 3]
