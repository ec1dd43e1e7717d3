"""Count-only mode (glop_scan_count): per-pattern occurrence counts against the oracle's match lists."""
import random

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def _counts(pats, text, prefix_len=0):
    a = glop.Automaton(pats, prefix_len=prefix_len)
    t = np.ascontiguousarray(text, dtype=np.uint8).reshape(-1)
    d = torch.from_numpy(t.copy()).cuda() if t.size else torch.zeros(0, dtype=torch.uint8, device="cuda")
    hist, total = a.count(d)
    out = hist.cpu().numpy()
    a.close()
    return out, total


def _expect(matches, n):
    m = np.asarray(matches, np.uint32).reshape(-1, 2)
    return np.bincount(m[:, 1].astype(np.int64), minlength=n)


def test_worked_example_and_nesting():
    h, n = _counts([b"HIS", b"SHE"], np.frombuffer(b"SHIS", np.uint8))
    assert h.tolist() == [1, 0] and n == 1
    pats = [b"a", b"aa", b"aaa", b"aa"]  # nested, with a duplicate
    h, n = _counts(pats, np.frombuffer(b"aaaa", np.uint8))
    assert h.tolist() == [4, 3, 2, 3] and n == 12


@pytest.mark.parametrize("seed", range(6))
def test_random_small(seed):
    rnd = random.Random(seed)
    alpha = bytes(rnd.sample(range(256), rnd.choice([2, 3, 16])))
    pats = [bytes(rnd.choice(alpha) for _ in range(rnd.randint(1 if seed % 2 else 4, 12))) for _ in range(40)]
    text = np.frombuffer(bytes(rnd.choice(alpha) for _ in range(rnd.choice([0, 1, 1000, 70000, 200003]))), np.uint8)
    h, n = _counts(pats, text)
    exp = _expect(oracle.naive(text.tobytes(), pats), len(pats))
    assert np.array_equal(h, exp) and n == int(exp.sum())


def test_config2_slice_and_prefix_mode():
    w = W.config2(8 * W.MiB + 777)
    for k in (0, 8):
        h, n = _counts(w.patterns, w.text, prefix_len=k)
        exp = _expect(oracle.ac_mt(w.text, w.patterns.csr(), prefix_len=k), w.patterns.n)
        assert np.array_equal(h, exp), k
        assert n == int(exp.sum())


def test_config3_slice_single_buffer():
    w = W.config3(4 * W.MiB)
    h, n = _counts(w.patterns, w.text)
    exp = _expect(oracle.ac_mt(w.text, w.patterns.csr()), w.patterns.n)
    assert np.array_equal(h, exp) and n == int(exp.sum())


def test_full_size_config2_agrees_with_the_scan():
    # at full size: the same counts as the match list of the (oracle-checked) scan
    w = W.config2()
    a = glop.Automaton(w.patterns)
    d = torch.from_numpy(w.text).cuda()
    hist, total = a.count(d)
    m, n = a.scan(d)
    exp = torch.bincount(m[:, 1].long(), minlength=w.patterns.n)
    assert total == n
    assert torch.equal(hist, exp)
