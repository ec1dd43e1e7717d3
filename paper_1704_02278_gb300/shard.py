"""Sharding the scan across ranks (one process per GPU), host logic only.

The scan needs no exchange while it runs (Sec. 4: chunks that overlap by the
longest pattern - 1 bytes find every match; each chunk keeps the matches that
start inside it).  So a text splits into per-rank byte ranges plus that
overlap, batches split by whole segments, and the results of the ranks are
concatenated in rank order -- the only collective is that final gather.
"""
from __future__ import annotations

import numpy as np


def text_shard(n: int, rank: int, world: int, max_pattern_len: int):
    """(owned_lo, owned_hi, read_hi): rank scans text[owned_lo:read_hi] and keeps matches starting in
    [owned_lo, owned_hi).  read_hi adds the overlap of max_pattern_len - 1 bytes (clipped to n)."""
    chunk = (n + world - 1) // world if world else n
    lo = min(n, rank * chunk)
    hi = min(n, lo + chunk)
    return lo, hi, min(n, hi + max(max_pattern_len - 1, 0))


def keep_owned(matches: np.ndarray, owned_lo: int, owned_hi: int) -> np.ndarray:
    """Matches (offset relative to owned_lo, pattern_id) of a shard -> absolute offsets, owned starts only."""
    m = np.asarray(matches, dtype=np.uint32).reshape(-1, 2)
    off = m[:, 0].astype(np.int64) + owned_lo
    sel = off < owned_hi
    out = np.empty((int(sel.sum()), 2), np.uint32)
    out[:, 0] = off[sel]
    out[:, 1] = m[sel, 1]
    return out


def segment_shard(seg_offsets, rank: int, world: int):
    """Contiguous run of whole segments [s_lo, s_hi) for rank, about equal bytes per rank."""
    seg = np.asarray(seg_offsets, dtype=np.int64)
    nseg = len(seg) - 1
    total = int(seg[-1] - seg[0]) if nseg > 0 else 0
    bounds = [0]
    for r in range(1, world):
        goal = seg[0] + total * r // world
        bounds.append(int(np.searchsorted(seg[1:], goal, side="right")))
    bounds.append(nseg)
    for i in range(1, len(bounds)):
        bounds[i] = max(bounds[i], bounds[i - 1])
    return bounds[rank], bounds[rank + 1]


def merge_ranked(parts):
    """Concatenate per-rank sorted results in rank order (already globally sorted by construction)."""
    parts = [np.asarray(p) for p in parts if len(p)]
    return np.concatenate(parts) if parts else np.zeros((0, 2), np.uint32)
