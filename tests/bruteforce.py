"""Ground truth by brute force, for tiny traces (test helpers).

* ``exact_cardinalities``: the precise method of Section 3.2 -- the set of distinct
  opposite hosts of every host over the window W(T-k+1, k), counted exactly.
* ``LastSeen``: the meaning of a distance recorder stated as a set-level fact.  A recorder
  holds the distance from the current slice to the most recent slice in which some pair
  mapped to it (Section 3.2), so it is enough to remember, for every cell, the last slice
  that touched it.  Every count the estimator uses (row census, union SRE, union SLE) then
  follows from "touched within the last k slices", without the increment mechanism of
  Algorithm 3.  The cell mapping uses the oracle's hash functions, so these checks pin the
  window logic and the candidate rule, not the hash family.
"""
from __future__ import annotations

import numpy as np

NEVER = np.iinfo(np.int64).min // 4


def exact_cardinalities(slices, T: int, k: int, first_slice: int = 0) -> dict:
    """|OP(aip, T-k+1, k)| for every aip seen in the window ending at slice T."""
    lo = max(first_slice, T - k + 1)
    parts = [slices[s - first_slice] for s in range(lo, T + 1)]
    if not parts:
        return {}
    allp = np.concatenate(parts).astype(np.uint64)
    keys = np.unique((allp[:, 0] << np.uint64(32)) | allp[:, 1])
    a = (keys >> np.uint64(32)).astype(np.uint32)
    ua, cnt = np.unique(a, return_counts=True)
    return dict(zip(ua.tolist(), cnt.tolist()))


class LastSeen:
    """Per-cell last touching slice, fed slice by slice with the oracle's hashes."""

    def __init__(self, orc, start_slice: int = 0):
        self.o = orc
        u, v, g, gl = orc.u, orc.v, orc.g, orc.gl
        self.last_re = np.full((u, v, g), NEVER, np.int64)
        self.last_le = np.full((u, v, gl), NEVER, np.int64)
        self.T = start_slice
        self.sampled_hosts = set()
        tau = orc.tau
        self.mask = np.uint32((1 << tau) - 1) if tau < 32 else None

    def _cols(self, a):
        return [(self.o.hash(i, a) & np.uint32(self.o.v - 1)).astype(np.int64) for i in range(self.o.u)]

    def feed(self, pairs):
        """Pairs of the open slice T."""
        if pairs.shape[0] == 0:
            return
        o = self.o
        a = pairs[:, 0].copy()
        b = pairs[:, 1].copy()
        cols = self._cols(a)
        jl = (o.hash(o.u, b) & np.uint32(o.gl - 1)).astype(np.int64)
        hs = o.hash(o.u + 2, b)
        # LSB(h) >= tau  <=>  the low tau bits of h are all zero (LSB(0) = 32 >= tau).
        samp = (hs == 0) if self.mask is None else ((hs & self.mask) == 0)
        jr = (o.hash(o.u + 1, b) & np.uint32(o.g - 1)).astype(np.int64)
        for i in range(o.u):
            self.last_le[i, cols[i], jl] = self.T
            self.last_re[i, cols[i][samp], jr[samp]] = self.T
        self.sampled_hosts.update(a[samp].tolist())

    # -- counts at the end of the open slice T (before the slide) --------------------
    def in_window_le(self, shift=0):
        return self.last_le >= self.T - self.o.k + 1 + shift

    def in_window_re(self, shift=0):
        return self.last_re >= self.T - self.o.k + 1 + shift

    def census(self):
        return self.in_window_le().reshape(self.o.u, -1).sum(axis=1).astype(np.uint64)

    def union_count(self, aip: int, which: str, shift: int = 0) -> int:
        """|URE(aip)|^k or |ULE(aip)|^k; shift=1 is the post-slide window (d + 1 < k)."""
        o = self.o
        cols = [int(c[0]) for c in self._cols(np.array([aip], np.uint32))]
        iw = self.in_window_re(shift) if which == "re" else self.in_window_le(shift)
        allrows = np.ones(iw.shape[2], bool)
        for i in range(o.u):
            allrows &= iw[i, cols[i]]
        return int(allrows.sum())

    def distances_after_slide(self):
        """Recorder distances as seen from slice T + 1, capped at 2^z - 1."""
        dmax = (1 << self.o.z) - 1
        T1 = self.T + 1
        re = np.where(self.last_re == NEVER, dmax, np.minimum(T1 - self.last_re, dmax))
        le = np.where(self.last_le == NEVER, dmax, np.minimum(T1 - self.last_le, dmax))
        return re.astype(np.uint16), le.astype(np.uint16)

    def next_slice(self):
        self.T += 1
        self.sampled_hosts = set()
