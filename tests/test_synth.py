"""The seeded input generator: determinism and the stated traffic shape (no GPU)."""
import numpy as np

import synth
from bruteforce import exact_cardinalities


def test_slices_are_deterministic_and_independent():
    spec = synth.workload("tiny").traffic
    a = synth.pairs_to_numpy(synth.generate_slice(spec, 5))
    b = synth.pairs_to_numpy(synth.generate_slice(spec, 5))
    c = synth.pairs_to_numpy(synth.generate_slice(spec, 6))
    assert a.shape == (spec.pkts_per_slice, 2) and a.dtype == np.uint32
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_hash_coefficients_in_range():
    a, b = synth.hash_coefficients(3, 64)
    assert (a >= 1).all() and (a < synth.MERSENNE_61).all() and (b < synth.MERSENNE_61).all()
    a2, _ = synth.hash_coefficients(3, 64)
    assert np.array_equal(a, a2)


def test_tiny_planted_hosts_have_their_cardinality():
    w = synth.workload("tiny")
    tr = [synth.pairs_to_numpy(t) for t in synth.generate_trace(w.traffic, 16)]
    card16 = exact_cardinalities(tr, 15, 16)
    addr, card, _ = synth.planted_hosts(w.traffic)
    # 20 planted hosts with 500..3000 fresh distinct destinations over the 16 slices
    assert len(addr) == 20 and (card >= 500).all() and (card <= 3000).all()
    for a, c in zip(addr.tolist(), card.tolist()):
        assert card16[a] == c
    srcs = np.unique(np.concatenate(tr)[:, 0])
    assert srcs.size <= (1 << 12) + 20


def test_longwin_flood_and_heavy_source():
    w = synth.workload("longwin").replace(pkts_per_slice=1 << 16, flood_sources=1 << 14,
                                          flood_slices=(0, 4))
    s = synth.pairs_to_numpy(synth.generate_slice(w.traffic, 1))
    aips, cnt = np.unique(s[:, 0], return_counts=True)
    assert cnt.max() >= 0.09 * s.shape[0]          # the heavy source
    assert (cnt == 1).sum() >= (1 << 14) // 4 * 0.9  # one-packet spoofed sources


def test_flow_bursts_repeat_each_pair_back_to_back():
    """burst_mean = 8: background pairs come in runs of a geometric length (mean 8), the slice
    keeps its packet count, and the planted hosts keep their destinations."""
    w = synth.workload("tiny")
    b = w.replace(burst_mean=8.0)
    s = synth.pairs_to_numpy(synth.generate_slice(b.traffic, 4))
    assert s.shape == (w.pkts_per_slice, 2)
    key = (s[:, 0].astype(np.uint64) << np.uint64(32)) | s[:, 1].astype(np.uint64)
    starts = np.concatenate([[True], key[1:] != key[:-1]])
    runs = np.diff(np.concatenate([np.flatnonzero(starts), [key.size]]))
    # each distinct pair forms one run (uniform destinations over 2^20 almost never repeat)
    assert np.unique(key).size >= 0.99 * runs.size
    planted = set(synth.planted_hosts(w.traffic)[0].tolist())
    bg = np.array([a not in planted for a in s[starts, 0].tolist()])
    assert 7.0 < runs[bg].mean() < 9.0
    # planted hosts: the same destinations as without bursts
    p = synth.pairs_to_numpy(synth.generate_slice(w.traffic, 4))
    pk = lambda x: {tuple(r) for r in x[np.isin(x[:, 0], list(planted))].tolist()}
    assert pk(s) == pk(p)
    assert np.array_equal(s, synth.pairs_to_numpy(synth.generate_slice(b.traffic, 4)))
