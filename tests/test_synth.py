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
