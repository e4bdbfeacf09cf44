"""The precise method and the rates of the accuracy study (Section 5), on the CPU: exact
super points against a plain per-host set count, including hosts and opposite hosts with the
top bit set (negative as int32), and the FPR/FNR/TFR definitions."""
import numpy as np
import torch

from paper_1803_10369_b300 import accuracy


def test_exact_super_points_against_sets():
    rng = np.random.default_rng(3)
    hosts = rng.integers(0, 1 << 32, size=40, dtype=np.uint64)
    batches, want = [], {}
    for _ in range(3):
        a = hosts[rng.integers(0, len(hosts), size=5000)]
        b = rng.integers(0, 1 << 32, size=5000, dtype=np.uint64) % np.uint64(400)
        b[::7] |= np.uint64(0x80000000)
        pairs = np.stack([a, b], axis=1).astype(np.uint32)
        batches.append(torch.from_numpy(pairs.view(np.int32)))
        for x, y in pairs.tolist():
            want.setdefault(x, set()).add(y)
    for theta in (1, 50, 200, 350, 10 ** 6):
        truth = {x for x, s in want.items() if len(s) >= theta}
        assert accuracy.exact_super_points(batches, theta) == truth


def test_rates_follow_the_definition():
    r = accuracy.rates(reported={1, 2, 3, 9}, truth={1, 2, 4, 5})
    assert (r["N"], r["N_plus"], r["N_minus"]) == (4, 2, 2)
    assert r["fpr"] == 0.5 and r["fnr"] == 0.5 and r["tfr"] == 1.0
    assert accuracy.rates(set(), set())["tfr"] == 0.0
