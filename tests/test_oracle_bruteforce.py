"""The oracle against brute force on tiny traces (no GPU).

Every recorder distance, row census, union count, candidate list and carried list of the
oracle must equal what follows from "the last slice that touched a cell" (bruteforce.py),
which states the meaning of a distance recorder (Section 3.2) without the increment
mechanism of Algorithm 3.  Plus the invariants of the sliding window: a host unseen for a
full window contributes nothing, k = 1 is the discrete window, and the carry of Algorithm 3
keeps a host whose opposite hosts all lie in the last k - 1 slices.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from bruteforce import LastSeen, exact_cardinalities

CASES = [
    # u, v, g, gl, z, k, theta, n_src, n_dst, pkts, slices
    (2, 8, 8, 16, 3, 3, 16, 40, 200, 300, 12),
    (3, 16, 16, 32, 2, 3, 40, 60, 400, 500, 9),    # k = 2^z - 1
    (1, 4, 8, 8, 1, 1, 8, 20, 100, 120, 6),        # discrete window
    (4, 32, 16, 64, 8, 5, 64, 200, 3000, 2000, 10),
    (2, 16, 32, 32, 16, 7, 200, 80, 5000, 1500, 10),
]


@pytest.mark.parametrize("case", CASES)
def test_oracle_matches_last_seen_semantics(case):
    u, v, g, gl, z, k, theta, n_src, n_dst, pkts, slices = case
    a, b = synth.hash_coefficients(hash(case) & 0xFFFF, u + 3)
    start = 1000
    o = oracle.Oracle(u, v, g, gl, z, k, theta, a, b, start_slice=start)
    bf = LastSeen(o, start_slice=start)
    carry_prev = set()
    rng = np.random.default_rng(len(case) + pkts)
    for s in range(slices):
        n = int(rng.integers(0, pkts + 1)) if s % 4 != 3 else 0   # ragged and empty slices
        pairs = synth.random_pairs(s * 31 + u, n, n_src, n_dst)
        o.push(pairs)
        bf.feed(pairs)
        rep = o.end_slice()

        assert np.array_equal(rep["cnt"], bf.census())
        up = np.prod(bf.census().astype(np.float64) / (gl * v))
        assert rep["up"] == pytest.approx(up, rel=1e-12, abs=0)

        new = sorted(x for x in bf.sampled_hosts if bf.union_count(x, "re") >= o.rho_g)
        csip = sorted(set(new) | carry_prev)
        assert rep["aip"].tolist() == csip
        for aip, w, est, f in zip(rep["aip"], rep["w"], rep["est"], rep["flags"]):
            assert w == bf.union_count(int(aip), "le")
            assert bool(f & oracle.NEW) == (int(aip) in new)
            assert bool(f & oracle.CARRIED) == (int(aip) in carry_prev)
            e, sf = oracle.estimate(gl, up, w)
            assert (math.isinf(e) and math.isinf(est)) or est == pytest.approx(e, rel=1e-12)
            assert bool(f & oracle.SUPER) == (bool(sf) or e >= theta)

        carry = sorted(x for x in csip if bf.union_count(x, "re", shift=1) >= o.rho_g)
        assert o.carry().tolist() == carry
        carry_prev = set(carry)

        re, le = o.state()
        bre, ble = bf.distances_after_slide()
        assert np.array_equal(re, bre) and np.array_equal(le, ble)
        bf.next_slice()
    o.close()


def test_k1_is_the_discrete_window():
    """k = 1 (z = 1): every slice equals a fresh estimator array on that slice alone, and the
    carried list is always empty (Section 3.1)."""
    u, v, g, gl, theta = 3, 32, 16, 64, 24
    a, b = synth.hash_coefficients(4, u + 3)
    run = oracle.Oracle(u, v, g, gl, 1, 1, theta, a, b)
    for s in range(8):
        pairs = synth.random_pairs(900 + s, 1500, 100, 4000)
        run.push(pairs)
        r1 = run.end_slice()
        fresh = oracle.Oracle(u, v, g, gl, 1, 1, theta, a, b, start_slice=s)
        fresh.push(pairs)
        r2 = fresh.end_slice()
        for key in ("aip", "w", "flags", "cnt"):
            assert np.array_equal(r1[key], r2[key])
        assert np.array_equal(r1["est"], r2["est"])
        assert run.carry().size == 0
        fresh.close()
    run.close()


def _mk_host_pairs(aip, bips):
    return np.stack([np.full(len(bips), aip, np.uint32), np.asarray(bips, np.uint32)], axis=1)


def test_host_unseen_for_a_window_contributes_nothing():
    u, v, g, gl, z, k, theta = 4, 64, 32, 128, 4, 3, 64
    a, b = synth.hash_coefficients(8, u + 3)
    X = 0xC0A80001
    rng = np.random.default_rng(3)
    bg = [synth.random_pairs(70 + s, 800, 300, 10_000) for s in range(7)]
    xs = [rng.choice(1 << 32, size=400, replace=False).astype(np.uint32) for _ in range(3)]
    runs = []
    for with_x in (True, False):
        o = oracle.Oracle(u, v, g, gl, z, k, theta, a, b)
        reps, states = [], []
        for s in range(7):
            p = bg[s]
            if with_x and s < 3:
                p = np.concatenate([p, _mk_host_pairs(X, xs[s])])
            o.push(p)
            re, le = o.state()
            states.append((re < k, le < k))
            reps.append(o.end_slice())
        runs.append((reps, states))
        o.close()
    # X is last seen in slice 2; from slice 2 + k = 5 on it must leave no trace.
    for t in (5, 6):
        ra, sa = runs[0][0][t], runs[0][1][t]
        rb, sb = runs[1][0][t], runs[1][1][t]
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        assert np.array_equal(ra["cnt"], rb["cnt"])
        assert X not in ra["aip"].tolist() or not (ra["flags"][ra["aip"].tolist().index(X)] & oracle.NEW)
        common = np.intersect1d(ra["aip"], rb["aip"])
        for x in common:
            ia, ib = ra["aip"].tolist().index(x), rb["aip"].tolist().index(x)
            assert ra["w"][ia] == rb["w"][ib] and ra["est"][ia] == rb["est"][ib]
        # entries in only one run can only come from a carry chain
        for r, other in ((ra, rb), (rb, ra)):
            only = np.setdiff1d(r["aip"], other["aip"])
            for x in only:
                f = r["flags"][r["aip"].tolist().index(x)]
                assert f & oracle.CARRIED and not f & oracle.NEW


def test_carry_keeps_a_host_seen_only_in_the_last_k_minus_1_slices():
    """Algorithm 3's example: all of X's opposite hosts lie in slices t+1 .. t+k-1, X sends
    nothing in slice t+k, yet X is reported for W(t+1, k) because it was carried."""
    u, v, g, gl, z, k, theta = 4, 256, 64, 1024, 4, 4, 256
    a, b = synth.hash_coefficients(21, u + 3)
    X = 0x0A0B0C0D
    o = oracle.Oracle(u, v, g, gl, z, k, theta, a, b)
    rng = np.random.default_rng(17)
    xs = rng.choice(1 << 32, size=3 * 300, replace=False).astype(np.uint32)
    slices = []
    for s in range(k + 1):                       # slices 0 .. k with t = 0
        p = synth.random_pairs(500 + s, 2000, 500, 50_000)
        if 1 <= s <= k - 1:
            p = np.concatenate([p, _mk_host_pairs(X, xs[(s - 1) * 300:s * 300])])
        slices.append(p)
        o.push(p)
        rep = o.end_slice()
        if s == k - 1:
            assert X in rep["aip"].tolist()
    i = rep["aip"].tolist().index(X)
    assert rep["flags"][i] & oracle.CARRIED and not rep["flags"][i] & oracle.NEW
    truth = exact_cardinalities(slices, k, k)[X]
    assert truth == 900
    assert rep["flags"][i] & oracle.SUPER
    assert abs(rep["est"][i] - truth) < 0.15 * truth
    o.close()


def test_start_slice_is_only_a_label():
    u, v, g, gl, z, k, theta = 2, 16, 16, 32, 5, 6, 40
    a, b = synth.hash_coefficients(2, u + 3)
    outs = []
    for start in (0, 12345, (1 << 40) + 7):
        o = oracle.Oracle(u, v, g, gl, z, k, theta, a, b, start_slice=start)
        got = []
        for s in range(9):
            o.push(synth.random_pairs(s, 700, 90, 2000))
            r = o.end_slice()
            got.append((r["aip"].tolist(), r["w"].tolist(), r["flags"].tolist()))
        assert o.slice == start + 9
        outs.append((got, o.state()))
        o.close()
    for got, st in outs[1:]:
        assert got == outs[0][0]
        assert all(np.array_equal(x, y) for x, y in zip(st, outs[0][1]))


def test_planted_super_points_are_found_on_the_tiny_workload():
    """Accuracy (not parity): with g' = 1024 and theta = 128, every planted host whose window
    cardinality is at least 2 theta is reported as a super point (Definition 2)."""
    w = synth.workload("tiny").replace(gl=1024, theta=128)
    a, b = synth.hash_coefficients(w.hash_seed, w.u + 3)
    o = oracle.Oracle.for_workload(w, a, b)
    tr = [synth.pairs_to_numpy(t) for t in synth.generate_trace(w.traffic, 8)]
    for s in range(8):
        o.push(tr[s])
        rep = o.end_slice()
    truth = exact_cardinalities(tr, 7, w.k)
    big = [x for x, c in truth.items() if c >= 2 * w.theta]
    sup = set(rep["aip"][(rep["flags"] & oracle.SUPER) != 0].tolist())
    assert big and all(x in sup for x in big)
    o.close()
