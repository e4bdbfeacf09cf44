"""The oracle's inline candidate mode (Algorithm 2 as printed: the union SRE test at packet
time, with the super point indicator bits SI of Section 4.1) against what the paper fixes
about it, on the CPU:

* the inline candidate lists are contained in the order-free ones (the union SRE only grows
  within a slice), slice after slice, and the common hosts get the same estimates;
* without estimator sharing between hosts the two modes give the same candidate lists;
* a host whose SI bit is already set in all of its estimators is not inserted (the SI
  suppression the paper accepts), while one with another SI bit is;
* at each slice end the SI bits are exactly those of the carried hosts (Algorithm 3), and a
  carried host is not inserted again.
"""
import numpy as np
import pytest

import oracle
import synth

SUPER_SAT = oracle.SUPER | oracle.SATURATED


def _pair(w, inline):
    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    return oracle.Oracle.for_workload(w, ha, hb, inline=inline)


def _si_bit(o, aip):
    return int(o.hash(o.u + 2, [aip])[0]) >> 28


def _cols(o, aip):
    return [int(o.hash(i, [aip])[0]) & (o.v - 1) for i in range(o.u)]


TINY = synth.workload("tiny")


@pytest.mark.parametrize("w", [
    TINY.replace(n_slices=8),
    TINY.replace(n_slices=8, u=2, v=64, theta=128, seed=9),
    TINY.replace(n_slices=6, z=1, k=1, seed=10),
])
def test_inline_lists_are_contained_in_the_order_free_lists(w):
    canon, inl = _pair(w, False), _pair(w, True)
    shrunk = 0
    for s in range(w.n_slices):
        pk = synth.pairs_to_numpy(synth.generate_slice(w.traffic, s))
        canon.push(pk)
        inl.push(pk)
        rc, ri = canon.end_slice(), inl.end_slice()
        a_c, a_i = rc["aip"].tolist(), ri["aip"].tolist()
        assert set(a_i) <= set(a_c), f"slice {s}"
        shrunk += len(a_c) - len(a_i)
        pos = {a: x for x, a in enumerate(a_c)}
        for x, a in enumerate(a_i):
            y = pos[a]
            assert ri["w"][x] == rc["w"][y]
            assert (ri["flags"][x] & SUPER_SAT) == (rc["flags"][y] & SUPER_SAT)
            assert ri["est"][x] == rc["est"][y] or (np.isinf(ri["est"][x]) and np.isinf(rc["est"][y]))
        # the recorders themselves do not depend on the candidate rule
        for A, B in zip(canon.state(), inl.state()):
            assert np.array_equal(A, B)
    canon.close()
    inl.close()


def test_without_shared_estimators_both_modes_agree():
    """u = 2 rows of v = 2^16 columns and hosts whose columns are distinct in both rows: a
    host's union SRE depends on its own packets only, so the test at its last sampled packet
    sees the end-of-slice count, and no other host can set its SI bits."""
    u, v, g, gl, z, k, theta = 2, 1 << 16, 64, 64, 4, 3, 256
    a, b = synth.hash_coefficients(77, u + 3)
    canon = oracle.Oracle(u, v, g, gl, z, k, theta, a, b)
    inl = oracle.Oracle(u, v, g, gl, z, k, theta, a, b, inline=True)
    rng = np.random.default_rng(5)
    hosts, used = [], [set(), set()]
    for h in rng.integers(1, 1 << 32, size=400, dtype=np.uint64).tolist():
        c = _cols(canon, h)
        if all(c[i] not in used[i] for i in range(u)):
            hosts.append(h)
            for i in range(u):
                used[i].add(c[i])
        if len(hosts) == 120:
            break
    n_cand = 0
    for s in range(7):
        pairs = []
        for x, h in enumerate(hosts):
            card = int(rng.integers(1, 600)) if (x + s) % 3 else 0
            pairs += [(h, int(d)) for d in rng.integers(0, 1 << 32, size=card, dtype=np.uint64)]
        pairs = np.array(pairs, dtype=np.uint32).reshape(-1, 2)
        pairs = pairs[rng.permutation(len(pairs))]
        canon.push(pairs)
        inl.push(pairs)
        rc, ri = canon.end_slice(), inl.end_slice()
        assert ri["aip"].tolist() == rc["aip"].tolist(), f"slice {s}"
        assert np.array_equal(ri["w"], rc["w"])
        n_cand += len(rc["aip"])
    assert n_cand > 50


def _suppression_setup():
    """u = 1 row of v = 4 columns, tau = 0 (every pair sampled), threshold ceil(rho g) = 18."""
    u, v, g, gl, z, k, theta = 1, 4, 64, 64, 4, 3, 64
    a, b = synth.hash_coefficients(31, u + 3)
    probe = oracle.Oracle(u, v, g, gl, z, k, theta, a, b)
    assert probe.tau == 0 and probe.rho_g == 18
    x = 1000
    cx, bx = _cols(probe, x), _si_bit(probe, x)
    same = next(h for h in range(2000, 200000) if _cols(probe, h) == cx and _si_bit(probe, h) == bx)
    other = next(h for h in range(2000, 200000) if _cols(probe, h) == cx and _si_bit(probe, h) != bx)
    probe.close()
    return (u, v, g, gl, z, k, theta, a, b), x, same, other


def test_si_bit_suppresses_a_host_sharing_its_estimators():
    args, x, same, other = _suppression_setup()
    # x reaches the threshold with 40 destinations; then `same` (same estimator, same SI
    # bit) and `other` (same estimator, another SI bit) send one packet each
    pairs = [(x, 10 + d) for d in range(40)] + [(same, 7), (other, 8)]
    pairs = np.array(pairs, dtype=np.uint32)
    inl = oracle.Oracle(*args[:7], args[7], args[8], inline=True)
    canon = oracle.Oracle(*args[:7], args[7], args[8])
    inl.push(pairs)
    canon.push(pairs)
    ri, rc = inl.end_slice(), canon.end_slice()
    assert sorted(rc["aip"].tolist()) == sorted([x, same, other])
    assert sorted(ri["aip"].tolist()) == sorted([x, other])   # `same` was suppressed


def test_inline_test_runs_at_packet_time():
    """A host whose only packet comes before its estimator fills is not inserted, although
    the union SRE passes at the end of the slice (the order-free rule admits it)."""
    args, x, same, other = _suppression_setup()
    pairs = np.array([(other, 8)] + [(x, 10 + d) for d in range(40)], dtype=np.uint32)
    inl = oracle.Oracle(*args[:7], args[7], args[8], inline=True)
    canon = oracle.Oracle(*args[:7], args[7], args[8])
    inl.push(pairs)
    canon.push(pairs)
    assert sorted(canon.end_slice()["aip"].tolist()) == sorted([x, other])
    assert inl.end_slice()["aip"].tolist() == [x]


def test_si_holds_exactly_the_carried_hosts_after_each_slice_end():
    w = TINY.replace(n_slices=8, k=4)
    o = _pair(w, True)
    for s in range(w.n_slices):
        pk = synth.pairs_to_numpy(synth.generate_slice(w.traffic, s))
        carried_in = set(o.carry().tolist())
        o.push(pk)
        r = o.end_slice()
        for a, f in zip(r["aip"].tolist(), r["flags"].tolist()):
            # a carried host already has its SI bit: it is never inserted again
            assert not (a in carried_in and f & oracle.NEW)
        want = np.zeros((o.u, o.v), np.uint16)
        for a in o.carry().tolist():
            bit = _si_bit(o, a)
            for i, c in enumerate(_cols(o, a)):
                want[i, c] |= 1 << bit
        assert np.array_equal(o.si(), want), f"slice {s}"
    o.close()
