"""Groups of links against the CPU oracle.

Each link of a group is its own estimator array (one per edge router, Section 3.1), so each
link's result is defined by the method alone: Algorithm 2 over that link's packets, the slice
end of Section 4.2 and Algorithm 3.  Every test runs one oracle beside every group link, with
the link's parameters, start slice and packets, and compares every report (bit-exact
integers, estimates within 1e-5 relative) and the exported recorder state with it.  A second
check compares each group link with the same link run alone through srla_create.

Covered: links of different geometry, recorder width (one-bit, 8-bit, 16-bit), z and window
in one graph launch per slice, host and device pushes, links that skip slices, an autotune
in the middle of a run, attach and detach between slices with slot and arena reuse, and the
64-link batched geometry (mixed 8/16-bit recorders, windows 16..300, SLE 2^16..2^22 cells per
row) with its packet rates scaled down so that the oracle keeps up.
"""
import dataclasses
import math

import numpy as np
import pytest

import synth
from gpu_helpers import compare_reports, compare_state, oracle_for
from paper_1803_10369_b300 import srla

pytestmark = pytest.mark.gpu

TINY = synth.workload("tiny")


def _links():
    many = synth.Workload(
        name="many-candidates", u=2, v=64, g=64, gl=64, dr_bytes=1, z=4, k=3, theta=64, n_slices=6,
        traffic=synth.TrafficSpec(seed=11, pkts_per_slice=200_000, n_src=1 << 16, zipf_s=0.6,
                                  dst_model="uniform", dst_space=1 << 24),
        max_sampled=1 << 17, max_candidates=1 << 17)
    # rows nearly saturated: the sweep's saturated-estimator bytes are used from slice 2 on
    nearly = synth.Workload(
        name="nearly-saturated", u=2, v=256, g=512, gl=256, dr_bytes=1, z=4, k=3, theta=64, n_slices=6,
        traffic=synth.TrafficSpec(seed=12, pkts_per_slice=200_000, n_src=1 << 16, zipf_s=0.6,
                                  dst_model="uniform", dst_space=1 << 24),
        max_sampled=1 << 17, max_candidates=1 << 17)
    return [
        (TINY, {}),
        (TINY.replace(dr_bytes=2, z=16, k=9, theta=128, gl=256, seed=21, pkts_per_slice=30_000), {}),
        (TINY.replace(z=4, k=15, seed=22, dst_model="pool", pool_max=16), {}),
        (TINY.replace(u=2, v=256, g=32, gl=128, dr_bytes=2, z=12, k=100, theta=64, seed=23,
                      pkts_per_slice=50_000), {"pair_slots_log2": -1}),
        (TINY.replace(z=1, k=1, seed=24, pkts_per_slice=40_000), {}),
        (TINY.replace(dr_bytes=0, z=1, k=1, g=8, gl=256, seed=25, pkts_per_slice=40_000), {}),
        (TINY.replace(z=3, k=6, seed=26, start_slice=5, pkts_per_slice=20_000), {}),
        (TINY.replace(heavy_frac=0.3, dst_model="pool", pool_max=16, seed=28, theta=256), {}),  # heavy build
        (many, {}),
        (nearly, {}),
    ]


def _same(got, want, where):
    """Group link against the same link alone (CUDA against CUDA, a second check)."""
    assert got["aip"].tolist() == want["aip"].tolist(), where
    for key in ("w", "flags", "est"):
        assert np.array_equal(got[key], want[key]), (where, key)
    for key in ("slice", "n_pkts", "n_sampled", "n_new", "n_candidates", "n_carry_out", "w_star", "overflow"):
        assert got["stats"][key] == want["stats"][key], (where, key)
    assert got["stats"]["up"] == want["stats"]["up"], where
    assert np.array_equal(got["stats"]["census"], want["stats"]["census"]), where


def _params(w, **over):
    ha, hb = synth.hash_coefficients(w.hash_seed + w.traffic.seed, w.u + 3)
    return srla.params_for(w, ha, hb, **over)


def _group(n_links=12, arena=1 << 30, max_pkts=4 << 20, max_report=1 << 19):
    return srla.Group(max_links=n_links, max_pkts=max_pkts, arena_bytes=arena, max_host_pkts=1 << 20,
                      max_report=max_report)


def test_group_links_match_oracle(cuda_device):
    links = _links()
    g = _group()
    ids, orc, solo = [], [], []
    for w, over in links:
        p = _params(w, **over)
        ids.append(g.attach(p))
        orc.append(oracle_for(p))
        solo.append(srla.Link(p, device=cuda_device))
    rng = np.random.default_rng(3)
    for s in range(6):
        for i, (w, _) in enumerate(links):
            if (s + i) % 5 == 4:
                continue  # this link gets no packets in this slice
            pk = synth.generate_slice(w.traffic, s)
            orc[i].push(synth.pairs_to_numpy(pk))
            if rng.random() < 0.5:
                g.push(ids[i], pk.to(cuda_device))
            else:
                g.push(ids[i], pk)  # host batch, staged by the group
            solo[i].push(pk.to(cuda_device))
        if s == 2:  # tuning repeats the slice's own scan with other launch shapes: no effect on results
            threads, task = g.autotune(reps=1)
            assert threads in (128, 256, 512) and task in (1 << 14, 1 << 16, 1 << 18)
            assert all(g.scan_policy(l) in range(4) for l in ids)
        gs = g.end_slice()
        allr = g.report_all(gs)
        for i in range(len(links)):
            ro = orc[i].end_slice()
            compare_reports(ro, allr[ids[i]], f"slice {s} link {i} (report_all)")
            compare_reports(ro, g.report(ids[i], gs), f"slice {s} link {i} (report)")
            _same(allr[ids[i]], solo[i].report(solo[i].end_slice()), f"slice {s} link {i} (alone)")
            compare_state(orc[i], g.state_arrays(ids[i]), f"slice {s} link {i}")
    assert max(int(o_n) for o_n in (allr[l]["stats"]["n_candidates"] for l in ids)) > 3 * 4096  # multi-tile sort
    g.close()


def test_links_attach_and_detach_between_slices(cuda_device):
    links = _links()[:4]
    g = _group(n_links=3, arena=256 << 20)
    live = {}  # group link -> (workload index, oracle)

    def attach(i, start):
        w, over = links[i]
        p = _params(w.replace(start_slice=start), **over)
        live[g.attach(p)] = (i, oracle_for(p))

    attach(0, 0)
    attach(1, 100)
    for s in range(8):
        if s == 3:
            attach(2, 7)
        if s == 5:
            gone = next(l for l, (i, _) in live.items() if i == 0)
            g.detach(gone)
            del live[gone]
        if s == 6:
            attach(3, 40)  # reuses the detached link's slot and arena space
        for link, (i, o) in live.items():
            pk = synth.generate_slice(links[i][0].traffic, s)
            g.push(link, pk.to(cuda_device))
            o.push(synth.pairs_to_numpy(pk))
        gs = g.end_slice()
        allr = g.report_all(gs)
        for link, (i, o) in live.items():
            compare_reports(o.end_slice(), allr[link], f"slice {s} workload {i}")
            compare_state(o, g.state_arrays(link), f"slice {s} workload {i}")
    g.close()


def _policy(s, i):
    """Slices 0-7: the four policies rotate over the links.  Slices 8-11: every link on a
    policy without the read-first build, so the group launches its lean scan instantiation."""
    if s < 8:
        return (s + i) % 4
    return (srla.SCAN_POLICY_ADAPTIVE, srla.SCAN_POLICY_OFF)[(s + i) % 2]


def test_group_scan_policies_match_oracle(cuda_device):
    """The four aggregation policies (pair table adaptive or off, plain or read-first build)
    rotate over the links slice by slice, then only the policies without the read-first build
    (the lean scan instantiation); every report and state still equals the oracle's."""
    links = _links()[:8] + [(TINY.replace(seed=27, dst_model="pool", pool_max=4, dr_bytes=2, z=16, k=5), {})]
    g = _group()
    ids, orc, widths = [], [], []
    for w, over in links:
        p = _params(w, **over)
        ids.append(g.attach(p))
        orc.append(oracle_for(p))
        widths.append(p.dr_bytes)
    rf_policies = (srla.SCAN_POLICY_ADAPTIVE_RF, srla.SCAN_POLICY_OFF_RF)
    # slices whose scan is the read-first instantiation: some 8/16-bit link may choose that build
    rf_slices = sum(any(_policy(s, i) in rf_policies and widths[i] for i in range(len(links))) for s in range(12))
    for s in range(12):
        for i, (w, _) in enumerate(links):
            g.set_scan_policy(ids[i], _policy(s, i))
            pk = synth.generate_slice(w.traffic, s)
            orc[i].push(synth.pairs_to_numpy(pk))
            g.push(ids[i], pk.to(cuda_device))
        allr = g.report_all(g.end_slice())
        for i in range(len(links)):
            assert g.scan_policy(ids[i]) == _policy(s, i)
            compare_reports(orc[i].end_slice(), allr[ids[i]], f"slice {s} link {i} policy {_policy(s, i)}")
            compare_state(orc[i], g.state_arrays(ids[i]), f"slice {s} link {i}")
    assert g.scan_builds() == (12 - rf_slices, rf_slices) and rf_slices >= 1 and 12 - rf_slices >= 4
    with pytest.raises(srla.SRLAError) as e:
        g.set_scan_policy(ids[0], 4)
    assert e.value.code == srla.E_INVAL
    g.close()


def _scaled_batched_links(n_links, scale):
    """The batched workload's links (synth.batched_links) with packet rates and planted hosts
    divided by `scale`: same geometry, recorder widths and windows."""
    out = []
    for w, plog in synth.batched_links(n_links):
        t = w.traffic
        t = dataclasses.replace(t, pkts_per_slice=max(2048, t.pkts_per_slice // scale),
                                n_planted=max(1, t.n_planted // 8), planted_card=(1 << 8, 1 << 12))
        out.append((dataclasses.replace(w, traffic=t), plog))
    return out


def test_batched_geometry_64_links_match_oracle(cuda_device):
    """64 links of the batched workload's geometry in one group, 20 slices (past the shortest
    windows), every report against its oracle, every link's state at the end.  The first 10
    slices run the default policy (adaptive table, read-first build when it is off), the last
    10 the adaptive table with the plain build only (the group's lean scan instantiation)."""
    links = _scaled_batched_links(64, 32)
    params = [srla.params_for(w, *synth.hash_coefficients(w.hash_seed, w.u + 3), pair_slots_log2=plog)
              for w, plog in links]
    assert {p.dr_bytes for p in params} == {1, 2} and min(p.k for p in params) <= 20
    arena = sum(srla.Group.link_bytes(p) for p in params) + (64 << 20)
    total = sum(w.pkts_per_slice for w, _ in links)
    g = srla.Group(max_links=64, max_pkts=4 * total + (1 << 20), arena_bytes=arena, max_report=1 << 20,
                   device=cuda_device)
    ids = [g.attach(p) for p in params]
    orc = [oracle_for(p) for p in params]
    n_slices = 20
    for s in range(n_slices):
        if s == n_slices // 2:
            for l in ids:
                g.set_scan_policy(l, srla.SCAN_POLICY_ADAPTIVE)
        for i, (w, _) in enumerate(links):
            pk = synth.generate_slice(w.traffic, s)
            orc[i].push(synth.pairs_to_numpy(pk))
            g.push(ids[i], pk.to(cuda_device))
        allr = g.report_all(g.end_slice())
        for i in range(len(links)):
            compare_reports(orc[i].end_slice(), allr[ids[i]], f"slice {s} link {i} ({links[i][0].name})")
    for i in range(len(links)):
        compare_state(orc[i], g.state_arrays(ids[i]), f"end link {i}")
    assert g.scan_builds() == (n_slices // 2, n_slices // 2)
    g.close()


def test_group_rules(cuda_device):
    w = TINY
    g = _group(n_links=2, arena=srla.Group.link_bytes(_params(w)) + (4 << 20))
    a = g.attach(_params(w))
    with pytest.raises(srla.SRLAError) as e:  # arena full
        g.attach(_params(w))
    assert e.value.code == srla.E_NOMEM
    g.push(a, synth.generate_slice(w.traffic, 0).to(cuda_device))
    with pytest.raises(srla.SRLAError) as e:  # packets already pushed in the open slice
        g.attach(_params(w.replace(v=64)))
    assert e.value.code == srla.E_ORDER
    with pytest.raises(srla.SRLAError) as e:  # state export only at a slice boundary
        g.state_arrays(a)
    assert e.value.code == srla.E_ORDER
    s0 = g.end_slice()
    g.end_slice()
    g.end_slice()
    with pytest.raises(srla.SRLAError) as e:  # only the two latest slices can be reported
        g.report_all(s0)
    assert e.value.code == srla.E_ORDER
    small = _params(w.replace(v=64, gl=64, g=64), pair_slots_log2=10)
    b = g.attach(small)
    with pytest.raises(srla.SRLAError) as e:  # every slot is taken
        g.attach(small)
    assert e.value.code == srla.E_CAPACITY
    g.detach(b)
    with pytest.raises(srla.SRLAError):  # a free slot has no state
        g.state_arrays(b)
    g.close()


def test_failed_attach_leaves_the_group_working(cuda_device):
    """The second link's recorders fit the arena but the rebuilt sweep list of both links does
    not (512 spare bytes: room for one tiny link's list, not two): the attach fails with
    E_NOMEM, is rolled back, and the first link keeps matching the oracle."""
    small = _params(TINY, pair_slots_log2=10)
    lb = srla.Group.link_bytes(small)
    g = _group(n_links=2, arena=2 * lb + 512)
    a = g.attach(small)
    with pytest.raises(srla.SRLAError) as e:
        g.attach(_params(TINY.replace(seed=31), pair_slots_log2=10))
    assert e.value.code == srla.E_NOMEM
    o = oracle_for(small)
    for s in range(4):
        pk = synth.generate_slice(TINY.traffic, s)
        g.push(a, pk.to(cuda_device))
        o.push(synth.pairs_to_numpy(pk))
        compare_reports(o.end_slice(), g.report(a, g.end_slice()), f"slice {s}")
    compare_state(o, g.state_arrays(a), "end")
    g.close()
