"""Groups of links: every link's report in the group equals the report of the same link run
alone (a single-link handle fed the same packets), slice by slice, while links of different
geometry, recorder width and window share one graph launch per slice, and while links attach
and detach between slices.  The single-link path is itself checked against the oracle."""
import numpy as np
import pytest
import torch

import synth
from paper_1803_10369_b300 import srla

pytestmark = pytest.mark.gpu

TINY = synth.workload("tiny")


def _links():
    many = synth.Workload(
        name="many-candidates", u=2, v=64, g=64, gl=64, dr_bytes=1, z=4, k=3, theta=64, n_slices=6,
        traffic=synth.TrafficSpec(seed=11, pkts_per_slice=200_000, n_src=1 << 16, zipf_s=0.6,
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
        (many, {}),
    ]


def _same(got, want, where):
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


def _group(n_links=8, arena=1 << 30):
    return srla.Group(max_links=n_links, max_pkts=4 << 20, arena_bytes=arena, max_host_pkts=1 << 20,
                      max_report=1 << 18)


def test_group_equals_links_alone(cuda_device):
    links = _links()
    g = _group()
    solo, ids = [], []
    for w, over in links:
        p = _params(w, **over)
        ids.append(g.attach(p))
        solo.append(srla.Link(p, device=cuda_device))
    rng = np.random.default_rng(3)
    for s in range(6):
        for i, (w, _) in enumerate(links):
            if (s + i) % 5 == 4:
                continue  # this link gets no packets in this slice
            pk = synth.generate_slice(w.traffic, s)
            if rng.random() < 0.5:
                g.push(ids[i], pk.to(cuda_device))
            else:
                g.push(ids[i], pk)  # host batch, staged by the group
            solo[i].push(pk.to(cuda_device))
        if s == 2:  # tuning repeats the slice's own scan with other launch shapes: no effect on results
            threads, task = g.autotune(reps=1)
            assert threads in (128, 256, 512) and task in (1 << 14, 1 << 16, 1 << 18)
        gs = g.end_slice()
        want = [solo[i].report(solo[i].end_slice()) for i in range(len(links))]
        allr = g.report_all(gs)
        for i in range(len(links)):
            _same(allr[ids[i]], want[i], f"slice {s} link {i} (report_all)")
            _same(g.report(ids[i], gs), want[i], f"slice {s} link {i} (report)")
    assert max(r["stats"]["n_candidates"] for r in want) > 3 * 4096  # the cooperative sort ran
    g.close()


def test_links_attach_and_detach_between_slices(cuda_device):
    links = _links()[:4]
    g = _group(n_links=3, arena=256 << 20)
    live = {}  # group link -> (workload index, solo link)

    def attach(i, start):
        w, over = links[i]
        p = _params(w.replace(start_slice=start), **over)
        live[g.attach(p)] = (i, srla.Link(p, device=cuda_device))

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
        for link, (i, solo) in live.items():
            pk = synth.generate_slice(links[i][0].traffic, s).to(cuda_device)
            g.push(link, pk)
            solo.push(pk)
        gs = g.end_slice()
        allr = g.report_all(gs)
        for link, (i, solo) in live.items():
            _same(allr[link], solo.report(solo.end_slice()), f"slice {s} workload {i}")
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
    g.close()


def test_failed_attach_leaves_the_group_working(cuda_device):
    """The second link's recorders fit the arena but the rebuilt sweep list of both links does
    not (512 spare bytes: room for one tiny link's list, not two): the attach fails with
    E_NOMEM, is rolled back, and the first link keeps matching the same link run alone."""
    small = _params(TINY, pair_slots_log2=10)
    lb = srla.Group.link_bytes(small)
    g = _group(n_links=2, arena=2 * lb + 512)
    a = g.attach(small)
    with pytest.raises(srla.SRLAError) as e:
        g.attach(_params(TINY.replace(seed=31), pair_slots_log2=10))
    assert e.value.code == srla.E_NOMEM
    solo = srla.Link(small, device=cuda_device)
    for s in range(4):
        pk = synth.generate_slice(TINY.traffic, s).to(cuda_device)
        g.push(a, pk)
        solo.push(pk)
        _same(g.report(a, g.end_slice()), solo.report(solo.end_slice()), f"slice {s}")
    g.close()
