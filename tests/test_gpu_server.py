"""The serving loop against the CPU oracle.

Links arrive, wait for admission under a byte budget, run, and depart.  Each served link is
an independent estimator array (Section 3.1), so from its admission on its results are
defined by the method over its own packets (Algorithm 2, Section 4.2, Algorithm 3).  Every
admitted link runs beside an oracle with its parameters and packets; every tick's report and
the link's exported state are compared with it (bit-exact integers, estimates within 1e-5
relative).  As a second check each link is also compared with the same link run alone, so
that a result is shown to be the same alone and in the mix.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import compare_reports, compare_state, oracle_for
from paper_1803_10369_b300 import srla

pytestmark = pytest.mark.gpu

TINY = synth.workload("tiny")


def _same(got, want, where):
    assert got["aip"].tolist() == want["aip"].tolist(), where
    for key in ("w", "flags", "est"):
        assert np.array_equal(got[key], want[key]), (where, key)
    for key in ("n_pkts", "n_sampled", "n_new", "n_candidates", "n_carry_out"):
        assert got["stats"][key] == want["stats"][key], (where, key)
    assert np.array_equal(got["stats"]["census"], want["stats"]["census"]), where


def test_served_links_match_oracle(cuda_device):
    works = [TINY.replace(seed=40 + i, pkts_per_slice=20_000 + 5_000 * i, k=3 + i, start_slice=10 * i)
             for i in range(4)]
    params = []
    for i, w in enumerate(works):
        ha, hb = synth.hash_coefficients(300 + i, w.u + 3)
        params.append(srla.params_for(w, ha, hb, pair_slots_log2=12))
    one = srla.Group.link_bytes(params[0])
    srv = srla.Server(max_links=4, max_pkts=1 << 20, budget_bytes=2 * one + (1 << 20), arena_bytes=4 * one + (16 << 20))
    run, started, step = {}, {}, {}  # key -> (oracle, link alone)
    srv.open(0, params[0])
    srv.open(1, params[1])
    srv.open(2, params[2])  # waits: the budget holds two links
    rng = np.random.default_rng(9)
    for t in range(9):
        if t == 2:
            srv.open(3, params[3])   # queued behind link 2
        if t == 4:
            srv.close(0)             # frees room: link 2 is admitted at this tick
        if t == 6:
            srv.close(1)             # link 3 follows
        for key in list(run):
            pk = synth.generate_slice(works[key].traffic, step[key])
            step[key] += 1
            dev = pk.to(cuda_device)
            cuts = np.sort(rng.integers(0, pk.shape[0], size=3))
            pieces = np.split(np.arange(pk.shape[0]), cuts)
            for pc in pieces:  # several submits of uneven sizes
                if pc.size:
                    assert srv.submit(key, dev[pc[0]:pc[-1] + 1])
            run[key][0].push(synth.pairs_to_numpy(pk))
            run[key][1].push(dev)
        sl, admitted, waiting = srv.tick()
        res = srv.poll(sl)
        for key in list(run):
            if key in (0,) and t >= 4 or key == 1 and t >= 6:
                assert key not in res
                del run[key]
                continue
            o, alone = run[key]
            compare_reports(o.end_slice(), res[key], f"tick {t} link {key}")
            _same(res[key], alone.report(alone.end_slice()), f"tick {t} link {key} (alone)")
            compare_state(o, srv.state_arrays(key), f"tick {t} link {key}")
        # links admitted at this tick: their first slice closed empty; packets come next tick
        for key in res:
            if key not in run and key not in started:
                o, alone = oracle_for(params[key]), srla.Link(params[key], device=cuda_device)
                run[key] = (o, alone)
                started[key] = t
                step[key] = 0
                compare_reports(o.end_slice(), res[key], f"tick {t} link {key} (admitted)")
                _same(res[key], alone.report(alone.end_slice()), f"tick {t} link {key} (admitted, alone)")
        assert admitted == len(res)
        if t == 1:
            assert set(res) == {0, 1} and waiting == 1
    assert started.get(2) == 4 and started.get(3) == 6
    with pytest.raises(srla.SRLAError) as e:  # a departed link has no state
        srv.state_arrays(0)
    assert e.value.code == srla.E_ORDER
    srv.destroy()


def test_served_workload_geometry_matches_oracle(cuda_device):
    """Links of the served workload's identities (synth.served_links: Zipf(1.1) sources, 1-50
    planted hosts, mixed recorder widths and windows), rates scaled down 64x, arriving and
    departing between ticks; each served link against its oracle every tick."""
    import dataclasses

    ident = synth.served_links(24)
    works, params = [], []
    for w, plog in ident:
        t = dataclasses.replace(w.traffic, pkts_per_slice=max(2048, w.traffic.pkts_per_slice // 64),
                                n_planted=max(1, w.traffic.n_planted // 4), planted_card=(1 << 8, 1 << 12))
        w = dataclasses.replace(w, traffic=t)
        works.append(w)
        params.append(srla.params_for(w, *synth.hash_coefficients(w.hash_seed, w.u + 3), pair_slots_log2=plog))
    arena = sum(srla.Group.link_bytes(p) for p in params) + (64 << 20)
    budget = sum(sorted(srla.Group.link_bytes(p) for p in params)[-8:])  # room for about 8 links at once
    srv = srla.Server(max_links=12, max_pkts=1 << 22, budget_bytes=budget, arena_bytes=arena, max_report=1 << 20,
                      device=cuda_device)
    rng = np.random.default_rng(17)
    order = list(range(len(ident)))
    opened, run, step = set(), {}, {}
    for t in range(14):
        for _ in range(2 if t < 10 else 0):  # arrivals
            if order:
                k = order.pop(0)
                srv.open(k, params[k])
                opened.add(k)
        for k in list(run):  # departures
            if rng.random() < 0.15:
                srv.close(k)
                del run[k]
        for k, o in run.items():
            pk = synth.generate_slice(works[k].traffic, step[k])
            step[k] += 1
            assert srv.submit(k, pk.to(cuda_device))
            o.push(synth.pairs_to_numpy(pk))
        sl, admitted, waiting = srv.tick()
        res = srv.poll(sl)
        assert admitted == len(res)
        for k in list(run):
            compare_reports(run[k].end_slice(), res[k], f"tick {t} link {k}")
            if t % 4 == 3:
                compare_state(run[k], srv.state_arrays(k), f"tick {t} link {k}")
        for k in res:
            if k not in run:
                o = oracle_for(params[k])
                compare_reports(o.end_slice(), res[k], f"tick {t} link {k} (admitted)")
                run[k] = o
                step[k] = 0
    assert len(opened) > 12
    srv.destroy()
