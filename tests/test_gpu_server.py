"""The serving loop: links arrive, wait for admission under a byte budget, run, and depart;
every admitted link's results, slice by slice, equal those of the same link run alone from
its admission on (same batches, pushed in several pieces), whatever else is in the mix."""
import numpy as np
import pytest

import synth
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


def test_served_links_equal_links_alone(cuda_device):
    works = [TINY.replace(seed=40 + i, pkts_per_slice=20_000 + 5_000 * i, k=3 + i, start_slice=10 * i)
             for i in range(4)]
    params = []
    for i, w in enumerate(works):
        ha, hb = synth.hash_coefficients(300 + i, w.u + 3)
        params.append(srla.params_for(w, ha, hb, pair_slots_log2=12))
    one = srla.Group.link_bytes(params[0])
    srv = srla.Server(max_links=4, max_pkts=1 << 20, budget_bytes=2 * one + (1 << 20), arena_bytes=4 * one + (16 << 20))
    solo, started, step = {}, {}, {}
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
        for key in list(solo):
            pk = synth.generate_slice(works[key].traffic, step[key]).to(cuda_device)
            step[key] += 1
            cuts = np.sort(rng.integers(0, pk.shape[0], size=3))
            pieces = np.split(np.arange(pk.shape[0]), cuts)
            for pc in pieces:  # several submits of uneven sizes
                if pc.size:
                    assert srv.submit(key, pk[pc[0]:pc[-1] + 1])
            solo[key].push(pk)
        sl, admitted, waiting = srv.tick()
        res = srv.poll(sl)
        for key in list(solo):
            if key in (0,) and t >= 4 or key == 1 and t >= 6:
                assert key not in res
                del solo[key]
                continue
            _same(res[key], solo[key].report(solo[key].end_slice()), f"tick {t} link {key}")
        # links admitted at this tick start their solo twin now (their first packets come next tick)
        for key in res:
            if key not in solo and key not in started:
                solo[key] = srla.Link(params[key], device=cuda_device)
                started[key] = t
                step[key] = 0
                want = solo[key].report(solo[key].end_slice())  # an empty first slice, as in the server
                _same(res[key], want, f"tick {t} link {key} (admitted)")
        assert admitted == len(res)
        if t == 1:
            assert set(res) == {0, 1} and waiting == 1
    assert started.get(2) == 4 and started.get(3) == 6
    srv.destroy()
