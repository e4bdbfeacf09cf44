"""The inline candidate mode (Algorithm 2 as printed, SRLA_MODE_INLINE) on the GPU.

Its candidate lists depend on which packets the parallel threads see first, so they are not
compared element by element.  What is fixed, and checked here against the oracle:

* the recorders (exported distances) and the row census do not depend on the candidate
  rule: bit-exact against the oracle, slice after slice;
* every inline candidate is a candidate of the order-free rule (the union SRE only grows
  within a slice), and gets the same union SLE weight, estimate and super point flag;
* a carried host already has its SI bits, so it is never inserted again (no entry is both
  CARRIED and NEW), also after a checkpoint round trip;
* the inline lists find most of the order-free candidates (here at least 80 %).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import EST_RTOL
from paper_1803_10369_b300 import srla

pytestmark = pytest.mark.gpu

TINY = synth.workload("tiny")
SUPER_SAT = srla.SUPER | srla.SATURATED


def _pair(w):
    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    o = oracle.Oracle.for_workload(w, ha, hb)
    link = srla.Link(srla.params_for(w, ha, hb, mode=srla.MODE_INLINE))
    return o, link


@pytest.mark.parametrize("w", [
    TINY,
    TINY.replace(dr_bytes=2, z=16, k=4, theta=128, seed=12),
    TINY.replace(dr_bytes=0, z=1, k=1, g=8, gl=1024, theta=128, seed=13),
    synth.workload("paper").replace(planted_spread=3, pkts_per_slice=1_000_000, n_slices=4),
], ids=["tiny", "u16-theta128", "bits-discrete", "paper-1M"])
def test_inline_lists_within_order_free_lists(w, cuda_device):
    o, link = _pair(w)
    found = total = 0
    for s in range(w.n_slices):
        pk = synth.generate_slice(w.traffic, s)
        o.push(synth.pairs_to_numpy(pk))
        link.push(pk.to(cuda_device))
        ro = o.end_slice()
        rg = link.report(link.end_slice())
        where = f"{w.name} slice {s}"
        assert np.array_equal(rg["stats"]["census"], ro["cnt"]), where
        pos = {a: x for x, a in enumerate(ro["aip"].tolist())}
        for x, a in enumerate(rg["aip"].tolist()):
            assert a in pos, f"{where}: {a} is not an order-free candidate"
            y = pos[a]
            assert rg["w"][x] == ro["w"][y], where
            assert (rg["flags"][x] & SUPER_SAT) == (ro["flags"][y] & SUPER_SAT), where
            e, eo = float(rg["est"][x]), float(ro["est"][y])
            assert (np.isinf(e) and np.isinf(eo)) or abs(e - eo) <= EST_RTOL * abs(eo), where
            assert not (rg["flags"][x] & srla.CARRIED and rg["flags"][x] & srla.NEW), where
        found += len(rg["aip"])
        total += len(ro["aip"])
        re_g, le_g, T_g, carry_g = link.state_arrays()
        re_o, le_o = o.state()
        assert T_g == o.slice and np.array_equal(re_g, re_o) and np.array_equal(le_g, le_o), where
        assert set(carry_g.tolist()) <= set(o.carry().tolist()), where
    assert total > 0 and found >= 0.8 * total, (found, total)
    link.close()
    o.close()


def test_inline_checkpoint_keeps_carried_hosts_out(cuda_device):
    w = TINY.replace(k=6)
    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    p = srla.params_for(w, ha, hb, mode=srla.MODE_INLINE)
    a = srla.Link(p)
    for s in range(4):
        a.push(synth.generate_slice(w.traffic, s).to(cuda_device))
        a.report(a.end_slice())
    blob = a.export_state()
    b = srla.Link(p)
    b.import_state(blob)
    n_carried = 0
    for s in range(4, 8):
        pk = synth.generate_slice(w.traffic, s).to(cuda_device)
        for link in (a, b):
            link.push(pk)
            r = link.report(link.end_slice())
            f = r["flags"]
            assert not np.any((f & srla.CARRIED) & ((f & srla.NEW) >> 1)), s
            n_carried += int(np.count_nonzero(f & srla.CARRIED))
    assert n_carried > 0
    a.close()
    b.close()
