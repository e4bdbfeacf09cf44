"""Parity at the full sizes of the benchmarked workloads, in the launch configuration the
benchmark uses (same handle parameters, device-resident batches of a whole slice).

The oracle replays every slice from an empty array, so these runs are a few slices long;
planted hosts spread their destinations over a few slices so that candidate lists, carries
and estimates are all exercised.  The steady-state benchmark runs the same kernels.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import compare_reports, compare_state, make_pair

pytestmark = pytest.mark.gpu


def _run(w, slices, cuda_device, first_trace_slice=0, state_every=1):
    o, link = make_pair(w)
    n_cand = 0
    for i, s in enumerate(range(first_trace_slice, first_trace_slice + slices)):
        pk = synth.generate_slice(w.traffic, s, device=cuda_device)
        o.push(synth.pairs_to_numpy(pk))
        link.push(pk)
        ro = o.end_slice()
        rg = link.report(link.end_slice())
        compare_reports(ro, rg, f"{w.name} slice {s}")
        n_cand = max(n_cand, ro["n_candidates"])
        if (i + 1) % state_every == 0:
            compare_state(o, link, f"{w.name} slice {s}")
    link.close()
    o.close()
    return n_cand


def test_paper_scale_sizes(cuda_device):
    """u=8, v=2^14, g=128, g'=256, 16-bit recorders, k=300, 5M packets per slice."""
    w = synth.workload("paper").replace(planted_spread=3)
    n_cand = _run(w, 4, cuda_device)
    assert n_cand >= 100


def test_long_window_flood_and_stamp_wraparound(cuda_device):
    """k=1024, 2M packets per slice with a heavy source and the spoofed-source flood, starting
    8 slices before the 16-bit stamps wrap."""
    w = synth.workload("longwin").replace(planted_spread=3)
    _run(w, 3, cuda_device, first_trace_slice=4, state_every=3)


def test_paper_scale_flow_bursts(cuda_device):
    """Paper-scale traffic sent in bursts of the same pair (geometric, mean 8 packets): warps
    meet runs of one pair, which the scan's duplicate elision must skip without losing any."""
    w = synth.workload("burst").replace(planted_spread=3)
    n_cand = _run(w, 3, cuda_device, state_every=3)
    assert n_cand >= 100


def test_paper_scale_uniform_destinations(cuda_device):
    """The literal uniform-destination reading of the paper-scale traffic (saturating)."""
    w = synth.workload("paper").replace(dst_model="uniform", dst_space=1 << 20, planted_spread=3,
                                        pkts_per_slice=2_000_000)
    _run(w, 2, cuda_device, state_every=2)


def test_paper_own_parameters(cuda_device):
    """The paper's own parameters: u=4, v=65536, g=8 (tau=7, ceil(rho*g)=3), g'=1024, 16-bit
    recorders (512 MiB of SLE), k=300, 4.5M packets per slice."""
    w = synth.workload("paperown").replace(planted_spread=3)
    n_cand = _run(w, 4, cuda_device, state_every=2)
    assert n_cand >= 100


def test_discrete_window_one_bit_recorders(cuda_device):
    """The discrete window (z=1, k=1) at the paper's own sketch sizes with one-bit recorders:
    every slice starts from empty recorders and nothing is carried."""
    w = synth.workload("discrete")
    n_cand = _run(w, 3, cuda_device, state_every=1)
    assert n_cand >= 40
