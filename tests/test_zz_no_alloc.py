"""The allocation-free entry point (srla_batch_report_static) against the workspace path.

Callers that cannot allocate device memory (real-time capture threads, for which cudaMalloc
and cudaFree may stall the whole device, and plugins that only get fixed buffers from their
host framework) use one fixed scratch array compiled into the library.  Its report for a device batch must equal what a
freshly created estimator reports after pushing that batch and closing its first slice.
Two calls in a row check that the shared scratch is cleared between calls.  This file sorts
last so that a failure here does not hide the rest of the suite.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import EST_RTOL
from paper_1803_10369_b300 import srla

pytestmark = pytest.mark.gpu


def _same(a, b, where):
    assert a["aip"].tolist() == b["aip"].tolist(), where
    assert np.array_equal(a["w"], b["w"]) and np.array_equal(a["flags"], b["flags"]), where
    ea, eb = a["est"].astype(np.float64), b["est"].astype(np.float64)
    assert np.array_equal(np.isinf(ea), np.isinf(eb)), where
    fin = ~np.isinf(eb)
    assert (np.abs(ea[fin] - eb[fin]) <= EST_RTOL * np.abs(eb[fin])).all(), where
    for key in ("n_sampled", "n_new", "n_candidates", "n_carry_out", "w_star", "overflow", "n_pkts"):
        assert a["stats"][key] == b["stats"][key], (where, key)
    assert np.array_equal(a["stats"]["census"], b["stats"]["census"]), where


@pytest.mark.parametrize("variant", ["tiny", "tiny-2byte-theta128"])
def test_static_scratch_report_matches_workspace_path(variant, cuda_device):
    w = synth.workload("tiny")
    if variant != "tiny":
        w = w.replace(dr_bytes=2, z=16, k=8, theta=128)
    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    params = srla.params_for(w, ha, hb)
    for call in range(2):  # two calls in a row, different batches
        pk = synth.generate_slice(w.traffic, 3 + call, device=cuda_device)
        got = srla.batch_report_static(params, pk)
        link = srla.Link(params, device=cuda_device)
        link.push(pk)
        want = link.report(link.end_slice())
        link.close()
        assert want["stats"]["n_candidates"] > 0
        _same(got, want, f"{variant} call {call}")


def test_static_scratch_rejects_oversized_parameters(cuda_device):
    import torch

    w = synth.workload("paper")
    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    params = srla.params_for(w, ha, hb)
    assert srla.workspace_bytes(params) > srla.STATIC_SCRATCH_BYTES
    pk = torch.zeros((16, 2), dtype=torch.int32, device=cuda_device)
    with pytest.raises(srla.SRLAError) as e:
        srla.batch_report_static(params, pk)
    assert e.value.code == srla.E_NOMEM


def test_static_scratch_refuses_a_capturing_stream(cuda_device):
    """The call synchronizes its stream, so on a stream being captured it returns INVAL
    before any other CUDA call; the capture stays intact (its graph replays)."""
    import torch

    w = synth.workload("tiny")
    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    params = srla.params_for(w, ha, hb)
    pk = synth.generate_slice(w.traffic, 0, device=cuda_device)
    # a first call outside any capture (the library's device code and scratch array are
    # loaded by then), which works
    assert srla.batch_report_static(params, pk)["stats"]["n_pkts"] == pk.shape[0]
    x = torch.zeros(4, device=cuda_device)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(cuda_device)
    torch.cuda.synchronize(cuda_device)
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        with pytest.raises(srla.SRLAError) as e:
            srla.batch_report_static(params, pk, stream=side)
        assert e.value.code == srla.E_INVAL
    graph.replay()
    torch.cuda.synchronize(cuda_device)
    assert x.tolist() == [1.0] * 4
    # and after the capture it works again
    assert srla.batch_report_static(params, pk)["stats"]["n_pkts"] == pk.shape[0]
