"""Failure detection without a GPU fault: every device-side wait of the library is bounded.

The cooperative candidate sort meets at grid barriers; a block that never arrives must not
hang the GPU.  The self-test launches blocks on the same barrier code with some blocks that
never join (a flag that nothing sets): the waiting blocks give up after a bounded number of
polls and the host reads SRLA_E_TIMEOUT; the context stays usable (a link created afterwards
still matches the oracle)."""
import pytest

import synth
from gpu_helpers import compare_reports, make_pair
from paper_1803_10369_b300 import srla

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("blocks,absent", [(2, 1), (8, 3), (64, 1)])
def test_barrier_wait_gives_up(blocks, absent, cuda_device):
    assert srla.wait_selftest(blocks=blocks, absent=absent, spin_limit=2000, device=cuda_device) == srla.E_TIMEOUT


def test_barrier_completes_when_all_arrive(cuda_device):
    assert srla.wait_selftest(blocks=16, absent=0, spin_limit=1 << 20, device=cuda_device) == srla.OK


def test_context_usable_after_a_timeout(cuda_device):
    assert srla.wait_selftest(blocks=4, absent=2, spin_limit=1000, device=cuda_device) == srla.E_TIMEOUT
    w = synth.workload("tiny").replace(n_slices=3)
    o, link = make_pair(w)
    for s in range(w.n_slices):
        pk = synth.generate_slice(w.traffic, s)
        o.push(synth.pairs_to_numpy(pk))
        link.push(pk.to(cuda_device))
        compare_reports(o.end_slice(), link.report(link.end_slice()), f"slice {s}")
    link.close()
    o.close()


def test_store_probe_writes_the_footprint(cuda_device):
    import torch

    buf = torch.zeros(1 << 16, dtype=torch.uint8, device=cuda_device)
    srla.scatter_probe(buf, 2, 1 << 18, seed=3)
    torch.cuda.synchronize(cuda_device)
    cells = buf.view(torch.int16)
    assert int((cells != 0).sum()) > 0.9 * cells.numel()  # 8 stores per cell on average
