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


@pytest.mark.parametrize("cell_bytes", [1, 2, 4])
@pytest.mark.parametrize("policy", [srla.PROBE_ATOMIC_MAX, srla.PROBE_READ_FIRST])
def test_store_probe_policies_write_the_same_value(policy, cell_bytes, cuda_device):
    """Every policy leaves each touched cell holding the probe's value (seed | 1); the atomic
    maximum keeps larger values already present, and its CAS loop leaves the neighbouring
    cells of the same 32-bit word alone."""
    import torch

    dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[cell_bytes]
    n_cells = (1 << 16) // cell_bytes
    buf = torch.zeros(n_cells, dtype=dt, device=cuda_device)
    big = torch.arange(n_cells, device=cuda_device) % 7 == 0
    buf[big] = 100                              # larger than the value written below
    seed = 4                                    # the probe writes seed | 1 = 5
    srla.scatter_probe(buf, cell_bytes, 8 * n_cells, seed=seed, policy=policy)
    torch.cuda.synchronize(cuda_device)
    touched = buf != 0
    assert int(touched.sum()) > 0.99 * n_cells  # 8 writes per cell on average
    if policy == srla.PROBE_ATOMIC_MAX:
        assert bool((buf[big] == 100).all())
        rest = buf[~big]
        assert bool(((rest == 5) | (rest == 0)).all())
    else:  # a cell that differs is overwritten, 100 included; about e^-8 of the cells get no write
        assert bool(((buf == 5) | (buf == 0) | (big & (buf == 100))).all())
        assert float((buf[big] == 5).float().mean()) > 0.99
