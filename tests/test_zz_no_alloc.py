"""The allocation-free binning entry point against the allocating one.

sph_bin_sort_noalloc serves callers that cannot allocate device memory while
they run (their memory belongs to another framework's pool, or an
allocation's failure or synchronisation is not acceptable mid-loop).  It
keeps its scratch in one fixed array inside the library; here two calls in a
row, on different inputs, must give exactly the outputs of sph_bin_sort
(integer results: bit-exact), and an input too large for the fixed scratch
must be refused.  This file is collected last so that a stopping run has
already run every other test.
"""
import numpy as np
import pytest

from paper_2110_02621_gb300 import build, sph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    sph.lib()
    return torch


def _bin(torch, fn, x, lo, h, dims):
    dev = torch.device("cuda")
    n = len(x)
    n_cells = int(np.prod(dims))
    xd = torch.tensor(x, dtype=torch.float64, device=dev)
    key = torch.full((max(n, 1),), -7, dtype=torch.int32, device=dev)
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device=dev)
    start = torch.full((n_cells + 1,), -7, dtype=torch.int32, device=dev)
    st = fn(xd.data_ptr(), n, lo, h, dims, key.data_ptr(), order.data_ptr(), start.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, key.cpu().numpy()[:n], order.cpu().numpy()[:n], start.cpu().numpy()


def test_noalloc_matches_allocating_binning_twice(torch_cuda):
    torch = torch_cuda
    h = 0.013
    cs = 2 * h
    rng = np.random.default_rng(2110)
    # the first two grids (6,552 and 2,744 cells) take the one-block scan; the
    # third (98 x 78 x 73 = 558,012 cells, more than 512 blocks of 1,024) the
    # reduce / scan-of-sums / down-sweep kernels and the block-sums part of the
    # fixed scratch
    inputs = [rng.uniform(0, 1, (30011, 3)) * [0.6, 0.4, 0.3],
              rng.integers(0, 12, (9001, 3)) * cs + rng.uniform(0, cs, (9001, 3)) * (rng.uniform(size=(9001, 1)) < 0.5),
              rng.uniform(0, 1, (200003, 3)) * [96 * cs, 76 * cs, 71 * cs]]
    for x in inputs:  # calls in a row: each reuses the scratch of the one before
        lo = (0.0, 0.0, 0.0)
        dims = tuple(int(np.ceil((x[:, d].max() + 2 * cs) / cs)) for d in range(3))
        assert int(np.prod(dims)) in (6552, 2744, 558012)
        ref = _bin(torch, sph.sph_bin_sort, x, lo, h, dims)
        got = _bin(torch, sph.sph_bin_sort_noalloc, x, lo, h, dims)
        assert ref[0] == sph.SPH_OK and got[0] == sph.SPH_OK
        for a, b in zip(ref[1:], got[1:]):
            assert np.array_equal(a, b)


def test_noalloc_refuses_inputs_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    # valid (small) device buffers: the call must refuse before touching them
    buf = torch.zeros(1024, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    n = sph.SPH_BIN_SORT_NOALLOC_SCRATCH // 32 + 1  # more particles than the scratch holds
    assert sph.sph_bin_sort_noalloc(p, n, (0.0, 0.0, 0.0), 0.013, (4, 4, 4), p, p, p, stream) \
        == sph.SPH_ERR_CAPACITY
    # too many grid cells for the scratch
    assert sph.sph_bin_sort_noalloc(p, 10, (0.0, 0.0, 0.0), 0.013, (400, 400, 40), p, p, p, stream) \
        == sph.SPH_ERR_CAPACITY
    torch.cuda.synchronize()
    assert torch.count_nonzero(buf).item() == 0
