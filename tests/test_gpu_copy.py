"""kl_copy_in / kl_copy_out through the C ABI: a contiguous host array moves
to and from the interior of a padded device field bit for bit, every ghost
cell keeps its value, for every storage type, from page-locked and pageable
host memory, on the recommended layout (one 3D copy) and on a layout whose
plane pitch is not a whole number of rows (one 2D copy per level)."""

from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu

TORCH_DT = {0: "float64", 1: "float32", 2: "bfloat16", 3: "float16"}


def _grid(nx, ny, nz, g, dtype, odd_pitch):
    from paper_2303_12374_gb300 import kl
    if odd_pitch:
        sj = nx + 2 * g + 5
        sk = sj * (ny + 2 * g) + 7                 # not a multiple of sj
        origin = g * (1 + sj + sk)
        extent = sk * (nz + 2 * g)
    else:
        sj, sk, origin, extent = kl.kl_layout(nx, ny, nz, g, dtype)
    return kl.Grid(nx, ny, nz, g, sj, sk, origin, extent, 1, 0, 1.0 / nx, 1.0 / ny, 1.0 / nz,
                   1e-3, None)


@pytest.mark.parametrize("dtype", [0, 1, 2, 3])
@pytest.mark.parametrize("odd_pitch", [False, True])
@pytest.mark.parametrize("pinned", [True, False])
def test_copy_in_out_interior_bit_exact(dtype, odd_pitch, pinned):
    import torch
    from paper_2303_12374_gb300 import kl
    nx, ny, nz, g = 37, 21, 11, 3
    grid = _grid(nx, ny, nz, g, dtype, odd_pitch)
    tdt = getattr(torch, TORCH_DT[dtype])
    gen = torch.Generator().manual_seed(40 + dtype)
    host = torch.randn((nz, ny, nx), generator=gen).to(tdt)
    if pinned:
        host = host.pin_memory()
    dev = torch.full((grid.extent,), -7.0, dtype=tdt, device="cuda")
    stream = torch.cuda.Stream()
    kl.kl_copy_in(dtype, grid, host.data_ptr(), dev.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    view = dev.as_strided((nz, ny, nx), (grid.sk, grid.sj, 1), grid.origin)
    ibits = torch.int64 if dtype == 0 else torch.int32 if dtype == 1 else torch.int16
    assert torch.equal(view.cpu().view(ibits), host.view(ibits))
    # ghosts and padding untouched: exactly nx*ny*nz elements changed
    assert int((dev != -7.0).sum()) <= nx * ny * nz
    mask = torch.ones(grid.extent, dtype=torch.bool, device="cuda")
    mask.as_strided((nz, ny, nx), (grid.sk, grid.sj, 1), grid.origin).fill_(False)
    assert bool((dev[mask] == -7.0).all())
    out = torch.zeros((nz, ny, nx), dtype=tdt)
    if pinned:
        out = out.pin_memory()
    kl.kl_copy_out(dtype, grid, dev.data_ptr(), out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    assert torch.equal(out.view(ibits), host.view(ibits))
