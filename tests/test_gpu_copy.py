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


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_host_to_host_step_matches_oracle(oracle_mod, dtype):
    """The path a caller with host data takes (and the bench's e2e times):
    kl_copy_in of u, v, w from pinned host arrays, kl_step, kl_copy_out of
    ut, vt, wt, all on one stream; the host results equal the oracle's."""
    import torch
    from gpu_cases import TOL, make_inputs, oracle_ref, rel_err
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    nx, ny, nz = 70, 45, 23
    f = make_inputs(nx, ny, nz, seed=77, walls=True, stretch=2.0)
    p = Problem(nx, ny, nz, g=3, dtype=dtype, walls=True, zh=f["zh"], nu=1e-3)
    ctx = kl.kl_create(0, None)
    try:
        host_in = [torch.from_numpy(f[k].copy()).to(p.tdtype).pin_memory() for k in ("u", "v", "w")]
        host_out = [torch.empty((nz, ny, nx), dtype=p.tdtype).pin_memory() for _ in range(3)]
        dev_in = [p.empty() for _ in range(3)]
        dev_out = [p.empty() for _ in range(3)]
        s = torch.cuda.Stream()
        for h, d in zip(host_in, dev_in):
            kl.kl_copy_in(p.dtype, p.grid, h.data_ptr(), d.data_ptr(), s.cuda_stream)
        fl = kl.Fields(*[d.data_ptr() for d in dev_in], None, *[d.data_ptr() for d in dev_out])
        kl.kl_step(ctx, kl.Op(5, 1, p.dtype, 0), p.grid, fl, s.cuda_stream)
        for h, d in zip(host_out, dev_out):
            kl.kl_copy_out(p.dtype, p.grid, d.data_ptr(), h.data_ptr(), s.cuda_stream)
        s.synchronize()
        kl.kl_check(ctx)
        rin = {k: p.rounded(f[k]) for k in ("u", "v", "w")}
        ref = oracle_ref(oracle_mod, rin, f["zh"], adv=5, diff=1, walls=True, g=3)
        for h, r in zip(host_out, ref):
            got = h.to(torch.float64).numpy()
            assert rel_err(got, r) <= TOL[dtype]
    finally:
        kl.kl_destroy(ctx)
