"""kl_diag_noalloc: the diagnostics for callers that may not allocate GPU
memory while they run (an application that reserves its device memory up
front and owns the allocator, or a time loop that cannot take cudaMalloc's
synchronisation between steps).  It uses a static device array instead of
library allocations; its results must equal kl_diag's, call after call.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""

from __future__ import annotations

import numpy as np
import pytest

from gpu_cases import make_inputs, run_gpu

pytestmark = pytest.mark.gpu


def _compare(got, want, t):
    assert got[0] == want[0] and got[2] == want[2]
    for c in (1, 3):
        assert got[c] == pytest.approx(want[c], rel=1e-12)
    scale = np.abs(t).sum()
    for c in (4, 5):
        assert abs(got[c] - want[c]) <= 1e-12 * scale


def test_noalloc_diag_matches_kl_diag_on_consecutive_calls():
    import torch
    from paper_2303_12374_gb300 import kl
    ctx = kl.kl_create(0, None)
    try:
        # two different grids in a row: the second uses fewer scratch records
        # than the first, so leftovers of the first call would show
        for (nx, ny, nz), dtype in (((96, 80, 40), 1), ((33, 21, 12), 0)):
            f = make_inputs(nx, ny, nz, seed=nx, walls=True)
            p, _, outs, _ = run_gpu(ctx, f, adv=5, diff=1, dtype=dtype, walls=True, g=3)
            t = p.download(outs["ut"])
            ref = t + np.random.default_rng(nx).standard_normal(t.shape) * 1e-3
            ref_buf = p.upload(ref, dtype=torch.float64)
            wz = torch.full((nz,), 1.0 / nz, dtype=torch.float64, device="cuda")
            want = kl.kl_diag(ctx, p.dtype, p.grid, 0, outs["ut"].data_ptr(), ref_buf.data_ptr())
            for _ in range(2):
                got = kl.kl_diag_noalloc(p.dtype, p.grid, outs["ut"].data_ptr(),
                                         ref_buf.data_ptr(), wz.data_ptr())
                _compare(got, want, t)
            # without weights out[5] is the plain sum
            got = kl.kl_diag_noalloc(p.dtype, p.grid, outs["ut"].data_ptr(), None, None)
            assert got[3] == 0.0 and got[2] == 0.0
            assert abs(got[5] - got[4]) <= 1e-12 * np.abs(t).sum()
            assert abs(got[4] - want[4]) <= 1e-12 * np.abs(t).sum()
    finally:
        kl.kl_destroy(ctx)


def test_noalloc_diag_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    p = Problem(1024, 1024, 65, g=3, dtype="f32", walls=True, dz=1.0 / 65, device="cuda")
    small = torch.zeros(16, device="cuda")
    with pytest.raises(kl.KLError) as e:
        kl.kl_diag_noalloc(p.dtype, p.grid, small.data_ptr(), None, None)
    assert e.value.status == -1 and "static scratch" in str(e.value)
