"""Failure detection on the GPU without a fault: every device wait of the
kernels is bounded.  With a one-cycle limit the waits for TMA planes give up,
the CTAs record the time-out in the context's status word, drain their copies
in flight and return; kl_check reports KL_ERR_TIMEOUT and the same context,
with the default limit back, computes correct tendencies again."""

from __future__ import annotations

import numpy as np
import pytest

from gpu_cases import TOL, make_inputs, oracle_ref, rel_err, run_gpu

pytestmark = pytest.mark.gpu

KL_ERR_TIMEOUT = -8


@pytest.mark.parametrize("config,diff", [("zpack:w=4,ly=2,kc=8,ns=8,minb=1", 1),
                                         ("zpack:w=4,ly=2,kc=8,ns=8,minb=1", 2),
                                         ("zmarch:bx=32,by=4,px=1,py=2,kc=8,ns=8,minb=1", 1)])
def test_wait_gives_up_then_context_recovers(oracle_mod, config, diff):
    from paper_2303_12374_gb300 import kl
    f = make_inputs(80, 24, 16, seed=41, walls=True, var_nu=diff == 2)
    ctx = kl.kl_create(0, None)
    try:
        kl.kl_check(ctx)                                   # clean start
        kl.kl_set_wait_limit(ctx, 1)
        run_gpu(ctx, f, adv=5, diff=diff, dtype=1, walls=True, g=3, config=config)
        with pytest.raises(kl.KLError) as e:
            kl.kl_check(ctx)
        assert e.value.status == KL_ERR_TIMEOUT
        kl.kl_check(ctx)                                   # the check cleared the word
        kl.kl_set_wait_limit(ctx, 0)
        p, _, outs, rin = run_gpu(ctx, f, adv=5, diff=diff, dtype=1, walls=True, g=3,
                                  config=config)
        kl.kl_check(ctx)
        ref = oracle_ref(oracle_mod, rin, f["zh"], adv=5, diff=diff, walls=True, g=3)
        for name, r in zip(("ut", "vt", "wt"), ref):
            assert rel_err(p.download(outs[name]), r) <= TOL[1]
    finally:
        kl.kl_destroy(ctx)


def test_wait_limit_rejects_negative():
    from paper_2303_12374_gb300 import kl
    ctx = kl.kl_create(0, None)
    try:
        with pytest.raises(kl.KLError):
            kl.kl_set_wait_limit(ctx, -1)
    finally:
        kl.kl_destroy(ctx)
