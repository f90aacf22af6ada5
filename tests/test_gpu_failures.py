"""Failure detection on the GPU without a GPU fault.

- A bounded device wait that runs out: the staged stream-and-collide kernel
  waits for its bulk copies at most the context's wait limit.  With the limit
  set to 0 every stage wait reports expiry at once; the kernel records
  LBM_E_TIMEOUT, drains the copies it had issued (with the full one-second
  limit, so every copy lands before the CTA leaves) and ends its work.  The
  next blocking call returns LBM_E_TIMEOUT; once the limit is restored and the
  state replaced, the context steps normally again and matches the oracle.
- A device allocation that fails (injected on the host): creation returns
  LBM_E_NOMEM at every allocation point and frees what it had allocated.
"""
import gc

import numpy as np
import pytest

from gpu_helpers import assert_close, compare_state, gpu_params, pair
from paper_2006_12910_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_stage_wait_timeout_is_reported_and_the_context_recovers(errlog):
    nx, ny = 200, 48
    solid = workloads.disk_mask(nx, ny, [(60.3, 20.1, 6.5)])
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=1e-5)
    f0 = workloads.random_populations(nx, ny, seed=4242, amp=0.01, solid=solid)
    ref, ctx = pair(base, "f32s", solid=solid, f0=f0)
    ctx.set_launch(2, 64, 2)  # the staged kernel: bulk copies behind bounded mbarrier waits
    ctx.set_wait_limit(0)
    ctx.step(3)
    with pytest.raises(lbm.LbmError) as ei:
        ctx.sync()
    assert ei.value.code == -5
    # sticky until the state is replaced
    with pytest.raises(lbm.LbmError) as ei:
        ctx.sync()
    assert ei.value.code == -5
    ctx.set_wait_limit(10 ** 9)
    ctx.set_populations(f0)
    ctx.sync()
    ctx.step(40)
    ref.step(40)
    errs, tols = compare_state(ref, ctx, "f32s", solid)
    errlog(**errs)
    assert_close(errs, tols, "after recovery")


def test_failed_device_allocation_returns_nomem_and_frees_everything():
    torch = pytest.importorskip("torch")
    base = dict(nx=512, ny=512, periodic_x=1, periodic_y=1, walls_y=0, tau=0.8, lj_psi=1e-4, lj_rit=2.5)
    parts = [dict(x=100.3, y=200.2, R=6.0, rho_p=1.1), dict(x=300.7, y=80.4, R=8.0, rho_p=1.0)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    codes = []
    try:
        for nth in range(1, 200):
            lbm.debug_fail_alloc(nth)
            try:
                ctx = lbm.Context(gpu_params(base, "f32s", len(parts)), particles=[parts])
                ctx.step(2)
                ctx.sync()
            except lbm.LbmError as e:
                codes.append(e.code)
            else:
                ctx.close()
                break  # every allocation point of creation, particles and the first steps was hit
    finally:
        lbm.debug_fail_alloc(0)
    gc.collect()  # contexts whose particle allocation failed are destroyed with their Python objects
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # each of the failed calls would leak at least one 9.4 MB population arena
    assert len(codes) >= 10 and all(c == -2 for c in codes), codes
    assert free0 - free1 < (8 << 20), (free0 - free1)
    # and the hook is off again: a normal context works
    ctx = lbm.Context(gpu_params(base, "f32s", len(parts)), particles=[parts])
    ctx.step(4)
    ctx.sync()
    assert np.isfinite(ctx.checks()).all()
    ctx.close()
