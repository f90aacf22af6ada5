"""Brownian disks on the GPU: equipartition with the fluctuating fluid (Sec. 3
with Sec. 4), the statement the oracle is pinned to on the CPU, here with far
more samples.

Thirty-two independent 64 x 64 periodic domains (one launch per step), nine
neutrally buoyant R = 5 disks in each, kT = 1e-5, shifted FP32 store.  Each
translational component must give M<U^2>/kT = 1 - M/M_tot (the finite-box
factor of exact momentum conservation between the disks and the exterior
fluid) and I<Omega^2>/kT = 1, within 2 %, with a 95 % interval from block means
(blocks of 1,000 steps of one domain, treated as independent) below 1 %.
"""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_params
from paper_2006_12910_gb300 import lbm

pytestmark = pytest.mark.gpu

L, R, KT, NSIDE, NDOM = 64, 5.0, 1e-5, 3, 32
BURN, STEPS, EVERY = 2000, 20000, 10


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_brownian_disks_in_equipartition(tau, errlog):
    parts = [dict(x=(a + 0.5) * L / NSIDE + 0.37, y=(b + 0.5) * L / NSIDE + 0.21, R=R, rho_p=1.0)
             for a in range(NSIDE) for b in range(NSIDE)]
    ps = [gpu_params(dict(nx=L, ny=L, periodic_x=1, periodic_y=1, walls_y=0, tau=tau, kT=KT,
                          seed=9000 + d, domain_id=d), "f32s", len(parts)) for d in range(NDOM)]
    ctx = lbm.Context(ps, particles=[parts] * NDOM)
    ctx.step(BURN)
    n = STEPS // EVERY
    X = np.zeros((n, NDOM, len(parts), 3))
    for s in range(n):
        ctx.step(EVERY)
        for d in range(NDOM):
            X[s, d] = ctx.particles_array(dom=d)[:, 4:7]
    ctx.sync()
    M = math.pi * R * R
    I = 0.5 * M * R * R
    box = 1.0 - M / (L * L)  # disks of the fluid's density: M_tot is the box's mass
    u2 = M * 0.5 * (X[..., 0] ** 2 + X[..., 1] ** 2) / KT / box
    o2 = I * X[..., 2] ** 2 / KT
    blk = 1000 // EVERY

    def stats(v):
        m = v[: (n // blk) * blk].reshape(n // blk, blk, NDOM, -1).mean(axis=(1, 3)).ravel()
        return float(m.mean()), float(1.96 * m.std(ddof=1) / math.sqrt(m.size))

    tu, cu = stats(u2)
    tr, cr = stats(o2)
    errlog(tau=tau, M_U2_over_kT_box=tu, ci=cu, I_O2_over_kT=tr, ci_rot=cr)
    assert cu < 0.01 and cr < 0.01, (cu, cr)
    assert abs(tu - 1.0) < 0.02, (tu, cu)
    assert abs(tr - 1.0) < 0.02, (tr, cr)
