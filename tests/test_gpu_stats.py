"""Equilibrium statistics of the fluctuating LB on the GPU (Sec. 4, Eqs. NP1-NP2).

Linear fluctuating-LB theory (every non-conserved mode thermalised with
omega (2 - omega)) gives, per node, <m_k^2> = rho0 kT / c_s^2 = 3 kT for the
density, the two momentum components and the six kinetic modes of Table 1.
The oracle is pinned to the same statement on the CPU; here the CUDA path
(shifted FP32 and FP16 stores, one domain and a batch of uneven domains with
their own seeds and temperatures) must meet it within the same 2 %.
"""
import numpy as np
import pytest

from gpu_helpers import gpu_params
from oracle import oracle
from paper_2006_12910_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def mode_ratios(ctx, chi, kT, rho0=1.0, dom=0, thermalise=500, samples=400, every=10):
    ctx.step(thermalise)
    acc = []
    for _ in range(samples):
        ctx.step(every)
        f = ctx.populations(dom=dom).reshape(9, -1)
        m = chi @ f
        acc.append(np.concatenate([[((f.sum(0) - rho0) ** 2).mean()], (m[1:] ** 2).mean(1)]))
    return np.mean(acc, axis=0) / (3 * kT)


@pytest.mark.parametrize("store", ["f32s", "f16s"])
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_equipartition_every_mode_on_gpu(store, tau, errlog):
    chi, _ = oracle.basis()
    N, kT = 32, 1e-4
    base = dict(nx=N, ny=N, periodic_x=1, periodic_y=1, walls_y=0, tau=tau, kT=kT, seed=1234)
    ctx = lbm.Context(gpu_params(base, store))
    ratio = mode_ratios(ctx, chi, kT)
    errlog(store=store, tau=tau, ratios=ratio.tolist())
    assert np.abs(ratio - 1).max() < 0.02, ratio


def test_equipartition_in_uneven_ensemble(errlog):
    """Six domains of different sizes, seeds and temperatures stepped together:
    each thermalises to its own kT (domains draw independent noise)."""
    chi, _ = oracle.basis()
    sizes = [(32, 32), (48, 32), (32, 40), (40, 40), (64, 32), (32, 64)]
    kts = [5e-5, 1e-4, 2e-4, 8e-5, 1.5e-4, 1.2e-4]
    ps = [gpu_params(dict(nx=nx, ny=ny, periodic_x=1, periodic_y=1, walls_y=0, tau=1.0, kT=kT, seed=77 + d,
                          domain_id=d), "f32s")
          for d, ((nx, ny), kT) in enumerate(zip(sizes, kts))]
    ctx = lbm.Context(ps)
    ctx.step(500)
    acc = [[] for _ in sizes]
    for _ in range(300):
        ctx.step(10)
        for d in range(len(sizes)):
            f = ctx.populations(dom=d).reshape(9, -1)
            m = chi @ f
            acc[d].append(np.concatenate([[((f.sum(0) - 1.0) ** 2).mean()], (m[1:] ** 2).mean(1)]))
    # every mode of every domain: nodes x samples of each domain give the same
    # statistical weight as the single-domain test (32 x 32 x 400) or more
    for d, kT in enumerate(kts):
        ratio = np.mean(acc[d], axis=0) / (3 * kT)
        errlog(dom=d, kT=kT, ratios=ratio.tolist())
        n_eff = sizes[d][0] * sizes[d][1] * 300
        tol = 0.02 * np.sqrt(32 * 32 * 400 / n_eff) if n_eff < 32 * 32 * 400 else 0.02
        assert np.abs(ratio - 1).max() < max(tol, 0.02), (d, ratio)
