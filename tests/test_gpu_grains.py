"""The shape of the paper's first benchmark on the GPU (Sec. 6 benchmark 1): a
1620 x 1020 channel of seeded disk grains, periodic along the flow and walled
across it, a Newtonian fluid driven by a diagonal body force, and 45 disks of
radius 6.5 released in two closely packed arrays near the inlet (LJ-type
repulsion of Eq. MP2 between disks and against grains and walls).  Compared
with the FP64 oracle on the same inputs: a narrower copy with the FP64 store
to round-off, the full size with the shifted FP32 store."""
import numpy as np
import pytest

from gpu_helpers import assert_close, compare_state, gpu_params, oracle_params
from oracle import oracle
from paper_2006_12910_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def grains_pair(store, **kw):
    w = workloads.grains(**kw)
    base = dict(nx=w.nx, ny=w.ny, **w.params)
    f0 = np.empty((9, w.ny, w.nx))
    f0[:] = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    ref = oracle.Domain(oracle_params(base), solid=w.solid, particles=w.particles, f0=f0)
    ctx = lbm.Context(gpu_params(base, store, len(w.particles)), solids=[w.solid], particles=[w.particles])
    ctx.set_populations(f0)
    return w, ref, ctx


def test_grains_fp64_parity(errlog):
    w, ref, ctx = grains_pair("f64", nx=540, ny=340, n_obstacles=26)
    assert len(w.particles) >= 20 and w.solid.any()
    oracle.set_threads(0)
    ref.step(30)
    ctx.step(30)
    fluid = w.solid == 0
    fr, fg = ref.populations(), ctx.populations()
    err = float(np.abs(fg - fr)[:, fluid].max() / np.abs(fr[:, fluid]).max())
    perr = max(abs(a[k] - b[k]) for a, b in zip(ref.particles(), ctx.particles()) for k in ("x", "y", "U", "V", "Omega"))
    errlog(pointwise=err, particle=perr)
    assert err < 1e-12 and perr < 1e-12


def test_grains_full_size(errlog):
    """The full-size benchmark-1 shape, 200 steps, every fluid node against the
    oracle at the shifted-FP32 bounds (rho 1e-6, u 1e-4, f - omega_i rho0 5e-5)."""
    w, ref, ctx = grains_pair("f32s")
    assert len(w.particles) == 45
    oracle.set_threads(0)
    ref.step(200)
    ctx.step(200)
    errs, tols = compare_state(ref, ctx, "f32s", w.solid)
    perr = max(abs(a[k] - b[k]) for a, b in zip(ref.particles(), ctx.particles()) for k in ("x", "y", "U", "V"))
    errlog(**errs, particle=perr)
    assert_close(errs, tols, "grains")
    assert perr < 1e-6
