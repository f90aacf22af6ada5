"""The staged stream-collide kernel (row segments brought into shared memory by
bulk asynchronous copies, kernel 2 of lbm_set_launch) and the register kernel
on a resident-only grid (kernel 3, several items per warp) against the FP64
oracle, and bitwise against the register-pipelined kernel with one item per
warp.

Both kernels run the same per-node arithmetic in the same order, so on the same
inputs their stored populations must be identical bit for bit; the oracle
comparison uses the per-store tolerances of the parity tests.  The cases cover
every boundary kind the staged path handles differently from the register
path: the left / right halo of a row segment, periodic x seams (wrapped
elements read from global memory), open ends (Zou-He placeholders), periodic
and wall rows, the ragged last segment of a row, several domains, the
particle-overlapped step (staged items away from particles, register items
near them), and warps with more than 32 candidate items.
"""
import numpy as np
import pytest

from gpu_helpers import assert_close, compare_state, gpu_params, oracle_params, pair
from oracle import oracle
from paper_2006_12910_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu
# staged configurations, and the register kernel on a grid of resident CTAs only (3)
# or on 8 CTAs per SM (4)
STAGED = [(2, 64, 4), (2, 128, 2), (2, 128, 3), (2, 256, 1), (3, 128, 0), (3, 32, 0), (4, 128, 0)]
STORES = ["f64", "f32", "f32s", "f16s", "bf16s"]


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def twin(base, store, solid=None, particles=None, f0=None, launch=(2, 128, 3)):
    """Oracle, a context on the register kernel and one on the staged kernel."""
    ref, reg = pair(base, store, solid=solid, particles=particles, f0=f0)
    _, stg = pair(base, store, solid=solid, particles=particles, f0=f0)
    reg.set_launch(0, 128, 0)
    stg.set_launch(*launch)
    assert stg.launch()[:3] == tuple(launch)
    return ref, reg, stg


def check(ref, reg, stg, store, steps, solid=None, label=""):
    ref.step(steps)
    reg.step(steps)
    stg.step(steps)
    assert np.array_equal(reg.populations(), stg.populations()), f"{label}: staged != register kernel"
    errs, tols = compare_state(ref, stg, store, solid)
    assert_close(errs, tols, label)
    return errs


@pytest.mark.parametrize("launch", STAGED)
@pytest.mark.parametrize("store", STORES)
def test_staged_obstacles_walls_ragged(store, launch, errlog):
    nx, ny = 203, 37
    solid = workloads.disk_mask(nx, ny, [(40.2, 17.5, 6.3), (101.7, 8.0, 4.1), (150.0, 28.8, 5.0), (0.5, 20.0, 3.0)])
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.75, gx=2e-5)
    ref, reg, stg = twin(base, store, solid=solid, launch=launch)
    errs = check(ref, reg, stg, store, 200, solid, f"{store} {launch}")
    errlog(store=store, launch=launch, **errs)


@pytest.mark.parametrize("store", STORES)
def test_staged_inlet_outlet(store, errlog):
    nx, ny = 130, 41
    solid = workloads.disk_mask(nx, ny, [(45.0, 20.3, 7.1), (90.4, 10.2, 5.5)])
    base = dict(nx=nx, ny=ny, periodic_x=0, inlet_outlet=1, periodic_y=0, walls_y=1, tau=0.7,
                rho_in=1.001, rho_out=0.999)
    ref, reg, stg = twin(base, store, solid=solid)
    errs = check(ref, reg, stg, store, 200, solid, store)
    errlog(store=store, **errs)


@pytest.mark.parametrize("store", STORES)
def test_staged_periodic_noise(store, errlog):
    """Periodic in x and y (wrapped rows and seams) with thermal noise."""
    base = dict(nx=64, ny=48, periodic_x=1, periodic_y=1, walls_y=0, tau=0.8, kT=1e-5, seed=7, domain_id=2)
    ref, reg, stg = twin(base, store)
    ref.step(10)
    reg.step(10)
    stg.step(10)
    assert np.array_equal(reg.populations(), stg.populations())
    fr, fg = ref.populations(), stg.populations()
    err = float(np.abs(fg - fr).max() / np.abs(fr).max())
    errlog(store=store, pointwise=err)
    assert err < {"f64": 1e-12, "f32": 1e-5, "f32s": 1e-5, "f16s": 1e-3, "bf16s": 1e-2}[store]


@pytest.mark.parametrize("store", ["f64", "f32s", "f16s"])
def test_staged_power_law(store, errlog):
    nx, ny = 64, 32
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=1.0, gx=2e-5, power_law=1,
                n_pl=0.5, xi_pl=0.01, tau_min=0.51, tau_max=2.0)
    Y = np.arange(ny) + 0.5
    u = 4e-3 * Y * (ny - Y) / (ny / 2) ** 2
    f0 = np.zeros((9, ny, nx))
    for y in range(ny):
        f0[:, y, :] = oracle.feq(1.0, u[y], 0.0)[:, None]
    f0 *= 1 + 1e-4 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, None, :]
    ref, reg, stg = twin(base, store, f0=f0)
    errs = check(ref, reg, stg, store, 200, None, store)
    errlog(store=store, **errs)


@pytest.mark.parametrize("launch", [(2, 128, 3), (2, 64, 4), (3, 128, 0), (4, 128, 0)])
@pytest.mark.parametrize("store", ["f64", "f32s", "f16s"])
def test_staged_particles_overlapped(store, launch, errlog):
    """Particles: the items away from particles run on the staged kernel, the
    items near them on the register kernel after the particle kernel."""
    nx, ny = 96, 64
    solid = workloads.disk_mask(nx, ny, [(70.3, 40.2, 6.0)])
    parts = [dict(x=30.2, y=30.7, R=7.3, rho_p=1.2, U=0.02, V=-0.01, Omega=0.003),
             dict(x=48.6, y=33.1, R=6.1, rho_p=0.9, U=-0.01, V=0.0, Omega=-0.002),
             dict(x=62.5, y=16.4, R=4.6, rho_p=1.05, fixed=1)]
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=1e-5, gy=-2e-6,
                lj_psi=1e-3, lj_rit=2.5)
    ref, reg, stg = twin(base, store, solid=solid, particles=parts, launch=launch)
    errs = check(ref, reg, stg, store, 120, solid, store)
    assert reg.particles() == stg.particles()
    errlog(store=store, launch=launch, **errs)


@pytest.mark.parametrize("store", ["f64", "f32s"])
def test_staged_ensemble(store, errlog):
    ws = workloads.ensemble(ndom=5, sizes=((48, 40), (64, 32), (96, 72), (40, 40)), R=4.0)
    ps, plist, f0s = [], [], []
    refs = []
    for d, w in enumerate(ws):
        base = dict(nx=w.nx, ny=w.ny, **{k: v for k, v in w.params.items()})
        f0 = workloads.random_populations(w.nx, w.ny, seed=500 + d, amp=0.01)
        refs.append(oracle.Domain(oracle_params(base), particles=w.particles, f0=f0))
        ps.append(gpu_params(base, store, len(w.particles)))
        plist.append(w.particles)
        f0s.append(f0)
    ctxs = []
    for launch in [(0, 128, 0), (2, 128, 2), (3, 64, 0)]:
        ctx = lbm.Context(ps, particles=plist)
        for d, f0 in enumerate(f0s):
            ctx.set_populations(f0, dom=d)
        ctx.set_launch(*launch)
        ctx.step(30)
        ctxs.append(ctx)
    for r in refs:
        r.step(30)
    for d, r in enumerate(refs):
        a, b = ctxs[0].populations(dom=d), ctxs[1].populations(dom=d)
        assert np.array_equal(a, b), d
        assert np.array_equal(a, ctxs[2].populations(dom=d)), d
        e = float(np.linalg.norm(b - r.populations()) / np.linalg.norm(r.populations()))
        errlog(store=store, dom=d, f=e)
        assert e < (1e-12 if store == "f64" else 1e-5)


def test_staged_many_items_per_warp():
    """8192 x 2048 FP32: more than 32 candidate items per warp (the candidate
    screen refills), with particles so that near items are skipped."""
    nx, ny = 8192, 2048
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=1e-6)
    parts = [dict(x=100.0 + 390.0 * k, y=200.0 + 80.0 * (k % 20), R=9.5, rho_p=1.05, U=0.01, V=0.0, Omega=0.0)
             for k in range(20)]
    rng = np.random.default_rng(5)
    f0 = (oracle.feq(1.0, 0.0, 0.0)[:, None, None] * (1 + 0.01 * rng.standard_normal((9, ny, nx)))).astype(np.float64)
    ctxs = []
    for launch in [(1, 128, 0), (2, 64, 2), (3, 128, 0)]:
        ctx = lbm.Context(gpu_params(base, "f32s", len(parts)), particles=[parts])
        ctx.set_populations(f0)
        ctx.set_launch(*launch)
        ctx.step(4)
        ctxs.append(ctx)
    items = ny * (nx // 128)
    k, block, stages, grid = ctxs[1].launch()
    assert items > 32 * grid * (block // 32)
    assert np.array_equal(ctxs[0].populations(), ctxs[1].populations())
    assert ctxs[0].particles() == ctxs[1].particles()
    k, block, stages, grid = ctxs[2].launch()
    assert items > 8 * grid * (block // 32)  # several items per warp
    assert np.array_equal(ctxs[0].populations(), ctxs[2].populations())
    assert ctxs[0].particles() == ctxs[2].particles()


def test_set_launch_rejects_bad_values():
    base = dict(nx=32, ny=32, periodic_x=1, periodic_y=1, walls_y=0, tau=0.8)
    ctx = lbm.Context(gpu_params(base, "f32s"))
    before = ctx.launch()
    for bad in [(5, 128, 0), (0, 48, 0), (0, 1024, 0), (1, 256, 0), (3, 256, 0), (3, 160, 0), (2, 128, 0), (2, 128, 9),
                (2, 512, 2), (-1, 128, 0)]:
        with pytest.raises(lbm.LbmError):
            ctx.set_launch(*bad)
        assert ctx.launch() == before
    ctx.set_launch(2, 128, 2)
    assert ctx.launch()[:3] == (2, 128, 2)
    ctx.autotune(3)
    assert ctx.launch()[0] in (0, 1, 2, 3, 4)
