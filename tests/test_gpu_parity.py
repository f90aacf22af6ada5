"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative L2 over fluid nodes, gpu_helpers.TOL): the FP64 GPU path
within 1e-12 (1e-11 on the shifted populations); the shifted FP32 store within
1e-6 on density and 1e-4 on velocity after the stated steps (up to 1000), 5e-5
on f - omega_i rho0 and on rho - rho0; the shifted FP16 / BF16 stores are held
to looser, measured bounds (their storage rounding is 2^-11 / 2^-8 of the
shifted population); the unshifted FP32 store is reported against its own
measured bounds.  Noise runs are compared pointwise over 10 steps, the largest
difference over the largest shifted population |f - omega_i rho0|, within 1e-5
for the shifted FP32 store.
"""
import numpy as np
import pytest

from gpu_helpers import W9, assert_close, compare_state, gpu_params, oracle_params, pair, rel
from oracle import oracle
from paper_2006_12910_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu
STORES = ["f64", "f32", "f32s", "f16s", "bf16s"]


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("store", STORES)
def test_bgk_periodic_random_state(store, errlog):
    base = dict(nx=96, ny=50, periodic_x=1, periodic_y=1, walls_y=0, tau=0.7, gx=1e-5, gy=-3e-6)
    ref, ctx = pair(base, store)
    ref.step(200)
    ctx.step(200)
    errs, tols = compare_state(ref, ctx, store)
    errlog(store=store, **errs)
    assert_close(errs, tols, store)
    assert ctx.step_count == 200


@pytest.mark.parametrize("store", ["f64", "f32s"])
def test_poiseuille_channel_1000_steps(store, errlog):
    """256x64, tau=0.8, g=1e-6, periodic x, halfway walls, rest start, 1000 steps."""
    w = workloads.poiseuille()
    base = dict(nx=w.nx, ny=w.ny, **w.params)
    f0 = np.zeros((9, w.ny, w.nx))
    f0[:] = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    ref, ctx = pair(base, store, f0=f0)
    ref.step(1000)
    ctx.step(1000)
    errs, tols = compare_state(ref, ctx, store)
    errlog(store=store, **errs)
    assert_close(errs, tols, store)
    m_ref, m_gpu = ref.checks(), ctx.checks()
    assert abs(m_gpu[0] - m_ref[0]) / m_ref[0] < (1e-13 if store == "f64" else 1e-7)


@pytest.mark.parametrize("store", STORES)
def test_obstacles_walls_ragged(store, errlog):
    """Ragged width (203 is no multiple of any vector width), obstacles, walls."""
    nx, ny = 203, 37
    solid = workloads.disk_mask(nx, ny, [(40.2, 17.5, 6.3), (101.7, 8.0, 4.1), (150.0, 28.8, 5.0), (0.5, 20.0, 3.0)])
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.75, gx=2e-5)
    ref, ctx = pair(base, store, solid=solid)
    ref.step(300)
    ctx.step(300)
    errs, tols = compare_state(ref, ctx, store, solid)
    errlog(store=store, **errs)
    assert_close(errs, tols, store)
    assert np.all(ctx.populations()[:, solid.astype(bool)] == 0.0)


@pytest.mark.parametrize("store", STORES)
def test_inlet_outlet_with_obstacles(store, errlog):
    nx, ny = 130, 41
    solid = workloads.disk_mask(nx, ny, [(45.0, 20.3, 7.1), (90.4, 10.2, 5.5)])
    base = dict(nx=nx, ny=ny, periodic_x=0, inlet_outlet=1, periodic_y=0, walls_y=1, tau=0.7,
                rho_in=1.001, rho_out=0.999)
    ref, ctx = pair(base, store, solid=solid)
    ref.step(300)
    ctx.step(300)
    errs, tols = compare_state(ref, ctx, store, solid)
    errlog(store=store, **errs)
    assert_close(errs, tols, store)
    rho = ctx.moments()[0]
    tol_rho = {"f64": 1e-14, "f32": 1e-6, "f32s": 1e-6, "f16s": 1e-5, "bf16s": 1e-4}[store]
    assert np.abs(rho[1:-1, 0] - 1.001).max() < tol_rho
    assert np.abs(rho[1:-1, -1] - 0.999).max() < tol_rho


@pytest.mark.parametrize("store", STORES)
@pytest.mark.parametrize("n", [0.5, 0.75, 1.5])
def test_power_law_channel(store, n, errlog):
    """Developed channel start (a parabola plus a small x-modulation).  A random
    start is not used here: with n < 1 the unclamped tau* is steep near zero
    strain, and on random data the oracle itself amplifies a 1e-15 perturbation
    to 1e-6 within 100 steps, so no implementation could be compared at 1e-12."""
    nx, ny = 64, 32
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=1.0, gx=2e-5, power_law=1,
                n_pl=n, xi_pl=0.01, tau_min=0.51, tau_max=2.0)
    Y = np.arange(ny) + 0.5
    u = 4e-3 * Y * (ny - Y) / (ny / 2) ** 2
    f0 = np.zeros((9, ny, nx))
    for y in range(ny):
        f0[:, y, :] = oracle.feq(1.0, u[y], 0.0)[:, None]
    f0 *= 1 + 1e-4 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, None, :]
    ref, ctx = pair(base, store, f0=f0)
    ref.step(300)
    ctx.step(300)
    errs, tols = compare_state(ref, ctx, store)
    errlog(store=store, n=n, **errs)
    if store == "bf16s":
        # BF16 keeps 8 mantissa bits of the shifted population: the small
        # non-equilibrium strain that sets tau* is lost, so the profile drifts
        # (reported, not gated).
        assert errs["u"] < 0.5 and errs["rho"] < 1e-3
        return
    assert_close(errs, tols, f"{store} n={n}")


@pytest.mark.parametrize("store", ["f64", "f32s"])
@pytest.mark.parametrize("variant", ["kappa=1", "kappa=0.5^(n-1)", "nu in [1e-5, 0.1]"])
@pytest.mark.parametrize("n", [0.75, 1.5])
def test_power_law_paper_variants(store, variant, n, errlog):
    """The other kappa values of Eq. nn4 that Sec. 5 cites, and the paper's own
    bounds on nu* (1e-5 <= nu* <= 0.1, i.e. tau* in [0.50003, 0.8]), on the
    developed channel start of test_power_law_channel."""
    nx, ny = 64, 32
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=1.0, gx=2e-5, power_law=1,
                n_pl=n, xi_pl=0.01, tau_min=0.51, tau_max=2.0)
    if variant == "kappa=1":
        base["kappa_pl"] = 1.0
    elif variant == "kappa=0.5^(n-1)":
        base["kappa_pl"] = 0.5 ** (n - 1)
    else:
        base.update(tau_min=0.5 + 3 * 1e-5, tau_max=0.5 + 3 * 0.1)
    Y = np.arange(ny) + 0.5
    u = 4e-3 * Y * (ny - Y) / (ny / 2) ** 2
    f0 = np.zeros((9, ny, nx))
    for y in range(ny):
        f0[:, y, :] = oracle.feq(1.0, u[y], 0.0)[:, None]
    f0 *= 1 + 1e-4 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, None, :]
    ref, ctx = pair(base, store, f0=f0)
    ref.step(300)
    ctx.step(300)
    errs, tols = compare_state(ref, ctx, store)
    errlog(store=store, variant=variant, n=n, **errs)
    assert_close(errs, tols, f"{store} {variant} n={n}")


@pytest.mark.parametrize("store", STORES)
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_fluctuating_lb_10_steps_pointwise(store, tau, errlog):
    base = dict(nx=64, ny=64, periodic_x=1, periodic_y=1, walls_y=0, tau=tau, kT=1e-5, seed=20061294, domain_id=3)
    ref, ctx = pair(base, store)
    ref.step(10)
    ctx.step(10)
    fr, fg = ref.populations(), ctx.populations()
    err = float(np.abs(fg - fr).max() / np.abs(fr).max())
    fneq = fr - W9[:, None, None]
    err_neq = float(np.abs(fg - fr).max() / np.abs(fneq).max())
    errs, tols = compare_state(ref, ctx, store)
    errlog(store=store, pointwise=err, pointwise_neq=err_neq, **errs)
    # unshifted FP32: measured 1.5e-5 (its rounding is 2^-24 of omega_i, not of f - omega_i rho0)
    lim = {"f64": 1e-12, "f32": 5e-5, "f32s": 1e-5, "f16s": 1e-3, "bf16s": 1e-2}[store]
    assert err_neq < lim
    assert_close(errs, tols, store)


@pytest.mark.parametrize("store", ["f64", "f32s", "f16s"])
def test_moving_particles_with_lj(store, errlog):
    nx, ny = 96, 64
    solid = workloads.disk_mask(nx, ny, [(70.3, 40.2, 6.0)])
    parts = [dict(x=30.2, y=30.7, R=7.3, rho_p=1.2, U=0.02, V=-0.01, Omega=0.003),
             dict(x=48.6, y=33.1, R=6.1, rho_p=0.9, U=-0.01, V=0.0, Omega=-0.002),
             dict(x=62.5, y=16.4, R=4.6, rho_p=1.05, fixed=1)]
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=1e-5, gy=-2e-6,
                lj_psi=1e-3, lj_rit=2.5)
    ref, ctx = pair(base, store, solid=solid, particles=parts)
    ref.step(150)
    ctx.step(150)
    errs, tols = compare_state(ref, ctx, store, solid)
    pr, pg = ref.particles(), ctx.particles()
    perr = max(abs(a[k] - b[k]) for a, b in zip(pr, pg) for k in ("x", "y", "U", "V", "Omega", "theta"))
    ferr = max(rel(ctx.particle_forces(i)[:9], ref.diag(i)[:9]) for i in range(3))
    cnt = all(np.array_equal(ctx.particle_forces(i)[9:11], ref.diag(i)[9:11]) for i in range(3))
    errlog(store=store, particle=perr, forces=ferr, **errs)
    assert_close(errs, tols, store)
    assert cnt
    assert perr < {"f64": 1e-11, "f32s": 1e-5, "f16s": 1e-3}[store]
    assert ferr < {"f64": 1e-10, "f32s": 1e-4, "f16s": 5e-2}[store]


@pytest.mark.parametrize("store", ["f64", "f32s"])
def test_lj_contacts_pairs_walls_obstacles(store, errlog):
    """Eq. MP2 active every step: a particle pair two nodes apart, a particle two
    nodes from the lower wall and one two nodes from an obstacle."""
    nx, ny = 100, 60
    solid = workloads.disk_mask(nx, ny, [(75.0, 38.0, 7.0)])
    parts = [dict(x=20.3, y=30.2, R=6.2, rho_p=1.1, U=0.005, V=0.0, Omega=0.001),
             dict(x=33.3, y=31.0, R=5.8, rho_p=1.0, U=-0.004, V=0.001, Omega=0.0),
             dict(x=50.4, y=6.2, R=5.5, rho_p=1.2, U=0.0, V=-0.003, Omega=0.0),
             dict(x=75.2, y=22.5, R=6.6, rho_p=1.0, U=0.0, V=0.004, Omega=-0.001)]
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=1e-5, lj_psi=1e-3, lj_rit=2.5)
    f0 = workloads.random_populations(nx, ny, seed=77, amp=0.01, solid=solid)
    ref, ctx = pair(base, store, solid=solid, particles=parts, f0=f0)
    worst = 0.0
    for _ in range(8):
        ref.step(10)
        ctx.step(10)
        for i in range(4):
            dg, do = ctx.particle_forces(i), ref.diag(i)
            assert np.array_equal(dg[9:11], do[9:11])
            worst = max(worst, rel(dg[6:9], do[6:9]) if np.abs(do[6:9]).max() > 0 else np.abs(dg[6:9]).max())
    pr, pg = ref.particles(), ctx.particles()
    perr = max(abs(a[k] - b[k]) for a, b in zip(pr, pg) for k in ("x", "y", "U", "V", "Omega"))
    errlog(store=store, lj=worst, particle=perr)
    assert worst < (1e-12 if store == "f64" else 1e-6)
    assert perr < (1e-12 if store == "f64" else 1e-6)
    assert np.abs(ref.diag(0)[6:8]).max() > 0 and np.abs(ref.diag(2)[6:8]).max() > 0


@pytest.mark.parametrize("store", ["f64", "f32s"])
def test_particle_mass_conservation_exact(store):
    nx, ny = 64, 64
    parts = [dict(x=30.2, y=30.7, R=8.3, rho_p=1.0, U=0.03, V=-0.02, Omega=0.004)]
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=1, walls_y=0, tau=0.7)
    ref, ctx = pair(base, store, particles=parts)
    m0 = ctx.checks()[0]
    ctx.step(300)
    m1 = ctx.checks()[0]
    assert abs(m1 - m0) / m0 < (1e-13 if store == "f64" else 1e-6)


@pytest.mark.parametrize("store", ["f64", "f32s"])
def test_ensemble_of_uneven_domains(store, errlog):
    ws = workloads.ensemble(ndom=5, sizes=((48, 40), (64, 32), (96, 72), (40, 40)), R=4.0)
    refs, ps, plist, f0s = [], [], [], []
    for d, w in enumerate(ws):
        base = dict(nx=w.nx, ny=w.ny, **{k: v for k, v in w.params.items()})
        f0 = workloads.random_populations(w.nx, w.ny, seed=500 + d, amp=0.01)
        refs.append(oracle.Domain(oracle_params(base), particles=w.particles, f0=f0))
        ps.append(gpu_params(base, store, len(w.particles)))
        plist.append(w.particles)
        f0s.append(f0)
    ctx = lbm.Context(ps, particles=plist)
    for d, f0 in enumerate(f0s):
        ctx.set_populations(f0, dom=d)
    for r in refs:
        r.step(40)
    ctx.step(40)
    for d, r in enumerate(refs):
        e = rel(ctx.populations(dom=d), r.populations())
        errlog(store=store, dom=d, f=e)
        assert e < (1e-12 if store == "f64" else 1e-5), (d, e)
        pg, po = ctx.particles(dom=d)[0], r.particles()[0]
        assert abs(pg["x"] - po["x"]) < (1e-12 if store == "f64" else 1e-6)


@pytest.mark.parametrize("store", ["f64", "f32s", "f16s"])
def test_checkpoint_resume_bitwise(store, tmp_path):
    nx, ny = 80, 48
    parts = [dict(x=30.2, y=20.7, R=6.3, rho_p=1.1, U=0.02, V=0.01, Omega=0.001)]
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=1, walls_y=0, tau=0.9, kT=1e-5, seed=99)
    _, a = pair(base, store, particles=parts)
    _, b = pair(base, store, particles=parts)
    a.step(60)
    b.step(30)
    b.save(tmp_path / "ck.bin")
    c = lbm.Context(gpu_params(base, store, 1))
    c.load_checkpoint(tmp_path / "ck.bin")
    assert c.step_count == 30
    c.step(30)
    assert np.array_equal(a.populations(), c.populations())
    assert a.particles() == c.particles()


def test_moments_device_and_async_match_host():
    torch = pytest.importorskip("torch")
    base = dict(nx=70, ny=30, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=1e-5)
    ref, ctx = pair(base, "f32s")
    ctx.step(25)
    rho, ux, uy = ctx.moments()
    t = [torch.empty((30, 70), dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx.moments_device(*t)
    ctx.sync()
    assert np.allclose(t[0].cpu().numpy(), rho, rtol=1e-7, atol=0)
    assert np.allclose(t[1].cpu().numpy(), ux, rtol=1e-6, atol=1e-12)
    ctx.moments_async()
    ctx.step(5)
    ra, uxa, uya = ctx.moments_async_wait()
    assert np.allclose(ra, rho, rtol=1e-7, atol=0) and np.allclose(uya, uy, rtol=1e-6, atol=1e-12)


def test_instability_is_reported():
    base = dict(nx=32, ny=32, periodic_x=1, periodic_y=1, walls_y=0, tau=0.8)
    _, ctx = pair(base, "f32s")
    f = ctx.populations()
    f[:, 5, 5] = -1.0  # negative density on one node: a host-made invalid state
    ctx.set_populations(f)
    ctx.step(2)
    with pytest.raises(lbm.LbmError) as ei:
        ctx.sync()
    assert ei.value.code == -4


def test_invalid_calls_raise():
    base = dict(nx=32, ny=32, periodic_x=1, periodic_y=1, walls_y=0, tau=0.8)
    ctx = lbm.Context(gpu_params(base, "f32s", 1))
    with pytest.raises(lbm.LbmError):
        ctx.step(-1)
    with pytest.raises(lbm.LbmError):
        ctx.add_particles(0, [dict(x=10, y=10, R=3, rho_p=1), dict(x=20, y=10, R=3, rho_p=1)])
    with pytest.raises(lbm.LbmError):
        ctx.checks(dom=3)


def test_full_size_porous_workload(errlog):
    """The benchmark workload at full size (2048x1024, ~300 obstacles, 20 particles,
    Zou-He ends, FP32 shifted store), 200 steps, every node compared with the
    oracle (rho within 1e-6, u within 1e-4, f - omega_i rho0 within 5e-5), on each
    launch shape the benchmark's autotuner may pick for the register kernel (one
    item per warp, grid-stride over 16 or 8 CTAs per SM, resident-only grid); all
    must agree bit for bit."""
    w = workloads.porous()
    base = dict(nx=w.nx, ny=w.ny, **w.params)
    f0 = np.empty((9, w.ny, w.nx))
    f0[:] = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    ref, ctx = pair(base, "f32s", solid=w.solid, particles=w.particles, f0=f0)
    oracle.set_threads(0)
    steps = 200
    ref.step(steps)
    first = None
    for launch in [(1, 128, 0), (0, 128, 0), (3, 128, 0), (4, 128, 0)]:
        if first is not None:
            _, ctx = pair(base, "f32s", solid=w.solid, particles=w.particles, f0=f0)
        ctx.set_launch(*launch)
        ctx.step(steps)
        errs, tols = compare_state(ref, ctx, "f32s", w.solid)
        pr, pg = ref.particles(), ctx.particles()
        perr = max(abs(a[k] - b[k]) for a, b in zip(pr, pg) for k in ("x", "y", "U", "V", "Omega"))
        errlog(launch=launch, **errs, particle=perr)
        assert_close(errs, tols, f"porous {launch}")
        assert perr < 1e-6
        f = ctx.populations()
        if first is None:
            first = f
        else:
            assert np.array_equal(f, first), launch
        ctx.close()


def test_fp64_rate_probe():
    """The FP64 rate probe that sets the FP64 store's arithmetic roofline runs and
    reports a rate between a plausible floor and the FP32 rate of the part."""
    g = lbm.fp64_fma_rate()
    assert 50.0 < g < 1e5, g


def test_particles_read_after_step_without_full_sync():
    """lbm_particles right after lbm_step waits only for the step's force launch;
    the state it returns equals the one read after a full synchronisation, for
    one-step and eight-step graph launches, and matches the oracle."""
    nx, ny = 96, 64
    parts = [dict(x=30.2, y=30.7, R=7.3, rho_p=1.2, U=0.02, V=-0.01, Omega=0.003),
             dict(x=70.6, y=25.1, R=6.1, rho_p=0.9, U=-0.01, V=0.0, Omega=-0.002)]
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=1e-5)
    ref, ctx = pair(base, "f32s", particles=parts)
    keys = ("x", "y", "R", "rho_p", "U", "V", "Omega", "theta")
    for n in (1, 8, 3, 16):
        ctx.step(n)
        early = ctx.particles()
        ctx.sync()
        assert ctx.particles() == early, n
        arr = ctx.particles_array()
        assert arr.shape == (len(parts), 8)
        assert all(arr[i, j] == early[i][k] for i in range(len(parts)) for j, k in enumerate(keys))
    ref.step(28)
    pr, pg = ref.particles(), ctx.particles()
    assert max(abs(a[k] - b[k]) for a, b in zip(pr, pg) for k in ("x", "y", "U", "V")) < 1e-6
