"""The confined-channel fluctuating workload on the GPU: the shape of the paper's
second benchmark (Sec. 6 benchmark 2: a 3000 x 41 walled channel, one disk of
radius 7.5, kT = 5e-5, nu = 0.1, no external force).

- Parity: the full-size channel against the FP64 oracle, pointwise, on the same
  seeded noise (FP64 store to round-off, shifted FP32 store to the noise
  tolerance of the other fluctuating tests), particle state included.
- Thermalisation: every row of the fluid away from the disk, wall rows
  included, carries <rho u_x^2> = <rho u_y^2> = kT (Sec. 4; the result the
  paper recalls for a fluctuating fluid in a confined channel).
- Brownian disk: its translational and rotational kinetic temperatures are
  near kT, its velocity autocorrelation dies out, and its mean-squared
  displacement along the channel crosses over from ballistic (local exponent
  near 2) to diffusive (near 1), the behaviour the paper recalls for this
  benchmark.  A single disk over 60,000 steps gives intervals of a few
  percent; the 2 % statement is tested on many disks (test_gpu_brownian.py).
"""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_params, oracle_params
from oracle import oracle
from paper_2006_12910_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def channel_pair(store):
    w = workloads.confined_channel()
    base = dict(nx=w.nx, ny=w.ny, **w.params)
    f0 = np.empty((9, w.ny, w.nx))
    f0[:] = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    ref = oracle.Domain(oracle_params(base), particles=w.particles, f0=f0)
    ctx = lbm.Context(gpu_params(base, store, 1), particles=[w.particles])
    ctx.set_populations(f0)
    return w, ref, ctx


@pytest.mark.parametrize("store,steps,lim", [("f64", 20, 1e-12), ("f32s", 10, 1e-5)])
def test_confined_channel_parity(store, steps, lim, errlog):
    w, ref, ctx = channel_pair(store)
    oracle.set_threads(0)
    ref.step(steps)
    ctx.step(steps)
    fr, fg = ref.populations(), ctx.populations()
    # largest difference over the largest shifted population |f - omega_i rho0|
    w9 = oracle.feq(1.0, 0.0, 0.0)[:, None, None]
    err = float(np.abs(fg - fr).max() / np.abs(fr - w9).max())
    pr, pg = ref.particles()[0], ctx.particles()[0]
    perr = max(abs(pr[k] - pg[k]) for k in ("x", "y", "U", "V", "Omega"))
    errlog(store=store, steps=steps, pointwise=err, particle=perr)
    assert err < lim
    assert perr < (1e-12 if store == "f64" else 1e-7)


def test_confined_channel_thermalisation_and_brownian_disk(errlog):
    w = workloads.confined_channel()
    ctx = lbm.Context(gpu_params(dict(nx=w.nx, ny=w.ny, **w.params), "f32s", 1), particles=[w.particles])
    kT = w.params["kT"]
    q = w.particles[0]
    M = math.pi * q["R"] ** 2 * q["rho_p"]
    ctx.step(2000)
    # fluid: row temperatures over the nodes more than R + 10 away from the disk
    acc = np.zeros((2, w.ny))
    n_fluid = 40
    for _ in range(n_fluid):
        ctx.step(50)
        rho, ux, uy = ctx.moments()
        x = ctx.particles()[0]["x"]
        dx = np.abs(((np.arange(w.nx) - x) + w.nx / 2) % w.nx - w.nx / 2)
        far = dx > q["R"] + 10
        acc[0] += (rho * ux * ux)[:, far].mean(axis=1)
        acc[1] += (rho * uy * uy)[:, far].mean(axis=1)
    rows = acc / n_fluid / kT
    # disk: velocities every step
    n = 60000
    U = np.zeros((n, 3))
    for i in range(n):
        ctx.step(1)
        p = ctx.particles()[0]
        U[i] = (p["U"], p["V"], p["Omega"])
    ctx.sync()  # no device error over the run
    T = (U[:, :2] ** 2).mean(axis=0) * M / kT
    T_rot = (U[:, 2] ** 2).mean() * (0.5 * M * q["R"] ** 2) / kT
    # 95 % intervals from block means of 3,000 steps (about 30 velocity
    # correlation times of this disk, so the blocks are nearly independent)
    blk = 3000
    bm = (U[: n // blk * blk] ** 2).reshape(n // blk, blk, 3).mean(axis=1)
    bm *= np.array([M, M, 0.5 * M * q["R"] ** 2]) / kT
    ci = 1.96 * bm.std(axis=0, ddof=1) / math.sqrt(bm.shape[0])

    def acf(v, nl):
        f = np.fft.rfft(v, 2 * len(v))
        return np.fft.irfft(f * np.conj(f))[:nl] / (len(v) - np.arange(nl))

    C = acf(U[:, 0], 1001)
    xs = np.concatenate([[0.0], np.cumsum(U[:, 0])])  # r_c(t+1) = r_c(t) + U_p(t)
    msd = {lag: float(((xs[lag:] - xs[:-lag]) ** 2).mean()) for lag in (1, 10, 1000, 10000)}
    exp_short = math.log(msd[10] / msd[1]) / math.log(10)
    exp_long = math.log(msd[10000] / msd[1000]) / math.log(10)
    errlog(rows_x=rows[0].tolist(), rows_y=rows[1].tolist(), T=T.tolist(), T_rot=T_rot, ci=ci.tolist(),
           vacf_1000=float(C[1000] / C[0]), msd_exponent_1_10=exp_short, msd_exponent_1000_10000=exp_long)
    # each row: 40 snapshots of ~2,900 nodes; per-row standard error well under 1 %
    assert np.abs(rows - 1).max() < 0.03, rows
    # one disk between walls (no momentum conservation, so no box factor): its
    # kinetic temperatures must contain 1 in their 99 % intervals
    Ts = np.array([T[0], T[1], T_rot])
    assert np.all(np.abs(Ts - 1.0) < 2.58 / 1.96 * ci + 0.005), (Ts, ci)
    assert np.all(ci < 0.08), ci
    assert abs(C[1000] / C[0]) < 0.1
    assert exp_short > 1.7 and exp_long < 1.25, (exp_short, exp_long)
