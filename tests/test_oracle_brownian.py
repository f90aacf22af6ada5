"""Pin of the oracle's particle-fluid thermal coupling (Sec. 3 with Sec. 4).

A Brownian disk in a fluctuating fluid must carry the fluid's temperature:
equipartition gives <U^2> = <V^2> = kT/M and <Omega^2> = kT/I (Sec. 4: the
particle's kinetic energy balances the thermal energy of the fluid, as the
fluctuation-dissipation theorem requires).  In a periodic box the exterior
fluid and the particles conserve their total momentum exactly (noise and
momentum exchange both conserve it), so each translational component is
reduced by the finite-box factor 1 - M/M_tot, M_tot the mass of everything
that shares that momentum (the disks and the fluid outside them).  Angular
momentum is not conserved in a periodic box, so Omega has no such factor.

Workload: 64 x 64 periodic box, nine neutrally buoyant disks (R = 5,
rho_p = rho0 = 1) on a 3 x 3 grid, kT = 1e-5, tau = 1.0 and 0.8, four seeds
each, 20,000 steps after a 2,000-step start, velocities sampled every 10 steps.
The interval is the 95 % interval of block means (blocks of 1,000 steps, one
per disk and seed, treated as independent).  An explicit particle update
(boundary velocity at t instead of mid-step) fails this pin: it runs hot by
about 1/(1 - z/2M) (13-17 % here) and, for these neutral disks, turns unstable.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

PI = np.pi
L, R, KT, NSIDE = 64, 5.0, 1e-5, 3
BURN, STEPS, EVERY = 2000, 20000, 10
SEEDS = (101, 102, 103, 104)


def _run(job):
    tau, seed = job
    from oracle import oracle
    oracle.set_threads(1)
    parts = [dict(x=(a + 0.5) * L / NSIDE + 0.37, y=(b + 0.5) * L / NSIDE + 0.21, R=R, rho_p=1.0)
             for a in range(NSIDE) for b in range(NSIDE)]
    p = oracle.make_params(nx=L, ny=L, tau=tau, kT=KT, seed=seed)
    d = oracle.Domain(p, particles=parts)
    d.step(BURN)
    out = np.zeros((STEPS // EVERY, len(parts), 3))
    inside = 0
    for s in range(STEPS // EVERY):
        d.step(EVERY)
        q = d.particles()
        out[s] = [(x["U"], x["V"], x["Omega"]) for x in q]
        if s % 100 == 0:
            inside += int((d.owner() != 0).sum())
    return tau, out, inside / (STEPS // EVERY // 100)


@pytest.fixture(scope="module")
def samples(oracle):
    jobs = [(tau, s) for tau in (1.0, 0.8) for s in SEEDS]
    procs = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_run, jobs)
    return res


def _block_stats(series, block):
    """Mean and 95 % half-width of block means over every (seed, disk) series."""
    means = []
    for x in series:                      # x: samples x disks
        n = x.shape[0] // block
        means.extend(x[:n * block].reshape(n, block, -1).mean(axis=1).ravel())
    means = np.asarray(means)
    return means.mean(), 1.96 * means.std(ddof=1) / np.sqrt(means.size)


@pytest.mark.slow
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_brownian_disk_equipartition(samples, tau):
    M = 1.0 * PI * R * R
    I = 0.5 * M * R * R
    runs = [(out, inside) for t, out, inside in samples if t == tau]
    n_disk = NSIDE * NSIDE
    inside = np.mean([r[1] for r in runs])
    M_tot = n_disk * M + (L * L - inside) * 1.0
    box = 1.0 - M / M_tot
    u2 = [M * 0.5 * (out[:, :, 0] ** 2 + out[:, :, 1] ** 2) / KT / box for out, _ in runs]
    o2 = [I * out[:, :, 2] ** 2 / KT for out, _ in runs]
    block = 1000 // EVERY
    tu, cu = _block_stats(u2, block)
    tr, cr = _block_stats(o2, block)
    print(f"tau={tau}: M<U^2>/(kT(1-M/M_tot)) = {tu:.4f} +- {cu:.4f}, "
          f"I<Omega^2>/kT = {tr:.4f} +- {cr:.4f} (box factor {box:.5f})")
    # the interval is narrow enough for the 2 % statement to mean something
    assert cu < 0.015 and cr < 0.015
    assert abs(tu - 1.0) < 0.02
    assert abs(tr - 1.0) < 0.02
