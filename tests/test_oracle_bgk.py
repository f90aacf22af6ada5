"""Pins of the oracle's BGK collision, forcing, streaming and walls (Sec. 2).

Closed forms: the Newtonian start-up series of plane Poiseuille flow, the
steady parabola with the known halfway-bounce-back slip, exact mass
conservation and x-invariance.
"""
import numpy as np
import pytest


def startup_series(H, g, nu, t, kmax=4001):
    """Plane Poiseuille flow started from rest between walls at Y=0 and Y=H
    (Y = y + 1/2 for halfway walls): the steady parabola minus its decaying
    odd sine modes (separation of variables of u_t = nu u_yy + g)."""
    Y = np.arange(H) + 0.5
    u = g / (2 * nu) * Y * (H - Y)
    for k in range(1, kmax, 2):
        u -= (4 * g * H * H / (nu * np.pi ** 3 * k ** 3) * np.sin(k * np.pi * Y / H)
              * np.exp(-(k * np.pi / H) ** 2 * nu * t))
    return u


def test_collision_conserves_mass_and_shifts_momentum(oracle):
    """Sec. 2: collision keeps rho; with rho u = sum f e + tau rho g in the
    equilibrium, the post-collision momentum is sum f e + rho g."""
    rng = np.random.default_rng(1)
    e, w, _ = oracle.lattice()
    for tau in (0.6, 0.8, 1.7):
        p = oracle.make_params(tau=tau, gx=3e-4, gy=-1e-4)
        f = w * (1.0 + 0.05 * rng.standard_normal(9))
        out = oracle.collide_node(p, f)
        rho = f.sum()
        assert out.sum() == pytest.approx(rho, rel=1e-15)
        assert np.allclose(out @ e, f @ e + rho * np.array([3e-4, -1e-4]), atol=1e-16, rtol=0)


def test_collision_relaxes_to_equilibrium(oracle):
    """Eq. e.LB1 with dt/tau = 1 lands exactly on f_eq(rho, u_eq)."""
    rng = np.random.default_rng(2)
    _, w, _ = oracle.lattice()
    p = oracle.make_params(tau=1.0, gx=0.0)
    f = w * (1.0 + 0.05 * rng.standard_normal(9))
    e, _, _ = oracle.lattice()
    rho = f.sum()
    u = (f @ e) / rho
    assert np.allclose(oracle.collide_node(p, f), oracle.feq(rho, *u), atol=1e-16, rtol=0)


def test_poiseuille_startup_1000_steps(oracle):
    """256x64, tau=0.8, g=1e-6, periodic x, halfway walls: after 1000 steps the
    profile follows the start-up series (nu = c_s^2 (tau - 1/2), Sec. 2) within
    the O(dx^2) discretisation error; every column is identical; mass is exact."""
    H, g, tau = 64, 1e-6, 0.8
    nu = (tau - 0.5) / 3.0
    p = oracle.make_params(nx=256, ny=H, periodic_x=1, periodic_y=0, walls_y=1, tau=tau, gx=g)
    d = oracle.Domain(p)
    m0 = d.checks()[0]
    d.step(1000)
    rho, ux, uy = d.moments()
    prof = ux[:, 0]
    assert np.array_equal(ux, np.repeat(prof[:, None], 256, axis=1))
    s = startup_series(H, g, nu, 1000.0)
    assert np.linalg.norm(prof - s) / np.linalg.norm(s) < 1e-3
    assert abs(d.checks()[0] - m0) / m0 < 1e-13
    assert np.abs(uy).max() < 1e-15


@pytest.mark.parametrize("tau", [0.8, 0.5 + np.sqrt(3) / 4, 1.2])
def test_poiseuille_steady_with_bounce_back_slip(oracle, tau):
    """Steady BGK + halfway bounce-back: the parabola g Y (H-Y) / (2 nu) plus the
    uniform slip g (16 (tau-1/2)^2 - 3) / (8 (tau-1/2)), which vanishes at
    tau = 1/2 + sqrt(3)/4 (He, Zou, Luo & Dembo, J. Stat. Phys. 87, 1997)."""
    H, g = 32, 1e-6
    nu = (tau - 0.5) / 3.0
    p = oracle.make_params(nx=4, ny=H, periodic_x=1, periodic_y=0, walls_y=1, tau=tau, gx=g)
    d = oracle.Domain(p)
    d.step(int(12 * H * H / nu))
    prof = d.moments()[1][:, 0]
    Y = np.arange(H) + 0.5
    us = g * (16 * (tau - 0.5) ** 2 - 3) / (8 * (tau - 0.5))
    exact = g / (2 * nu) * Y * (H - Y) + us
    assert np.abs(prof - exact).max() / exact.max() < 1e-9


def test_mass_conserved_with_obstacles_and_periodic_y(oracle):
    """Halfway bounce-back at stationary solids conserves mass exactly (Sec. 3)."""
    rng = np.random.default_rng(3)
    nx, ny = 40, 30
    yy, xx = np.mgrid[0:ny, 0:nx]
    solid = ((xx - 12) ** 2 + (yy - 14) ** 2 <= 25) | ((xx - 30) ** 2 + (yy - 5) ** 2 <= 9)
    p = oracle.make_params(nx=nx, ny=ny, tau=0.7, gx=2e-5, gy=-1e-5)
    _, w, _ = oracle.lattice()
    f0 = w[:, None, None] * (1 + 0.01 * rng.standard_normal((9, ny, nx)))
    d = oracle.Domain(p, solid=solid.astype(np.uint8), f0=f0)
    m0 = d.checks()[0]
    d.step(300)
    assert abs(d.checks()[0] - m0) / m0 < 1e-13
    f = d.populations()
    assert np.all(f[:, solid] == 0.0)


def test_periodic_translation_invariance(oracle):
    """A fully periodic lattice commutes with a shift of the initial state."""
    rng = np.random.default_rng(4)
    nx, ny = 24, 18
    _, w, _ = oracle.lattice()
    f0 = w[:, None, None] * (1 + 0.02 * rng.standard_normal((9, ny, nx)))
    p = oracle.make_params(nx=nx, ny=ny, tau=0.9, gx=1e-4)
    a = oracle.Domain(p, f0=f0)
    b = oracle.Domain(p, f0=np.roll(f0, (5, 7), axis=(1, 2)))
    a.step(40)
    b.step(40)
    assert np.array_equal(np.roll(a.populations(), (5, 7), axis=(1, 2)), b.populations())
