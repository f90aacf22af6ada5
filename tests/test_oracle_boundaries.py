"""Pins of the oracle's open density columns (Zou-He inlet/outlet).

The paper drives benchmark 1 with a body force and periodic ends (Sec. 6);
the density-driven inlet/outlet follows Zou & He (1997).  Pins: the
prescribed density and zero transverse velocity hold exactly on the open
columns, every interior column obeys the exact discrete mass balance, and the
developed mid-channel flow is the Poiseuille parabola for the local pressure
gradient.
"""
import numpy as np


def _channel(oracle, nx, ny, tau, rin=1.001, rout=0.999):
    p = oracle.make_params(nx=nx, ny=ny, periodic_x=0, inlet_outlet=1, periodic_y=0,
                           walls_y=1, tau=tau, rho_in=rin, rho_out=rout)
    return oracle.Domain(p)


def _interface_flux(f):
    """Mass crossing x+1/2 in one streaming step; diagonal populations on a wall
    row are reflected by the wall and do not cross."""
    a = f[1].sum(0) + f[5][:-1].sum(0) + f[8][1:].sum(0)
    b = f[3].sum(0) + f[6][:-1].sum(0) + f[7][1:].sum(0)
    return a[:-1] - b[1:]


def test_open_columns_hold_density_and_zero_uy(oracle):
    d = _channel(oracle, 40, 11, 0.9)
    d.step(50)
    rho, ux, uy = d.moments()
    assert np.abs(rho[1:-1, 0] - 1.001).max() < 2e-15
    assert np.abs(rho[1:-1, -1] - 0.999).max() < 2e-15
    assert np.abs(uy[1:-1, 0]).max() < 1e-16 and np.abs(uy[1:-1, -1]).max() < 1e-16


def test_interior_column_mass_balance_exact(oracle):
    d = _channel(oracle, 40, 11, 0.7)
    d.step(30)
    f0 = d.populations()
    m0 = f0.sum(axis=(0, 1))
    d.step(1)
    m1 = d.populations().sum(axis=(0, 1))
    phi = _interface_flux(f0)
    dm = (m1 - m0)[1:-1]
    assert np.abs(dm - (phi[:-1] - phi[1:])).max() < 1e-14 * m0.max()


def test_developed_flow_is_poiseuille_for_local_gradient(oracle):
    nx, ny, tau = 64, 17, 0.8
    nu = (tau - 0.5) / 3.0
    d = _channel(oracle, nx, ny, tau)
    d.step(40000)
    rho, ux, _ = d.moments()
    rc = rho.mean(axis=0)
    m = nx // 2
    G = -(rc[m + 1] - rc[m - 1]) / 2.0 / 3.0  # -dp/dx with p = c_s^2 rho
    Y = np.arange(ny) + 0.5
    us = G * (16 * (tau - 0.5) ** 2 - 3) / (8 * (tau - 0.5))
    exact = (G / (2 * nu) * Y * (ny - Y) + us) / rc[m]
    assert np.abs(ux[:, m] - exact).max() / exact.max() < 1e-4
    # the steady flux through every interface is the same to round-off
    phi = _interface_flux(d.populations())
    assert (phi.max() - phi.min()) / phi.mean() < 1e-8
