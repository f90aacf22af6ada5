"""Pins of the oracle's particle module (Sec. 3, Eqs. MP1-MP8).

No closed-form drag exists in 2-D, so the module is pinned by:
  * brute-force enumeration of the boundary links (Fig. 1),
  * a held particle with U = Omega = 0 behaving exactly like a stationary disk
    obstacle (Eq. MP8 with u_b = 0 is plain halfway bounce-back),
  * steady momentum balance: drag on a held particle equals the body force on
    the fluid outside it (Eq. MP1 sign and factor 2),
  * the momentum ledger of a moving particle: exterior fluid + particle
    momentum changes only through the covered/uncovered bookkeeping,
  * exact lattice mass conservation (MP7 and MP8 add equal and opposite mass),
  * the Newton-Euler update in closed form (Eqs. MP5, MP6, old-U position),
  * Newton's third law and repulsion for the LJ-type force (Eq. MP2).
"""
import numpy as np
import pytest

PI = np.pi


def _inside(nx, ny, px, py, R, x, y, perx=True, pery=True):
    dx = x - px
    dy = y - py
    if perx:
        while dx >= 0.5 * nx:
            dx -= nx
        while dx < -0.5 * nx:
            dx += nx
    if pery:
        while dy >= 0.5 * ny:
            dy -= ny
        while dy < -0.5 * ny:
            dy += ny
    return dx * dx + dy * dy < R * R


def _random_state(oracle, nx, ny, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    u = amp * rng.standard_normal((2, ny, nx))
    r = 1 + 0.1 * amp * rng.standard_normal((ny, nx))
    f0 = np.zeros((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f0[:, y, x] = oracle.feq(r[y, x], u[0, y, x], u[1, y, x])
    return f0


@pytest.mark.parametrize("px,py,R", [(7.3, 8.1, 3.7), (0.4, 15.6, 2.9), (15.5, 0.5, 4.0)])
def test_links_equal_brute_force(oracle, px, py, R):
    nx = ny = 16
    e, _, _ = oracle.lattice()
    solid = np.zeros((ny, nx), np.uint8)
    solid[3, 12] = 1
    d = oracle.Domain(oracle.make_params(nx=nx, ny=ny), solid=solid,
                      particles=[dict(x=px, y=py, R=R, rho_p=1.0)])
    expect = []
    for y in range(ny):
        for x in range(nx):
            if not _inside(nx, ny, px, py, R, x, y) or solid[y, x]:
                continue
            for k in range(1, 9):
                fx, fy = (x + e[k][0]) % nx, (y + e[k][1]) % ny
                if solid[fy, fx] or _inside(nx, ny, px, py, R, fx, fy):
                    continue
                expect.append((y * nx + x, k))
    node, dirs = d.links(0)
    assert sorted(zip(node.tolist(), dirs.tolist())) == sorted(expect)
    own = d.owner()
    for y in range(ny):
        for x in range(nx):
            assert (own[y, x] == 1) == _inside(nx, ny, px, py, R, x, y)


def test_held_particle_is_a_stationary_obstacle(oracle):
    nx, ny, R, c = 30, 26, 5.2, (13.4, 12.7)
    yy, xx = np.mgrid[0:ny, 0:nx]
    disk = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 < R * R
    f0 = _random_state(oracle, nx, ny, 5)
    base = dict(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.75, gx=2e-5)
    a = oracle.Domain(oracle.make_params(**base), f0=f0,
                      particles=[dict(x=c[0], y=c[1], R=R, rho_p=1.0, fixed=1)])
    b = oracle.Domain(oracle.make_params(**base), f0=f0, solid=disk.astype(np.uint8))
    a.step(60)
    b.step(60)
    fa, fb = a.populations(), b.populations()
    assert np.array_equal(fa[:, ~disk], fb[:, ~disk])


def test_steady_drag_equals_body_force(oracle):
    N, g = 32, 1e-5
    d = oracle.Domain(oracle.make_params(nx=N, ny=N, tau=0.8, gx=g),
                      particles=[dict(x=15.3, y=16.0, R=5.0, rho_p=1.0, fixed=1)])
    d.step(20000)
    dg = d.diag(0)
    rho = d.moments()[0]
    ext_mass = rho[d.owner() == 0].sum()
    assert dg[0] == pytest.approx(ext_mass * g, rel=5e-5)
    # symmetric about y = 16: no lift, no torque
    assert abs(dg[1]) < 1e-12 * dg[0] and abs(dg[2]) < 1e-10 * dg[0]


def test_moving_particle_momentum_ledger_and_mass(oracle):
    nx, ny = 40, 36
    d = oracle.Domain(oracle.make_params(nx=nx, ny=ny, tau=0.7), f0=_random_state(oracle, nx, ny, 0),
                      particles=[dict(x=17.2, y=18.7, R=6.3, rho_p=1.3, U=0.03, V=-0.02, Omega=0.004)])
    m0 = d.checks()[0]

    def Q():
        q = d.particles()[0]
        m = q["rho_p"] * PI * q["R"] ** 2
        return d.exterior_momentum() + m * np.array([q["U"], q["V"]])

    hist = []
    for _ in range(200):
        Qt = Q()
        d.step(1)
        hist.append((Qt, d.diag(0), d.particles()[0]))
    flips = 0
    for t in range(len(hist) - 1):
        Qt, dgt, _ = hist[t]
        Qt1, dgt1, _ = hist[t + 1]
        q1 = hist[t][2]  # state at t+1
        lhs = (Qt1 + dgt1[3:5]) - (Qt + dgt[3:5])
        rhs = -np.array([q1["U"], q1["V"]]) * (dgt1[11] - dgt1[12])
        assert np.abs(lhs - rhs).max() < 1e-13
        flips += dgt1[9] + dgt1[10]
    assert flips > 10  # the particle really crossed lattice nodes
    assert abs(d.checks()[0] - m0) / m0 < 1e-13


def test_newton_euler_closed_form(oracle):
    """Constant F, T, g for n steps with no link friction (Z = 0): U_n = U_0 + n a,
    x_n = x_0 + n U_0 + a n(n-1)/2 (Eqs. MP5, MP6, position from the old U)."""
    q = dict(x=10.0, y=5.0, R=4.0, rho_p=1.5, U=0.01, V=-0.002, Omega=0.003, theta=0.1)
    Fx, Fy, T, gx, gy = 2e-3, -1e-3, 5e-4, 1e-6, 2e-6
    m = 1.5 * PI * 16.0
    I = 0.5 * m * 16.0
    ax = Fx / m + (1.5 - 1.0) / 1.5 * gx
    ay = Fy / m + (1.5 - 1.0) / 1.5 * gy
    al = T / I
    s = dict(q)
    n = 25
    for _ in range(n):
        s, _ = oracle.newton_euler(s, Fx, Fy, T, gx, gy, 1.0)
    assert s["U"] == pytest.approx(q["U"] + n * ax, rel=1e-13)
    assert s["x"] == pytest.approx(q["x"] + n * q["U"] + ax * n * (n - 1) / 2, rel=1e-13)
    assert s["y"] == pytest.approx(q["y"] + n * q["V"] + ay * n * (n - 1) / 2, rel=1e-13)
    assert s["theta"] == pytest.approx(q["theta"] + n * q["Omega"] + al * n * (n - 1) / 2, rel=1e-13)
    held, xm = oracle.newton_euler(dict(q, fixed=1), Fx, Fy, T, gx, gy, 1.0, Z=(3.0, 0, 0, 3.0, 0, 50.0))
    assert held["x"] == q["x"] and held["U"] == q["U"]
    assert list(xm) == [q["U"], q["V"], q["Omega"]]


def test_newton_euler_mid_step_friction_closed_form(oracle):
    """Link friction z along x alone, constant force F: with the boundary velocity at
    mid-step, m (U1 - U0) = F - z (U0 + U1)/2, so U_n - F/z = r^n (U_0 - F/z) with
    r = (m - z/2)/(m + z/2), and the mid-step velocity is (U0 + U1)/2."""
    q = dict(x=3.0, y=4.0, R=5.0, rho_p=1.0, U=2e-3, V=0.0, Omega=0.0)
    m = PI * 25.0
    z, F = 22.7, 3e-4
    r = (m - z / 2) / (m + z / 2)
    s = dict(q)
    for n in range(1, 40):
        U0 = s["U"]
        s, xm = oracle.newton_euler(s, F, 0.0, 0.0, 0.0, 0.0, 1.0, Z=(z, 0, 0, 0, 0, 0))
        assert s["U"] == pytest.approx(F / z + r ** n * (q["U"] - F / z), rel=1e-12)
        assert xm[0] == pytest.approx(0.5 * (U0 + s["U"]), rel=1e-15)
        assert s["V"] == 0.0 and s["Omega"] == 0.0


def test_newton_euler_mid_step_keeps_white_noise_equipartition(oracle):
    """The fluctuation-dissipation balance of the link exchange: the fluid's
    populations at equilibrium give the motion-independent link force a variance of
    2 z kT per step (Var f_k = w_k rho0 kT / c_s^2 on each of the z = sum 2 rho0 w_k /
    c_s^2 e_kx^2 links).  For the update U1 = r U0 + g F the stationary variance is
    g^2 2 z kT / (1 - r^2); with the mid-step boundary velocity it is exactly kT / m
    for any z (an explicit update, u_b at t, would give kT / (m - z/2))."""
    m = PI * 25.0
    for z in (1.0, 22.7, 60.0, 300.0):
        base = dict(x=0.0, y=0.0, R=5.0, rho_p=1.0, U=0.0, V=0.0, Omega=0.0)
        s1, _ = oracle.newton_euler(dict(base, U=1.0), 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, Z=(z, 0, 0, 0, 0, 0))
        s2, _ = oracle.newton_euler(dict(base), 1.0, 0.0, 0.0, 0.0, 0.0, 1.0, Z=(z, 0, 0, 0, 0, 0))
        r, g = s1["U"], s2["U"]
        kT = 1.0
        var = g * g * 2.0 * z * kT / (1.0 - r * r)
        assert var * m / kT == pytest.approx(1.0, rel=1e-12)


def test_newton_euler_coupled_friction_solves_the_linear_system(oracle):
    """Full 3x3 friction (translation-rotation coupling of an asymmetric link set):
    (M + Z/2) X1 = (M - Z/2) X0 + F + m (1 - rho0/rho_p) g, checked against a
    general linear solver (the oracle uses Cramer's rule)."""
    rng = np.random.default_rng(3)
    B = rng.standard_normal((3, 3))
    Zm = B @ B.T * 5.0
    Z = (Zm[0, 0], Zm[0, 1], Zm[0, 2], Zm[1, 1], Zm[1, 2], Zm[2, 2])
    q = dict(x=1.0, y=2.0, R=6.0, rho_p=1.2, U=1e-3, V=-2e-3, Omega=3e-4)
    m = 1.2 * PI * 36.0
    Mm = np.diag([m, m, 0.5 * m * 36.0])
    F = np.array([1e-3, -4e-4, 2e-3])
    g = (2e-6, -1e-6)
    X0 = np.array([q["U"], q["V"], q["Omega"]])
    G = F + np.array([m * (0.2 / 1.2) * g[0], m * (0.2 / 1.2) * g[1], 0.0])
    expect = np.linalg.solve(Mm + 0.5 * Zm, (Mm - 0.5 * Zm) @ X0 + G)
    s, xm = oracle.newton_euler(q, *F, *g, 1.0, Z=Z)
    got = np.array([s["U"], s["V"], s["Omega"]])
    assert np.allclose(got, expect, rtol=1e-12, atol=0)
    assert np.allclose(xm, 0.5 * (X0 + expect), rtol=1e-12, atol=0)
    assert s["x"] == q["x"] + q["U"] and s["y"] == q["y"] + q["V"]


def test_lj_pair_repulsive_and_power_13(oracle):
    F1 = oracle.lj_pair_force((1.0, 0.0), (0.0, 0.0), 20.0, 2.5)
    assert F1[0] == pytest.approx(20.0 * (1 / 2.5) ** -13, rel=1e-14) and F1[1] == 0.0
    F2 = oracle.lj_pair_force((0.0, 0.0), (1.0, 1.0), 20.0, 2.5)
    assert F2[0] < 0 and F2[1] < 0 and F2[0] == pytest.approx(F2[1], rel=1e-15)
    assert np.hypot(*F2) == pytest.approx(20.0 * (np.sqrt(2) / 2.5) ** -13, rel=1e-13)


def test_lj_third_law_and_wall_repulsion(oracle):
    nx, ny = 48, 30
    p = oracle.make_params(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, lj_psi=1e-4, lj_rit=2.5)
    parts = [dict(x=15.2, y=14.6, R=5.0, rho_p=1.0, fixed=1), dict(x=26.9, y=15.3, R=5.5, rho_p=1.0, fixed=1),
             dict(x=38.0, y=4.6, R=4.5, rho_p=1.0, fixed=1)]
    d = oracle.Domain(p, particles=parts)
    d.step(1)
    F0, F1, F2 = d.diag(0)[6:8], d.diag(1)[6:8], d.diag(2)[6:8]
    assert np.linalg.norm(F0) > 0
    assert np.allclose(F0, -F1, rtol=1e-12, atol=0)
    assert F0[0] < 0 < F1[0]          # pushed apart along x
    assert F2[1] > 0 and abs(F2[0]) < 1e-12 * F2[1]  # pushed away from the lower wall


def test_centred_particle_feels_no_torque(oracle):
    N = 24
    d = oracle.Domain(oracle.make_params(nx=N, ny=N, tau=0.9),
                      particles=[dict(x=12.0, y=12.0, R=4.5, rho_p=1.0)])
    d.step(10)
    dg = d.diag(0)
    assert abs(dg[2]) < 1e-13 and np.abs(dg[0:2]).max() < 1e-13
