"""Seeded synthetic inputs for the D2Q9 hot path.

This module only draws inputs: obstacle masks, particle placements, initial
population fields and the workload definitions.  It holds none of the lattice
Boltzmann arithmetic, so the CUDA library and the FP64 oracle can both be fed
from it without sharing any of the method.

Workloads (arXiv:2006.12910 gives no dataset; every workload is a seeded
synthetic stand-in with the paper's parameters where it states them):

* ``poiseuille``   256x64 BGK channel, tau=0.8, g=1e-6 along x, periodic x,
                   halfway walls in y (Sec. 2; the paper's smooth channel).
* ``porous``       2048x1024, ~300 non-overlapping disk obstacles R~U[8,24]
                   (gap >= 4), 20 free disks R=10, rho_p/rho=1.05, density
                   inlet/outlet 1.001/0.999, tau=0.7, halfway walls in y
                   (stand-in for benchmark 1, Sec. 6, whose grain field exists
                   only as a missing figure).
* ``flb``          512x512 periodic fluctuating LB, tau=1, kT=1e-5, one R=5
                   neutrally buoyant disk at the centre (benchmark 2, Sec. 6).
* ``power_law``    4096x256 channel, g=1e-6, n in {0.5, 0.75, 1.5}, xi=0.01,
                   tau clamp [0.51, 2] (benchmark 3, Sec. 5-6).
* ``ensemble``     96 periodic fluctuating domains, sizes drawn from
                   {128x128, 256x128, 384x256, 512x512}, kT~U[5e-6, 2e-5],
                   one R=5 disk each.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 20061291

# Stiffness of the pairwise repulsion of Eq. MP2 per node pair, in lattice units.
# The paper's psi = 20 comes with a normalisation it does not state; summed over
# node pairs in lattice units it would change a particle's velocity by ~0.5 per
# step at first contact.  1e-4 stops a particle approaching at 1e-3 within about
# one lattice spacing.
LJ_PSI = 1e-4

# Relative sizes of the nine population slots of a fluid at rest (the shape
# of the input field only; both sides receive the resulting numbers).
_REST_SHAPE = np.array([16.0, 4.0, 4.0, 4.0, 4.0, 1.0, 1.0, 1.0, 1.0]) / 36.0


def random_populations(nx: int, ny: int, seed: int, amp: float = 0.01,
                       solid: np.ndarray | None = None) -> np.ndarray:
    """Positive population field f[9][ny][nx]: the rest shape times (1 + amp*N(0,1))
    with a smooth random large-scale component so that streaming moves real
    structure.  Solid nodes (if given) are zero."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((9, ny, nx))
    yy, xx = np.mgrid[0:ny, 0:nx]
    smooth = np.zeros((9, ny, nx))
    for i in range(9):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        smooth[i] = np.sin(2 * np.pi * (kx * xx / nx + ky * yy / ny) + ph)
    f = _REST_SHAPE[:, None, None] * (1.0 + amp * (0.5 * noise + smooth))
    if solid is not None:
        f[:, solid.astype(bool)] = 0.0
    return f


def disk_mask(nx: int, ny: int, disks) -> np.ndarray:
    """Nodes with (x-cx)^2 + (y-cy)^2 <= R^2 for any disk (cx, cy, R)."""
    yy, xx = np.mgrid[0:ny, 0:nx]
    m = np.zeros((ny, nx), dtype=bool)
    for cx, cy, R in disks:
        x0, x1 = max(int(np.floor(cx - R)) - 1, 0), min(int(np.ceil(cx + R)) + 2, nx)
        y0, y1 = max(int(np.floor(cy - R)) - 1, 0), min(int(np.ceil(cy + R)) + 2, ny)
        sub = (xx[y0:y1, x0:x1] - cx) ** 2 + (yy[y0:y1, x0:x1] - cy) ** 2 <= R * R
        m[y0:y1, x0:x1] |= sub
    return m.astype(np.uint8)


def place_obstacles(nx: int, ny: int, n: int, rmin: float, rmax: float, gap: float,
                    margin_y: float, margin_x: float, seed: int, max_tries: int = 200000):
    """Seeded rejection sampling of non-overlapping disks: radius ~U[rmin, rmax],
    centre uniform with the disk kept margin_y from the y-walls and margin_x
    from the open ends, surface gap >= gap between disks."""
    rng = np.random.default_rng(seed)
    disks: list[tuple[float, float, float]] = []
    tries = 0
    while len(disks) < n and tries < max_tries:
        tries += 1
        R = rng.uniform(rmin, rmax)
        cx = rng.uniform(margin_x + R, nx - 1 - margin_x - R)
        cy = rng.uniform(margin_y + R, ny - 1 - margin_y - R)
        ok = True
        for ox, oy, orad in disks:
            if (cx - ox) ** 2 + (cy - oy) ** 2 < (R + orad + gap) ** 2:
                ok = False
                break
        if ok:
            disks.append((cx, cy, R))
    return disks


def place_particles(nx: int, ny: int, n: int, R: float, rho_p: float, obstacles, gap: float,
                    margin_y: float, x_range: tuple[float, float], seed: int,
                    max_tries: int = 200000):
    """Free disks of radius R placed by rejection with surface gap >= gap from
    obstacles, walls and each other; centres uniform in x_range."""
    rng = np.random.default_rng(seed)
    parts: list[dict] = []
    tries = 0
    while len(parts) < n and tries < max_tries:
        tries += 1
        cx = rng.uniform(max(x_range[0], R + gap), min(x_range[1], nx - 1 - R - gap))
        cy = rng.uniform(margin_y + R + gap, ny - 1 - margin_y - R - gap)
        ok = all((cx - ox) ** 2 + (cy - oy) ** 2 >= (R + orad + gap) ** 2 for ox, oy, orad in obstacles)
        ok = ok and all((cx - p["x"]) ** 2 + (cy - p["y"]) ** 2 >= (2 * R + gap) ** 2 for p in parts)
        if ok:
            parts.append(dict(x=cx, y=cy, R=R, rho_p=rho_p, U=0.0, V=0.0, Omega=0.0, theta=0.0, fixed=0))
    return parts


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    params: dict
    solid: np.ndarray | None
    particles: list
    steps: int
    note: str = ""


def poiseuille(nx: int = 256, ny: int = 64) -> Workload:
    return Workload("poiseuille", nx, ny,
                    dict(periodic_x=1, periodic_y=0, walls_y=1, inlet_outlet=0, tau=0.8, rho0=1.0,
                         gx=1e-6, gy=0.0), None, [], 1000,
                    "D2Q9 BGK Poiseuille channel, rest start")


def porous(nx: int = 2048, ny: int = 1024, n_obstacles: int = 300, n_particles: int = 20,
           seed: int = BASE_SEED + 2) -> Workload:
    scale = (nx * ny) / (2048 * 1024)
    n_obs = max(1, int(round(n_obstacles * scale)))
    n_par = max(1, int(round(n_particles * scale))) if n_particles else 0
    rmin, rmax = (8.0, 24.0) if min(nx, ny) >= 256 else (2.0, 5.0)
    rpart = 10.0 if min(nx, ny) >= 256 else 3.5
    obstacles = place_obstacles(nx, ny, n_obs, rmin, rmax, gap=4.0, margin_y=2.0, margin_x=6.0, seed=seed)
    solid = disk_mask(nx, ny, obstacles)
    parts = place_particles(nx, ny, n_par, rpart, 1.05, obstacles, gap=4.5, margin_y=2.0,
                            x_range=(0.1 * nx, 0.6 * nx), seed=seed + 1000) if n_par else []
    return Workload("porous", nx, ny,
                    dict(periodic_x=0, periodic_y=0, walls_y=1, inlet_outlet=1, tau=0.7, rho0=1.0,
                         gx=0.0, gy=0.0, rho_in=1.001, rho_out=0.999, lj_psi=LJ_PSI, lj_rit=2.5),
                    solid, parts, 20000,
                    f"{len(obstacles)} obstacles R~U[{rmin},{rmax}] gap 4, {len(parts)} particles "
                    f"R={rpart} rho_p=1.05, Zou-He 1.001/0.999")


def flb(nx: int = 512, ny: int = 512, seed: int = BASE_SEED + 3, R: float = 5.0,
        kT: float = 1e-5) -> Workload:
    parts = [dict(x=nx / 2 + 0.3, y=ny / 2 + 0.2, R=R, rho_p=1.0, U=0.0, V=0.0, Omega=0.0, theta=0.0, fixed=0)] if R > 0 else []
    return Workload("flb", nx, ny,
                    dict(periodic_x=1, periodic_y=1, walls_y=0, inlet_outlet=0, tau=1.0, rho0=1.0,
                         gx=0.0, gy=0.0, kT=kT, seed=seed), None, parts, 50000,
                    f"periodic FLB kT={kT}, one R={R} disk")


def confined_channel(nx: int = 3000, ny: int = 41, seed: int = BASE_SEED + 6, R: float = 7.5,
                     kT: float = 5e-5, nu: float = 0.1, rho_p: float = 1.05) -> Workload:
    """Fluctuating fluid at rest in a narrow walled channel with one disk
    released on the centre line: the shape of the paper's second benchmark
    (3000 x 41, R = 7.5, kT = 5e-5, nu = 0.1, no external force).  The paper
    gives no particle density there; the disk takes the density ratio of its
    first benchmark, 1.05."""
    parts = [dict(x=nx / 2 + 0.3, y=(ny - 1) / 2.0 + 0.1, R=R, rho_p=rho_p, U=0.0, V=0.0, Omega=0.0, theta=0.0,
                  fixed=0)] if R > 0 else []
    return Workload("confined_channel", nx, ny,
                    dict(periodic_x=1, periodic_y=0, walls_y=1, inlet_outlet=0, tau=0.5 + 3.0 * nu, rho0=1.0,
                         gx=0.0, gy=0.0, kT=kT, seed=seed, lj_psi=LJ_PSI, lj_rit=2.5), None, parts, 800000,
                    f"walled channel FLB kT={kT} nu={nu}, one R={R} disk rho_p={rho_p} on the centre line")


def power_law(n: float, nx: int = 4096, ny: int = 256, g: float = 1e-6, xi: float = 0.01) -> Workload:
    return Workload(f"power_law_n{n}", nx, ny,
                    dict(periodic_x=1, periodic_y=0, walls_y=1, inlet_outlet=0, tau=1.0, rho0=1.0,
                         gx=g, gy=0.0, power_law=1, n_pl=n, xi_pl=xi, tau_min=0.51, tau_max=2.0),
                    None, [], 2000, f"power-law channel n={n} xi={xi} g={g}")


def combined(nx: int = 2048, ny: int = 1024, n_pl: float = 0.75, xi: float = 0.01, kT: float = 1e-5,
             seed: int = BASE_SEED + 7) -> Workload:
    """Every feature at once, the combination the paper names as untested: the
    porous workload's obstacles, particles and density-driven flow, with a
    power-law fluid (n, xi; tau* clamped to [0.51, 2.0]) and thermal noise."""
    w = porous(nx, ny)
    w.name = "combined"
    w.params.update(power_law=1, n_pl=n_pl, xi_pl=xi, tau_min=0.51, tau_max=2.0, kT=kT, seed=seed)
    w.note += f", power law n={n_pl} xi={xi}, kT={kT}"
    return w


def grains(nx: int = 1620, ny: int = 1020, n_obstacles: int = 236, seed: int = BASE_SEED + 8,
           release_x: float = 100.0) -> Workload:
    """The shape of the paper's first benchmark, turned so that the flow runs along x:
    a 1620-long periodic direction (inlet and outlet) between no-flow walls 1020
    apart, a Newtonian fluid with nu = 0.136 (tau = 0.908) driven by a diagonal body
    force (1e-5 along the flow, 1e-6 across), seeded disk grains R ~ U[8, 24] with a
    surface gap of 4 outside the release zone x < release_x, and 45 disks of radius
    6.5 (density ratio 1.05) released at rest near the inlet in two closely packed
    arrays: 23 and 22 disks across the channel with surface gaps of 8.5 between
    neighbours and 5.5 between the arrays (fewer when the channel is narrower)."""
    R = 6.5
    obstacles = [d for d in place_obstacles(nx, ny, n_obstacles, 8.0, 24.0, gap=4.0, margin_y=2.0, margin_x=6.0,
                                            seed=seed) if d[0] - d[2] > release_x]
    solid = disk_mask(nx, ny, obstacles)
    parts = []
    x0 = 40.0
    fit = int((ny - 2 * (R + 4.0)) // (2 * R + 8.5)) + 1  # disks that fit across a narrower channel
    for row, count in ((0, min(23, fit)), (1, min(22, fit - 1))):
        x = x0 + row * (2 * R + 5.5)
        span = (count - 1) * (2 * R + 8.5)
        for k in range(count):
            y = (ny - 1) / 2.0 - span / 2.0 + k * (2 * R + 8.5) + 0.25
            parts.append(dict(x=x, y=y, R=R, rho_p=1.05, U=0.0, V=0.0, Omega=0.0, theta=0.0, fixed=0))
    return Workload("grains", nx, ny,
                    dict(periodic_x=1, periodic_y=0, walls_y=1, inlet_outlet=0, tau=0.5 + 3 * 0.136, rho0=1.0,
                         gx=1e-5, gy=1e-6, lj_psi=LJ_PSI, lj_rit=2.5),
                    solid, parts, 56000,
                    f"{len(obstacles)} grains R~U[8,24] gap 4, {len(parts)} disks R=6.5 rho_p=1.05 released near the inlet, "
                    f"diagonal force (1e-5, 1e-6), periodic along the flow, walls across")


ENSEMBLE_SIZES = ((128, 128), (256, 128), (384, 256), (512, 512))


def ensemble(ndom: int = 96, seed: int = BASE_SEED + 5, sizes=ENSEMBLE_SIZES, R: float = 5.0):
    """Uneven ensemble: per-domain size, Philox seed and kT drawn from seed."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(ndom):
        nx, ny = sizes[int(rng.integers(0, len(sizes)))]
        kT = float(rng.uniform(5e-6, 2e-5))
        s = int(rng.integers(1, 2 ** 63 - 1))
        w = flb(nx, ny, seed=s, R=R, kT=kT)
        w.name = f"ensemble[{d}]"
        w.params["domain_id"] = d
        out.append(w)
    return out
