"""The seeded input generators: reproducible, and with the structure the
workloads state (sizes, gaps, counts, nothing overlapping)."""
import itertools

import numpy as np

from paper_2006_12910_gb300 import workloads


def _disks_clear(disks, gap):
    for (x1, y1, r1), (x2, y2, r2) in itertools.combinations(disks, 2):
        if np.hypot(x1 - x2, y1 - y2) < r1 + r2 + gap - 1e-9:
            return False
    return True


def test_generators_are_reproducible():
    a, b = workloads.porous(512, 256), workloads.porous(512, 256)
    assert np.array_equal(a.solid, b.solid) and a.particles == b.particles
    c, d = workloads.grains(540, 340, n_obstacles=26), workloads.grains(540, 340, n_obstacles=26)
    assert np.array_equal(c.solid, d.solid) and c.particles == d.particles


def test_porous_obstacles_and_particles_are_clear_of_each_other():
    w = workloads.porous()
    obstacles = workloads.place_obstacles(w.nx, w.ny, 300, 8.0, 24.0, gap=4.0, margin_y=2.0, margin_x=6.0,
                                          seed=workloads.BASE_SEED + 2)
    assert len(obstacles) == 300 and _disks_clear(obstacles, 4.0)
    assert len(w.particles) == 20
    disks = obstacles + [(p["x"], p["y"], p["R"]) for p in w.particles]
    assert _disks_clear(disks, 4.0)
    assert 0.10 < w.solid.mean() < 0.14


def test_grains_release_arrays_as_stated():
    w = workloads.grains()
    assert (w.nx, w.ny) == (1620, 1020) and len(w.particles) == 45
    xs = sorted({p["x"] for p in w.particles})
    assert len(xs) == 2 and xs[1] - xs[0] == 2 * 6.5 + 5.5  # surface gap 5.5 between the arrays
    for x in xs:
        ys = sorted(p["y"] for p in w.particles if p["x"] == x)
        assert np.allclose(np.diff(ys), 2 * 6.5 + 8.5)  # surface gap 8.5 within an array
    # no disk touches a grain or a wall
    yy, xx = np.mgrid[0:w.ny, 0:w.nx]
    for p in w.particles:
        near = (xx - p["x"]) ** 2 + (yy - p["y"]) ** 2 < (p["R"] + 2.5) ** 2
        assert not w.solid[near].any()
        assert p["R"] + 2.5 < p["y"] + 0.5 and p["y"] + p["R"] + 2.5 < w.ny - 0.5
    assert w.params["tau"] == 0.5 + 3 * 0.136 and (w.params["gx"], w.params["gy"]) == (1e-5, 1e-6)


def test_confined_channel_shape():
    w = workloads.confined_channel()
    assert (w.nx, w.ny) == (3000, 41) and w.params["kT"] == 5e-5 and w.params["gx"] == 0.0
    assert abs(w.params["tau"] - 0.8) < 1e-15  # nu = 0.1
    (p,) = w.particles
    assert p["R"] == 7.5 and abs(p["y"] - 20.0) < 0.5 and p["rho_p"] == 1.05


def test_ensemble_draws_per_domain_seeds_sizes_and_temperatures():
    ws = workloads.ensemble()
    assert len(ws) == 96
    assert {(w.nx, w.ny) for w in ws} <= set(workloads.ENSEMBLE_SIZES)
    assert len({w.params["seed"] for w in ws}) == 96
    kts = [w.params["kT"] for w in ws]
    assert min(kts) >= 5e-6 and max(kts) <= 2e-5
    assert [w.params["domain_id"] for w in ws] == list(range(96))
