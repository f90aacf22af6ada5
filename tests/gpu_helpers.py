"""Shared set-up for the GPU parity tests: the same seeded inputs go to the FP64
oracle and to the CUDA library through its C ABI."""
import numpy as np

from oracle import oracle
from paper_2006_12910_gb300 import lbm, workloads

# Storage scale of the shifted half-precision kinds in the tests (power of two).
HALF_SCALE = 4096.0

# Relative-L2 tolerances over fluid nodes after the stated number of steps (see the
# tests): rho and u (the density and velocity criteria), the shifted populations
# f - omega_i rho0 (fneq: the part that carries the dynamics, undiluted by the rest
# value omega_i rho0), and rho - rho0 (drho), gated where the oracle's density
# deviation is resolvable (rms >= DRHO_MIN; a flow from rest in a closed channel keeps
# rho - rho0 at round-off, where a relative measure means nothing).
TOL = {
    "f64": dict(rho=1e-12, u=1e-12, f=1e-12, fneq=1e-11, drho=1e-11),
    # unshifted FP32 keeps f ~ omega_i with a 2^-24 ulp: every forcing increment of
    # ~1e-7 loses ~1 % to rounding, so this store cannot meet the FP32 bounds below
    # (u 1e-4); its bounds are the measured ones and it is reported, not held to them
    "f32": dict(rho=1e-5, u=1e-3, f=1e-5, fneq=2e-3, drho=1e-2),
    "f32s": dict(rho=1e-6, u=1e-4, f=1e-6, fneq=5e-5, drho=5e-5),
    "f16s": dict(rho=2e-5, u=5e-3, f=2e-5, fneq=5e-3, drho=5e-3),
    "bf16s": dict(rho=2e-4, u=5e-2, f=2e-4, fneq=5e-2, drho=5e-2),
}
DRHO_MIN = 1e-4

ORACLE_KEYS = {f[0] for f in oracle.Params._fields_}


def oracle_params(base: dict):
    return oracle.make_params(**{k: v for k, v in base.items() if k in ORACLE_KEYS})


def gpu_params(base: dict, store: str, max_particles: int = 0):
    kw = {k: v for k, v in base.items() if k in ORACLE_KEYS}
    return lbm.make_params(store=store, max_particles=max_particles,
                           store_scale=HALF_SCALE if store in ("f16s", "bf16s") else 1.0, **kw)


def pair(base: dict, store: str, solid=None, particles=None, f0=None):
    nx, ny = base["nx"], base["ny"]
    if f0 is None:
        f0 = workloads.random_populations(nx, ny, seed=1000 + nx + 7 * ny, amp=0.01, solid=solid)
    ref = oracle.Domain(oracle_params(base), solid=solid, particles=particles, f0=f0)
    ctx = lbm.Context(gpu_params(base, store, len(particles or [])), solids=[solid] if solid is not None else None,
                      particles=[particles] if particles else None)
    ctx.set_populations(f0)
    return ref, ctx


def rel(a, b, mask=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a = a[..., mask]
        b = b[..., mask]
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def compare_state(ref, ctx, store, solid=None, scale=1.0, rho0=1.0):
    """Relative L2 over fluid nodes, against the store's tolerance: rho and u (the
    density and velocity criteria), f, and the parts that carry the dynamics --
    rho - rho0 (drho) and the shifted populations f - omega_i rho0 (fneq), whose
    errors a comparison of rho ~ 1 and f ~ omega_i would dilute 100-1000 times."""
    fluid = None if solid is None else (np.asarray(solid) == 0)
    r0, ux0, uy0 = ref.moments()
    r1, ux1, uy1 = ctx.moments()
    f0, f1 = ref.populations(), ctx.populations()
    rest = (W9 * rho0)[:, None, None]
    e_rho = rel(r1, r0, fluid)
    e_u = rel(np.stack([ux1, uy1]), np.stack([ux0, uy0]), fluid)
    e_f = rel(f1, f0, fluid)
    e_drho = rel(r1 - rho0, r0 - rho0, fluid)
    e_fneq = rel(f1 - rest, f0 - rest, fluid)
    t = TOL[store]
    errs = dict(rho=e_rho, u=e_u, f=e_f, drho=e_drho, fneq=e_fneq)
    tols = {k: t[k] * scale for k in t}
    dr = (r0 - rho0) if fluid is None else (r0 - rho0)[fluid]
    if not (np.sqrt(np.mean(dr * dr)) >= DRHO_MIN):
        del tols["drho"]  # reported only
    return errs, tols


def assert_close(errs, tols, label=""):
    bad = {k: (errs[k], tols[k]) for k in tols if not (errs[k] <= tols[k])}
    assert not bad, f"{label}: {bad}"
