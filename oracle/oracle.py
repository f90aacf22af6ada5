"""ctypes wrapper of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The CUDA library never
imports, links or calls anything in this directory.

The oracle follows arXiv:2006.12910 Sec. 2 (Eqs. e.LB1-e.LB2), Sec. 3
(Eqs. MP1-MP8), Sec. 4 (Eqs. NP1-NP2, Table 1) and Sec. 5 (Eqs. nn1-nn5) in
plain double-precision loops; see ``lbm_oracle.h`` for the conventions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DIAG_N = 13


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP static loops)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wextra", "-Wno-unused-parameter", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("walls_y", ctypes.c_int32), ("inlet_outlet", ctypes.c_int32),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
        ("kT", ctypes.c_double), ("seed", ctypes.c_uint64), ("domain_id", ctypes.c_uint32),
        ("power_law", ctypes.c_int32), ("n_pl", ctypes.c_double), ("xi_pl", ctypes.c_double),
        ("tau_min", ctypes.c_double), ("tau_max", ctypes.c_double),
        ("lj_psi", ctypes.c_double), ("lj_rit", ctypes.c_double),
        ("kappa_pl", ctypes.c_double),
    ]


class Particle(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_double), ("y", ctypes.c_double), ("R", ctypes.c_double),
        ("rho_p", ctypes.c_double), ("U", ctypes.c_double), ("V", ctypes.c_double),
        ("Omega", ctypes.c_double), ("theta", ctypes.c_double),
        ("fixed", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_u8p = _P(ctypes.c_uint8)
_i32p = _P(ctypes.c_int32)
_u32p = _P(ctypes.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "or_create": (ctypes.c_void_p, [_P(Params)]),
                "or_destroy": (None, [ctypes.c_void_p]),
                "or_set_solid": (ctypes.c_int, [ctypes.c_void_p, _u8p]),
                "or_add_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _P(Particle)]),
                "or_init_equilibrium": (None, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
                "or_set_populations": (ctypes.c_int, [ctypes.c_void_p, _dp]),
                "or_get_populations": (None, [ctypes.c_void_p, _dp]),
                "or_step": (None, [ctypes.c_void_p, ctypes.c_int64]),
                "or_step_count": (ctypes.c_int64, [ctypes.c_void_p]),
                "or_moments": (None, [ctypes.c_void_p, _dp, _dp, _dp]),
                "or_get_particles": (ctypes.c_int, [ctypes.c_void_p, _P(Particle), ctypes.c_int]),
                "or_particle_diag": (None, [ctypes.c_void_p, ctypes.c_int, _dp]),
                "or_checks": (None, [ctypes.c_void_p, _dp]),
                "or_exterior_momentum": (None, [ctypes.c_void_p, _dp]),
                "or_links": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _i32p, _i32p, ctypes.c_int]),
                "or_owner": (None, [ctypes.c_void_p, _i32p]),
                "or_set_threads": (None, [ctypes.c_int]),
                "or_lattice": (None, [_i32p, _dp, _i32p]),
                "or_basis": (None, [_dp, _dp]),
                "or_feq": (None, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]),
                "or_solve_tau": (ctypes.c_double, [ctypes.c_double] * 5),
                "or_strain_A": (ctypes.c_double, [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
                "or_collide_node": (None, [_P(Params), _dp, _dp, ctypes.c_uint32, ctypes.c_uint32]),
                "or_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
                "or_thetas": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _dp]),
                "or_noise": (None, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]),
                "or_newton_euler": (None, [_P(Particle), _dp, _dp, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _dp]),
                "or_lj_pair_force": (None, [ctypes.c_double] * 6 + [_dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(_P(ct))


def make_params(**kw) -> Params:
    """Build an oracle parameter block; unspecified fields take neutral defaults."""
    d = dict(nx=16, ny=16, periodic_x=1, periodic_y=1, walls_y=0, inlet_outlet=0,
             tau=0.8, rho0=1.0, gx=0.0, gy=0.0, rho_in=1.0, rho_out=1.0, kT=0.0, seed=0,
             domain_id=0, power_law=0, n_pl=1.0, xi_pl=0.1, tau_min=0.5 + 1e-9,
             tau_max=1e9, lj_psi=0.0, lj_rit=2.5, kappa_pl=0.0)
    d.update(kw)
    return Params(**d)


def particle_array(parts) -> "ctypes.Array[Particle]":
    arr = (Particle * max(len(parts), 1))()
    for i, p in enumerate(parts):
        for k in ("x", "y", "R", "rho_p", "U", "V", "Omega", "theta"):
            setattr(arr[i], k, float(p.get(k, 0.0)))
        arr[i].fixed = int(p.get("fixed", 0))
    return arr


def particle_dicts(arr, n):
    keys = ("x", "y", "R", "rho_p", "U", "V", "Omega", "theta", "fixed")
    return [{k: getattr(arr[i], k) for k in keys} for i in range(n)]


class Domain:
    """One oracle lattice domain (post-collision populations f*(t), FP64)."""

    def __init__(self, params: Params, solid: np.ndarray | None = None, particles=None,
                 f0: np.ndarray | None = None):
        self.L = lib()
        self.p = params
        self.nx, self.ny = params.nx, params.ny
        h = self.L.or_create(ctypes.byref(params))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self.h = ctypes.c_void_p(h)
        if solid is not None:
            s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.ny, self.nx)
            self.L.or_set_solid(self.h, _ptr(s, ctypes.c_uint8))
        if f0 is not None:
            self.set_populations(f0)
        self.np = 0
        if particles:
            arr = particle_array(particles)
            self.overlaps = self.L.or_add_particles(self.h, len(particles), arr)
            self.np = len(particles)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.or_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        self.L.or_set_populations(self.h, _ptr(f, ctypes.c_double))

    def populations(self) -> np.ndarray:
        f = np.empty((9, self.ny, self.nx), dtype=np.float64)
        self.L.or_get_populations(self.h, _ptr(f, ctypes.c_double))
        return f

    def step(self, n: int = 1):
        self.L.or_step(self.h, int(n))

    @property
    def step_count(self) -> int:
        return int(self.L.or_step_count(self.h))

    def moments(self):
        shape = (self.ny, self.nx)
        rho, ux, uy = (np.empty(shape) for _ in range(3))
        self.L.or_moments(self.h, _ptr(rho, ctypes.c_double), _ptr(ux, ctypes.c_double),
                          _ptr(uy, ctypes.c_double))
        return rho, ux, uy

    def particles(self):
        arr = (Particle * max(self.np, 1))()
        n = self.L.or_get_particles(self.h, arr, self.np)
        return particle_dicts(arr, n)

    def diag(self, p: int) -> np.ndarray:
        out = np.zeros(DIAG_N)
        self.L.or_particle_diag(self.h, p, _ptr(out, ctypes.c_double))
        return out

    def checks(self) -> np.ndarray:
        out = np.zeros(3)
        self.L.or_checks(self.h, _ptr(out, ctypes.c_double))
        return out

    def exterior_momentum(self) -> np.ndarray:
        out = np.zeros(2)
        self.L.or_exterior_momentum(self.h, _ptr(out, ctypes.c_double))
        return out

    def links(self, p: int):
        n = self.L.or_links(self.h, p, None, None, 0)
        node = np.zeros(max(n, 1), dtype=np.int32)
        dirs = np.zeros(max(n, 1), dtype=np.int32)
        self.L.or_links(self.h, p, _ptr(node, ctypes.c_int32), _ptr(dirs, ctypes.c_int32), n)
        return node[:n], dirs[:n]

    def owner(self) -> np.ndarray:
        out = np.zeros((self.ny, self.nx), dtype=np.int32)
        self.L.or_owner(self.h, _ptr(out, ctypes.c_int32))
        return out


# ---- building blocks for the pin tests -------------------------------------------------

def lattice():
    e = np.zeros((9, 2), dtype=np.int32)
    w = np.zeros(9)
    opp = np.zeros(9, dtype=np.int32)
    lib().or_lattice(_ptr(e, ctypes.c_int32), _ptr(w, ctypes.c_double), _ptr(opp, ctypes.c_int32))
    return e, w, opp


def basis():
    chi = np.zeros((9, 9))
    wk = np.zeros(9)
    lib().or_basis(_ptr(chi, ctypes.c_double), _ptr(wk, ctypes.c_double))
    return chi, wk


def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().or_feq(rho, ux, uy, _ptr(out, ctypes.c_double))
    return out


def solve_tau(A, n, xi, tmin, tmax):
    return lib().or_solve_tau(A, n, xi, tmin, tmax)


def strain_A(f9, rho, jx, jy):
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    return lib().or_strain_A(_ptr(f9, ctypes.c_double), rho, jx, jy)


def collide_node(params: Params, f9, node=0, step=0):
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    out = np.zeros(9)
    lib().or_collide_node(ctypes.byref(params), _ptr(f9, ctypes.c_double), _ptr(out, ctypes.c_double),
                          node, step)
    return out


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def thetas(seed, node, step, domain=0):
    out = np.zeros(6)
    lib().or_thetas(seed, node, step, domain, _ptr(out, ctypes.c_double))
    return out


def noise(rho, kT, omega, theta6):
    th = np.ascontiguousarray(theta6, dtype=np.float64)
    out = np.zeros(9)
    lib().or_noise(rho, kT, omega, _ptr(th, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def newton_euler(particle: dict, Fx, Fy, T, gx, gy, rho0, Z=(0.0,) * 6):
    """One step of Eqs. MP5-MP6: returns (new particle dict, mid-step (U, V, Omega)).
    Z = upper triangle (xx, xy, xO, yy, yO, OO) of the link friction matrix."""
    arr = particle_array([particle])
    F = np.array([Fx, Fy, T], dtype=np.float64)
    Zv = np.ascontiguousarray(Z, dtype=np.float64)
    xm = np.zeros(3)
    lib().or_newton_euler(arr, _ptr(F, ctypes.c_double), _ptr(Zv, ctypes.c_double), gx, gy, rho0,
                          _ptr(xm, ctypes.c_double))
    return particle_dicts(arr, 1)[0], xm


def lj_pair_force(a, b, psi, rit):
    out = np.zeros(2)
    lib().or_lj_pair_force(a[0], a[1], b[0], b[1], psi, rit, _ptr(out, ctypes.c_double))
    return out


def set_threads(n: int):
    lib().or_set_threads(int(n))
