"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every step of the D2Q9 hot path runs in the CUDA library ``_lib/liblbm_gb300.so``;
this module only converts numpy arrays / torch tensors to pointers and raises
on error codes.  There is no CPU fallback: if the library is missing or cannot
be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LBM_OK = 0
ERRORS = {-1: "LBM_E_INVAL", -2: "LBM_E_NOMEM", -3: "LBM_E_CUDA", -4: "LBM_E_UNSTABLE",
          -5: "LBM_E_TIMEOUT", -6: "LBM_E_STATE", -7: "LBM_E_IO"}
STORES = {"f64": 0, "f32": 1, "f32s": 2, "f16s": 3, "bf16s": 4}
DIAG_N = 13

EXPORTED = [
    "lbm_create", "lbm_create_ensemble", "lbm_set_geometry", "lbm_add_particles", "lbm_set_populations",
    "lbm_get_populations", "lbm_step", "lbm_prepare_steps", "lbm_record_particles", "lbm_sync", "lbm_moments", "lbm_moments_device", "lbm_moments_async",
    "lbm_moments_async_wait", "lbm_particles", "lbm_particle_forces", "lbm_checks", "lbm_step_count",
    "lbm_save", "lbm_load", "lbm_autotune", "lbm_set_launch", "lbm_get_launch", "lbm_profile_steps", "lbm_time_stream", "lbm_fp64_fma_rate",
    "lbm_checks_noalloc", "lbm_set_wait_limit", "lbm_debug_fail_alloc", "lbm_last_error", "lbm_destroy",
]
NOALLOC_MAX_ROWS = 16384
PREPARE_MAX_STEPS = 256  # LBM_PREPARE_MAX_STEPS
PREPARE_SLOTS = 4        # LBM_PREPARE_SLOTS


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """Mirror of ``lbm_params`` (include/lbm.h)."""
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
        ("store", ctypes.c_int32), ("max_particles", ctypes.c_int32), ("store_scale", ctypes.c_double),
        ("kappa_pl", ctypes.c_double),
    ]


class Particle(ctypes.Structure):
    """Mirror of ``lbm_particle``."""
    _fields_ = [
        ("x", ctypes.c_double), ("y", ctypes.c_double), ("R", ctypes.c_double),
        ("rho_p", ctypes.c_double), ("U", ctypes.c_double), ("V", ctypes.c_double),
        ("Omega", ctypes.c_double), ("theta", ctypes.c_double),
        ("fixed", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None
_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_fp = _P(ctypes.c_float)
_vp = ctypes.c_void_p


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if needed); raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        L = ctypes.CDLL(path)
        sig = {
            "lbm_create": (ctypes.c_int, [_P(Params), _vp, _P(_vp)]),
            "lbm_create_ensemble": (ctypes.c_int, [ctypes.c_int, _P(Params), _vp, _P(_vp)]),
            "lbm_set_geometry": (ctypes.c_int, [_vp, ctypes.c_int, _P(ctypes.c_uint8)]),
            "lbm_add_particles": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _P(Particle)]),
            "lbm_set_populations": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
            "lbm_get_populations": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
            "lbm_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
            "lbm_prepare_steps": (ctypes.c_int, [_vp, ctypes.c_int64]),
            "lbm_record_particles": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
            "lbm_sync": (ctypes.c_int, [_vp]),
            "lbm_moments": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, _dp]),
            "lbm_moments_device": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
            "lbm_moments_async": (ctypes.c_int, [_vp, ctypes.c_int]),
            "lbm_moments_async_wait": (ctypes.c_int, [_vp, _fp, _fp, _fp]),
            "lbm_particles": (ctypes.c_int, [_vp, ctypes.c_int, _P(Particle), ctypes.c_int]),
            "lbm_particle_forces": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _dp]),
            "lbm_checks": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
            "lbm_step_count": (ctypes.c_int64, [_vp]),
            "lbm_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
            "lbm_load": (ctypes.c_int, [_vp, ctypes.c_char_p]),
            "lbm_autotune": (ctypes.c_int, [_vp, ctypes.c_int]),
            "lbm_set_launch": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
            "lbm_get_launch": (ctypes.c_int, [_vp, _P(ctypes.c_int64)]),
            "lbm_profile_steps": (ctypes.c_int, [_vp, ctypes.c_int64, _dp, _P(ctypes.c_int64)]),
            "lbm_time_stream": (ctypes.c_int, [_vp, ctypes.c_int32, _dp]),
            "lbm_fp64_fma_rate": (ctypes.c_int, [_vp, _dp]),
            "lbm_checks_noalloc": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.c_int32, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp]),
            "lbm_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_uint64]),
            "lbm_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int32]),
            "lbm_last_error": (ctypes.c_char_p, [_vp]),
            "lbm_destroy": (None, [_vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def make_params(**kw) -> Params:
    """Parameter block with neutral defaults; ``store`` may be a name from STORES."""
    d = dict(nx=16, ny=16, periodic_x=1, periodic_y=1, walls_y=0, inlet_outlet=0, tau=0.8, rho0=1.0,
             gx=0.0, gy=0.0, rho_in=1.0, rho_out=1.0, kT=0.0, seed=0, domain_id=0, power_law=0, n_pl=1.0,
             xi_pl=0.1, tau_min=0.5 + 1e-9, tau_max=1e9, lj_psi=0.0, lj_rit=2.5, store="f32s",
             max_particles=0, store_scale=1.0, kappa_pl=0.0)
    d.update(kw)
    if isinstance(d["store"], str):
        d["store"] = STORES[d["store"]]
    return Params(**d)


def particle_array(parts) -> "ctypes.Array[Particle]":
    arr = (Particle * max(len(parts), 1))()
    for i, p in enumerate(parts):
        for k in ("x", "y", "R", "rho_p", "U", "V", "Omega", "theta"):
            setattr(arr[i], k, float(p.get(k, 0.0)))
        arr[i].fixed = int(p.get("fixed", 0))
    return arr


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        a = a.reshape(shape)
    return a


class Context:
    """One ``lbm_ctx``: a domain (or an ensemble of domains) on the current GPU."""

    def __init__(self, params, stream=None, solids=None, particles=None):
        self.L = load()
        plist = params if isinstance(params, (list, tuple)) else [params]
        self.params = list(plist)
        self._pbuf = {}
        self.ndom = len(plist)
        arr = (Params * self.ndom)(*plist)
        h = ctypes.c_void_p()
        s = _stream_ptr(stream)
        if self.ndom == 1:
            rc = self.L.lbm_create(arr, s, ctypes.byref(h))
        else:
            rc = self.L.lbm_create_ensemble(self.ndom, arr, s, ctypes.byref(h))
        if rc != LBM_OK:
            raise LbmError(rc, self.L.lbm_last_error(None).decode())
        self.h = h
        if solids is not None:
            for d, sol in enumerate(solids if isinstance(solids, (list, tuple)) else [solids]):
                if sol is not None:
                    self.set_geometry(d, sol)
        if particles:
            plists = particles if isinstance(particles[0], (list, tuple)) else [particles]
            for d, pl in enumerate(plists):
                if pl:
                    self.add_particles(d, pl)

    def _ck(self, rc):
        if rc != LBM_OK and not (isinstance(rc, int) and rc > 0):
            raise LbmError(rc, self.L.lbm_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, dom=0):
        p = self.params[dom]
        return p.ny, p.nx

    def set_geometry(self, dom, solid):
        ny, nx = self.shape(dom)
        s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(ny, nx)
        self._ck(self.L.lbm_set_geometry(self.h, dom, s.ctypes.data_as(_P(ctypes.c_uint8))))

    def add_particles(self, dom, parts):
        arr = particle_array(parts)
        self._ck(self.L.lbm_add_particles(self.h, dom, len(parts), arr))

    def set_populations(self, f, dom=0):
        ny, nx = self.shape(dom)
        f = _f64(f, (9, ny, nx))
        self._ck(self.L.lbm_set_populations(self.h, dom, f.ctypes.data_as(_dp)))

    def populations(self, dom=0, out=None):
        ny, nx = self.shape(dom)
        out = np.empty((9, ny, nx)) if out is None else out
        self._ck(self.L.lbm_get_populations(self.h, dom, out.ctypes.data_as(_dp)))
        return out

    def step(self, n=1):
        self._ck(self.L.lbm_step(self.h, int(n)))

    def prepare_steps(self, n):
        """lbm_prepare_steps: build the step graphs of exactly n steps now (blocking)."""
        self._ck(self.L.lbm_prepare_steps(self.h, int(n)))

    def sync(self):
        self._ck(self.L.lbm_sync(self.h))

    @property
    def step_count(self):
        return int(self.L.lbm_step_count(self.h))

    def moments(self, dom=0):
        ny, nx = self.shape(dom)
        rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
        self._ck(self.L.lbm_moments(self.h, dom, rho.ctypes.data_as(_dp), ux.ctypes.data_as(_dp),
                                    uy.ctypes.data_as(_dp)))
        return rho, ux, uy

    def moments_device(self, rho, ux, uy, dom=0):
        """Write FP32 moments into three caller device buffers (e.g. torch tensors)."""
        ptr = [t.data_ptr() if hasattr(t, "data_ptr") else int(t) for t in (rho, ux, uy)]
        self._ck(self.L.lbm_moments_device(self.h, dom, *[ctypes.c_void_p(p) for p in ptr]))

    def moments_async(self, dom=0):
        self._ck(self.L.lbm_moments_async(self.h, dom))

    def moments_async_wait(self, dom=0):
        ny, nx = self.shape(dom)
        rho, ux, uy = (np.empty((ny, nx), dtype=np.float32) for _ in range(3))
        self._ck(self.L.lbm_moments_async_wait(self.h, rho.ctypes.data_as(_fp), ux.ctypes.data_as(_fp),
                                               uy.ctypes.data_as(_fp)))
        return rho, ux, uy

    def particles(self, dom=0):
        cap = max(int(self.params[dom].max_particles), 1)
        arr = (Particle * cap)()
        n = self._ck(self.L.lbm_particles(self.h, dom, arr, cap))
        keys = ("x", "y", "R", "rho_p", "U", "V", "Omega", "theta", "fixed")
        return [{k: getattr(arr[i], k) for k in keys} for i in range(n)]

    def particles_array(self, dom=0):
        """The same states as particles(), as a float64 array [n, 8] with columns x, y,
        R, rho_p, U, V, Omega, theta: one C call into a buffer kept between calls and
        one copy, for loops that read the particles every step."""
        buf = self._pbuf.get(dom)
        if buf is None:
            cap = max(int(self.params[dom].max_particles), 1)
            arr = (Particle * cap)()
            view = np.frombuffer(arr, dtype=np.float64).reshape(cap, 9)  # 8 doubles + the two int32 words
            buf = self._pbuf[dom] = (arr, view, cap)
        arr, view, cap = buf
        n = self._ck(self.L.lbm_particles(self.h, dom, arr, cap))
        return view[:n, :8].copy()

    def record_particles(self, buf, capacity=None):
        """lbm_record_particles: per-step particle states into `buf`, a page-locked float64
        host tensor (torch.empty(..., pin_memory=True)) of capacity x np_slots x 6 values
        (x, y, U, V, Omega, theta); None stops recording.  Record (t mod capacity) holds the
        states after step t."""
        if buf is None:
            self._ck(self.L.lbm_record_particles(self.h, None, 0))
            return
        cap = int(capacity if capacity is not None else buf.shape[0])
        self._ck(self.L.lbm_record_particles(self.h, ctypes.c_void_p(buf.data_ptr()), cap))

    @property
    def particle_slots(self):
        """Particle slots of the context (sum of max_particles over the domains)."""
        return sum(int(p.max_particles) for p in self.params)

    def particle_forces(self, i, dom=0):
        out = np.zeros(DIAG_N)
        self._ck(self.L.lbm_particle_forces(self.h, dom, i, out.ctypes.data_as(_dp)))
        return out

    def checks(self, dom=0):
        out = np.zeros(3)
        self._ck(self.L.lbm_checks(self.h, dom, out.ctypes.data_as(_dp)))
        return out

    def save(self, path):
        self._ck(self.L.lbm_save(self.h, str(path).encode()))

    def load_checkpoint(self, path):
        self._ck(self.L.lbm_load(self.h, str(path).encode()))

    def profile_steps(self, n):
        """Run n steps with per-kernel CUDA events: (ms force launch, ms raster + LJ launches, ms stream-collide, launches)."""
        out = np.zeros(3)
        nl = ctypes.c_int64(0)
        self._ck(self.L.lbm_profile_steps(self.h, int(n), out.ctypes.data_as(_dp), ctypes.byref(nl)))
        return float(out[0]), float(out[1]), float(out[2]), int(nl.value)

    def time_stream(self, n):
        """Total device ms of n back-to-back stream-collide passes over every item (state not advanced)."""
        ms = ctypes.c_double(0.0)
        self._ck(self.L.lbm_time_stream(self.h, int(n), ctypes.byref(ms)))
        return float(ms.value)

    def autotune(self, trial_steps=20):
        self._ck(self.L.lbm_autotune(self.h, int(trial_steps)))

    def set_launch(self, kernel, block, stages=0):
        """Stream-collide kernel (0 register, 1 register persistent, 2 staged), threads per block, stages."""
        self._ck(self.L.lbm_set_launch(self.h, int(kernel), int(block), int(stages)))

    def launch(self):
        """(kernel, block, stages, grid) of the stream-collide launches."""
        out = (ctypes.c_int64 * 4)()
        self._ck(self.L.lbm_get_launch(self.h, out))
        return tuple(int(v) for v in out)

    def set_wait_limit(self, ns):
        """lbm_set_wait_limit: limit of the bounded device waits in ns (0: every stage wait expires at once)."""
        self._ck(self.L.lbm_set_wait_limit(self.h, int(ns)))


def debug_fail_alloc(nth):
    """lbm_debug_fail_alloc: the nth device allocation from now on fails (0: off)."""
    r = load().lbm_debug_fail_alloc(int(nth))
    if r != 0:
        raise LbmError(r, "lbm_debug_fail_alloc")


def _stream_ptr(stream):
    """A CUDA stream handle from a torch.cuda.Stream (its cuda_stream), an int, or None."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return ctypes.c_void_p(int(stream)) if int(stream) else None


def checks_noalloc(d_populations, store, nx, ny, pitch, rho0, store_scale, d_solid, d_out3, stream=None):
    """lbm_checks_noalloc on caller-owned device buffers (pointers or tensors) on `stream` (a
    torch.cuda.Stream, a raw handle or None); returns the status code."""
    def ptr(t):
        if t is None:
            return None
        return ctypes.c_void_p(t.data_ptr() if hasattr(t, "data_ptr") else int(t))
    L = load()
    st = STORES[store] if isinstance(store, str) else int(store)
    return L.lbm_checks_noalloc(ptr(d_populations), st, int(nx), int(ny), int(pitch), float(rho0),
                                float(store_scale), ptr(d_solid), ptr(d_out3), _stream_ptr(stream))


def fp64_fma_rate(stream=None):
    """lbm_fp64_fma_rate: the device's FP64 FMA rate in GFLOP/s (2 flops per FMA)."""
    L = load()
    g = ctypes.c_double(0.0)
    r = L.lbm_fp64_fma_rate(_stream_ptr(stream), ctypes.byref(g))
    if r != 0:
        raise LbmError(r, (L.lbm_last_error(None) or b"").decode())
    return float(g.value)
