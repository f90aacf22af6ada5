"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/lbm.h declares; argument validation happens before any CUDA call."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "lbm.h")) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    from paper_2006_12910_gb300 import lbm
    L = lbm.load()
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(L, n)]
    assert missing == []
    assert sorted(lbm.EXPORTED) == declared


def test_param_struct_layout_matches_header():
    from paper_2006_12910_gb300 import lbm
    # 6 int32, 6 double, kT, seed, domain_id + power_law, 6 doubles, store + max_particles, store_scale,
    # kappa_pl
    assert ctypes.sizeof(lbm.Params) == 24 + 48 + 8 + 8 + 8 + 48 + 8 + 8 + 8
    assert lbm.Params.kappa_pl.offset == 160
    assert ctypes.sizeof(lbm.Particle) == 8 * 8 + 8


def test_invalid_parameters_rejected_without_gpu():
    from paper_2006_12910_gb300 import lbm
    L = lbm.load()
    cases = [dict(nx=2), dict(tau=0.5), dict(periodic_x=1, inlet_outlet=1), dict(periodic_y=0, walls_y=0),
             dict(store=7), dict(kT=-1.0), dict(store="f16s", store_scale=0.0),
             dict(power_law=1, n_pl=0.5, xi_pl=0.01, tau_min=0.4, tau_max=2.0), dict(max_particles=-1)]
    for kw in cases:
        p = lbm.make_params(**kw)
        h = ctypes.c_void_p()
        assert L.lbm_create(ctypes.byref(p), None, ctypes.byref(h)) == -1, kw
        assert h.value is None
        assert L.lbm_last_error(None)
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_step_count(None) == -1
    assert L.lbm_set_launch(None, 2, 128, 2) == -1
    assert L.lbm_get_launch(None, None) == -1
    assert L.lbm_time_stream(None, 4, None) == -1
    assert L.lbm_fp64_fma_rate(None, None) == -1
