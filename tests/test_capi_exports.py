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


def test_header_constants_match_the_binding():
    from paper_2006_12910_gb300 import lbm
    with open(os.path.join(ROOT, "include", "lbm.h")) as fh:
        txt = fh.read()
    defs = dict(re.findall(r"#define\s+(LBM_[A-Z_]+)\s+(\d+)", txt))
    assert int(defs["LBM_PREPARE_MAX_STEPS"]) == lbm.PREPARE_MAX_STEPS
    assert int(defs["LBM_PREPARE_SLOTS"]) == lbm.PREPARE_SLOTS


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
    assert L.lbm_prepare_steps(None, 20) == -1
    assert L.lbm_record_particles(None, None, 4) == -1
    assert L.lbm_step_count(None) == -1
    assert L.lbm_set_launch(None, 2, 128, 2) == -1
    assert L.lbm_get_launch(None, None) == -1
    assert L.lbm_time_stream(None, 4, None) == -1
    assert L.lbm_fp64_fma_rate(None, None) == -1


def _compiled_layout(tmp_path, header_dir, header, structs):
    """sizeof and offsetof of every field of the ctypes mirrors, as the host C
    compiler lays the C structs out."""
    import shutil
    import subprocess

    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = []
    for ctype, cls in structs:
        lines.append(f'printf("{ctype} sizeof %zu\\n", sizeof({ctype}));')
        for name, _ in cls._fields_:
            lines.append(f'printf("{ctype} {name} %zu\\n", offsetof({ctype}, {name}));')
    src = tmp_path / "layout.c"
    src.write_text(f'#include <stdio.h>\n#include <stddef.h>\n#include "{header}"\nint main(void) {{\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", header_dir, str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        ctype, name, value = line.split()
        got[(ctype, name)] = int(value)
    for ctype, cls in structs:
        assert got[(ctype, "sizeof")] == ctypes.sizeof(cls), ctype
        for name, _ in cls._fields_:
            assert got[(ctype, name)] == getattr(cls, name).offset, (ctype, name)


def test_binding_structs_match_the_header_as_compiled(tmp_path):
    """Every field of lbm_params and lbm_particle sits at the same offset in the
    binding's ctypes mirrors as in include/lbm.h compiled by the host C compiler."""
    from paper_2006_12910_gb300 import lbm
    _compiled_layout(tmp_path, os.path.join(ROOT, "include"), "lbm.h",
                     (("lbm_params", lbm.Params), ("lbm_particle", lbm.Particle)))


def test_oracle_structs_match_its_header_as_compiled(tmp_path):
    """The same for the oracle's parameter and particle blocks."""
    from oracle import oracle
    _compiled_layout(tmp_path, os.path.join(ROOT, "oracle"), "lbm_oracle.h",
                     (("or_params", oracle.Params), ("or_particle", oracle.Particle)))
