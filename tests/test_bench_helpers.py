"""Host logic of the benchmark (no GPU): the source hash that keys the profile's
traffic figure, the reading of that figure, and the error measures against the
oracle."""
import os

import numpy as np

import bench


def test_source_hash_is_stable_and_short():
    h = bench.csrc_hash()
    assert h == bench.csrc_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_traffic_is_reported_only_for_matching_sources(tmp_path, monkeypatch):
    md = tmp_path / "k1.md"
    md.write_text("x\n    source_hash: 0000000000000000\n"
                  "    traffic_bytes_per_launch[k_stream_collide,f32s]: 123456789\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(md))
    val, note = bench.recorded_traffic("k_stream_collide", "f32s")
    assert val is None and "0000000000000000" in note
    md.write_text(f"source_hash: {bench.csrc_hash()}\n"
                  "traffic_bytes_per_launch[k_stream_collide,f32s]: 123456789\n")
    val, note = bench.recorded_traffic("k_stream_collide", "f32s")
    assert val == 123456789.0
    val, _ = bench.recorded_traffic("k_stream_collide", "f16s")
    assert val is None
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", os.path.join(str(tmp_path), "missing.md"))
    assert bench.recorded_traffic("k_stream_collide", "f32s")[0] is None


def test_state_errors_measure_the_shifted_parts():
    rng = np.random.default_rng(0)
    ny, nx = 6, 7
    f = bench.W9[:, None, None] * (1 + 0.01 * rng.standard_normal((9, ny, nx)))
    rho = f.sum(0)
    ux = (f[1] + f[5] + f[8] - f[3] - f[6] - f[7]) / rho
    uy = (f[2] + f[5] + f[6] - f[4] - f[7] - f[8]) / rho
    ref = {"f": f, "mom": (rho, ux, uy), "parts": [dict(x=1.0, y=2.0, U=0.1, V=0.0, Omega=0.0)]}
    snap = {"f": f.copy(), "mom": (rho.copy(), ux.copy(), uy.copy()), "steps": 3,
            "parts": [dict(x=1.0, y=2.0, U=0.1, V=0.0, Omega=0.0)]}
    e = bench.state_errors(ref, snap, None)
    assert e["drho"] == 0.0 and e["u"] == 0.0 and e["fneq"] == 0.0 and e["particle"] == 0.0
    # a change of 1e-9 in one population is 1e-9 of f but much more of f - w rho0
    snap["f"][4, 2, 3] += 1e-9
    e = bench.state_errors(ref, snap, None)
    fneq = f - bench.W9[:, None, None]
    assert abs(e["fneq"] - 1e-9 / np.linalg.norm(fneq)) < 1e-15
    solid = np.zeros((ny, nx), np.uint8)
    solid[2, 3] = 1  # the changed node is solid: excluded
    assert bench.state_errors(ref, snap, solid)["fneq"] == 0.0
