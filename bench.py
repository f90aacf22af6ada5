"""Benchmark of the D2Q9 hot path on GB300: MLUPS of the porous-medium workload.

Workload (one step = one full timestep of the hot path over the whole domain):
2048x1024 D2Q9 lattice, ~300 seeded disk obstacles R~U[8,24] (gap >= 4),
20 free disk particles R=10 with rho_p/rho = 1.05 (Ladd moving bounce-back,
momentum-exchange force, covered/uncovered nodes, LJ repulsion, FP64
Newton-Euler), Zou-He density ends 1.001 / 0.999, halfway walls in y, tau=0.7,
FP32 arithmetic on shifted FP32 storage.  MLUPS = nodes * steps / (1e6 s),
counting every node as the paper does (Sec. 7).

Prints ONE JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes (read + write) per full stream-collide launch come from the ncu summary of
# the bench workload under profiles/; it records the hash of the CUDA sources it was
# taken on, and the number is reported only while the sources still hash the same.
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_stream_collide_porous_2048x1024.md")

METRIC = "D2Q9 MLUPS and % HBM roofline, FP32/FP16-store vs FP64 path at stated error"
# FP64 operations of one BGK collision with the velocity-shift force (unshifted FP64
# store, no noise, no power law), an FMA counted as 2: 14 adds for the moments, 3 + 3
# for the two shifted velocity components, 4 for 3/2 u.u, 1 for 3 rho, 6 for the rest
# population, 4 x 16 for the four opposite pairs and 2 for the diagonal projections;
# plus one division (1/rho), not counted.
FP64_FLOPS_PER_NODE = 97
UNIT = "MLUPS"
STORE_BYTES = {"f64": 8, "f32": 4, "f32s": 4, "f16s": 2, "bf16s": 2}


def csrc_hash() -> str:
    """SHA-256 (first 16 hex digits) of the CUDA sources and the C header, in name order."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2006_12910_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    with open(os.path.join(ROOT, "include", "lbm.h"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, store: str):
    """(bytes per launch, note) from the profile summary when its source hash matches the
    current sources, else (None, why)."""
    try:
        with open(TRAFFIC_PROFILE) as fh:
            text = fh.read()
    except OSError:
        return None, "no profile summary"
    want = csrc_hash()
    got, val = None, None
    for line in text.splitlines():
        line = line.strip().strip("`")
        if line.startswith("source_hash:"):
            got = line.split(":", 1)[1].strip()
        if line.startswith(f"traffic_bytes_per_launch[{kernel},{store}]:"):
            val = float(line.split(":", 1)[1].strip())
    if val is None:
        return None, "no traffic line for this kernel and store"
    if got != want:
        return None, f"profile taken on sources {got}, current {want}"
    return val, f"ncu, sources {want}"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest of every rank's value (the job's time is its slowest rank's):
    an all-reduce over the default process group, or x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank: int, steps: int, ms: float, world: int) -> float:
    """Whole-job throughput of N replicas (weak scaling): every rank advances its own
    copy of the workload, so the job updates world x nodes per step in the slowest
    rank's time."""
    return world * nodes_per_rank * steps / (ms * 1e-3) / 1e6


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lbm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                c = [x.strip() for x in line.split(",")]
                if len(c) >= 9:
                    rows.append(c)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        mx = max(num(r[2]) for r in rows)
        pw = [num(r[3]) for r in rows]
        pmax = max(p for p in pw if p == p) if any(p == p for p in pw) else 0.0
        load = [s for s, p in zip(sm, pw) if p == p and p >= 0.5 * pmax] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": pmax}


def workload_name(w) -> str:
    return f"porous {w.nx}x{w.ny} D2Q9: {w.note}, tau={w.params['tau']}, walls y"


def porous_workload(nx=2048, ny=1024):
    from paper_2006_12910_gb300 import workloads
    return workloads.porous(nx, ny)


def cpu_oracle_mlups(w, budget_s: float, steps_hint: int | None = None, threads: int = 0):
    """Time the FP64 oracle, as it stands, on the host cores (or `threads` of them) for
    ~budget_s."""
    from oracle import oracle
    oracle.build()
    if threads > 0:
        oracle.set_threads(threads)
    p = oracle.make_params(nx=w.nx, ny=w.ny, **{k: v for k, v in w.params.items()
                                                 if k in {f[0] for f in oracle.Params._fields_}})
    d = oracle.Domain(p, solid=w.solid, particles=w.particles)
    t0 = time.perf_counter()
    d.step(1)
    t1 = time.perf_counter()
    per = max(t1 - t0, 1e-6)
    n = steps_hint or max(1, int(budget_s / per))
    t0 = time.perf_counter()
    d.step(n)
    t = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(cores)  # back to every core
    return w.nx * w.ny * n / t / 1e6, n, t, (threads if threads > 0 else cores)


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    # Each reference step is one oracle timestep over a scaled-down sample of the
    # porous workload, sized so that warmup + steps fit in about two minutes.
    from paper_2006_12910_gb300 import workloads
    total_steps = args.steps + args.warmup
    probe = workloads.porous(512, 256)
    from oracle import oracle
    oracle.build()
    pp = oracle.make_params(nx=probe.nx, ny=probe.ny, **{k: v for k, v in probe.params.items()
                                                         if k in {f[0] for f in oracle.Params._fields_}})
    dprobe = oracle.Domain(pp, solid=probe.solid, particles=probe.particles)
    t0 = time.perf_counter()
    dprobe.step(2)
    rate = probe.nx * probe.ny * 2 / max(time.perf_counter() - t0, 1e-6)  # node updates per second
    budget = 100.0
    nodes = max(64 * 64, min(2048 * 1024, int(rate * budget / max(total_steps, 1))))
    ny = int(max(32, min(1024, round((nodes / 2) ** 0.5 / 8) * 8)))
    nx = int(max(64, min(2048, round(nodes / ny / 8) * 8)))
    w = workloads.porous(nx, ny)
    full = porous_workload()
    p = oracle.make_params(nx=w.nx, ny=w.ny, **{k: v for k, v in w.params.items()
                                                 if k in {f[0] for f in oracle.Params._fields_}})
    d = oracle.Domain(p, solid=w.solid, particles=w.particles)
    d.step(args.warmup)
    t0 = time.perf_counter()
    d.step(args.steps)
    t = time.perf_counter() - t0
    value = w.nx * w.ny * args.steps / t / 1e6
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"{w.nx}x{w.ny} sample of the porous workload ({w.note}), FP64 oracle, "
              f"{args.steps} timed steps after {args.warmup} warm-up")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(full), "nodes": full.nx * full.ny,
                       "fluid_nodes": int((full.solid == 0).sum()), "store": "f64 (CPU oracle)",
                       "sample": f"{w.nx}x{w.ny}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def channel_bench(lbm, workloads, stream, steps: int):
    """The confined-channel fluctuating workload (3000 x 41 walled channel, one R = 7.5
    Brownian disk, kT = 5e-5, nu = 0.1; the shape of the paper's second benchmark): MLUPS
    of the graph-replayed step, shifted FP32 store, autotuned.  Its 8.9 MB of populations
    stay in L2, so no HBM roofline applies; its statistics are checked by the tests."""
    import torch
    w = workloads.confined_channel()
    p = lbm.make_params(nx=w.nx, ny=w.ny, store="f32s", max_particles=1, **w.params)
    ctx = lbm.Context(p, stream=stream.cuda_stream, particles=[w.particles])
    ctx.autotune(10)
    ctx.step(400)
    ctx.sync()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    busy_device(stream)
    a0.record(stream)
    ctx.step(steps)
    a1.record(stream)
    a1.synchronize()
    ctx.sync()
    ms = a0.elapsed_time(a1)
    out = {"workload": f"confined channel {w.nx}x{w.ny}: {w.note}", "nodes": w.nx * w.ny, "steps": steps,
           "MLUPS": w.nx * w.ny * steps / (ms * 1e-3) / 1e6, "us_per_step": ms * 1e3 / steps,
           "launch": list(ctx.launch())}
    ctx.close()
    return out


def grains_bench(lbm, workloads, stream, steps: int, peak: float):
    """The paper's first-benchmark shape (1620 x 1020 grains, periodic along the flow,
    walls across, diagonal force, 45 disks of radius 6.5 released near the inlet): MLUPS
    of the graph-replayed step and the HBM fraction of the stream-collide pass, shifted
    FP32 store, autotuned."""
    import torch
    w = workloads.grains()
    fluid = int((w.solid == 0).sum())
    p = lbm.make_params(nx=w.nx, ny=w.ny, store="f32s", max_particles=len(w.particles), **w.params)
    ctx = lbm.Context(p, stream=stream.cuda_stream, solids=[w.solid], particles=[w.particles])
    ctx.autotune(10)
    ctx.step(200)
    ctx.sync()
    k1 = ctx.time_stream(100) / 100
    gbs = fluid * 72 / (k1 * 1e-3) / 1e9
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    busy_device(stream)
    a0.record(stream)
    ctx.step(steps)
    a1.record(stream)
    a1.synchronize()
    ctx.sync()
    ms = a0.elapsed_time(a1)
    out = {"workload": f"grains {w.nx}x{w.ny}: {w.note}", "nodes": w.nx * w.ny, "fluid_nodes": fluid,
           "steps": steps, "MLUPS": w.nx * w.ny * steps / (ms * 1e-3) / 1e6, "us_per_step": ms * 1e3 / steps,
           "kernel_ms": k1, "kernel_GBs": gbs, "frac": gbs / peak, "launch": list(ctx.launch())}
    ctx.close()
    return out


def combined_bench(lbm, workloads, stream, steps: int, peak: float):
    """Every feature at once on the benchmark geometry (2048 x 1024 porous workload with
    its particles, plus a power-law fluid n = 0.75 and thermal noise kT = 1e-5): the HBM
    fraction of the stream-collide pass (its variant with noise and tau*) and MLUPS of the
    graph-replayed step, shifted FP32 store, autotuned.  This combination turns unstable
    after a few hundred steps (particles with the power law and noise together; each pair
    alone is stable), so the step is timed over a short window from rest and an instability
    inside it is reported instead of a number."""
    import torch
    w = workloads.combined()
    fluid = int((w.solid == 0).sum())
    p = lbm.make_params(nx=w.nx, ny=w.ny, store="f32s", max_particles=len(w.particles), **w.params)
    ctx = lbm.Context(p, stream=stream.cuda_stream, solids=[w.solid], particles=[w.particles])
    out = {"workload": f"combined {w.nx}x{w.ny}: {w.note}", "nodes": w.nx * w.ny, "steps": steps}
    try:
        ctx.autotune(10)
        ctx.step(16)
        ctx.sync()
        k1 = ctx.time_stream(100) / 100
        gbs = fluid * 72 / (k1 * 1e-3) / 1e9
        out.update(kernel_ms=k1, kernel_GBs=gbs, frac=gbs / peak)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        busy_device(stream)
        a0.record(stream)
        ctx.step(steps)
        a1.record(stream)
        a1.synchronize()
        ctx.sync()
        ms = a0.elapsed_time(a1)
        out.update(MLUPS=w.nx * w.ny * steps / (ms * 1e-3) / 1e6, us_per_step=ms * 1e3 / steps,
                   launch=list(ctx.launch()))
    except lbm.LbmError as e:
        out["error"] = str(e)
    ctx.close()
    return out


def ensemble_bench(lbm, workloads, stream, steps32: int, steps64: int, samples: int):
    """The 96-domain fluctuating-LB ensemble (uneven sizes, per-domain Philox seed and kT,
    one R = 5 Brownian disk each): all domains in one context and one launch per step
    (shifted FP32 store, autotuned, CUDA graph), against one FP64 context per domain
    (per-domain launches, each context on its own stream).  Both report aggregate MLUPS;
    the FP32 run also reports the equilibrium statistics of fluid and particles."""
    import torch
    ws = workloads.ensemble()
    nodes = sum(w.nx * w.ny for w in ws)

    def params(w, store):
        return lbm.make_params(nx=w.nx, ny=w.ny, store=store, max_particles=len(w.particles), **w.params)

    out = {"domains": len(ws), "nodes": nodes, "sizes": sorted({(w.nx, w.ny) for w in ws})}
    ctx = lbm.Context([params(w, "f32s") for w in ws], stream=stream.cuda_stream, particles=[w.particles for w in ws])
    ctx.autotune(10)
    ctx.step(500)
    ctx.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    busy_device(stream)
    e0.record(stream)
    ctx.step(steps32)
    e1.record(stream)
    e1.synchronize()
    ctx.sync()
    ms = e0.elapsed_time(e1)
    out["f32s_one_launch"] = {"MLUPS": nodes * steps32 / (ms * 1e-3) / 1e6, "steps": steps32,
                              "launch": list(ctx.launch())}
    # equilibrium statistics: <rho u_a^2> = kT per node (fluid), <U_a^2> = kT / M (disks)
    fl, pu = [], []
    for _ in range(samples):
        ctx.step(50)
        for d, w in enumerate(ws):
            kT = w.params["kT"]
            rho, ux, uy = ctx.moments(dom=d)
            fl.append((float((rho * ux * ux).mean()) / kT, float((rho * uy * uy).mean()) / kT))
            q = ctx.particles(dom=d)[0]
            M = q["rho_p"] * np.pi * q["R"] ** 2
            pu.append((q["U"] ** 2 * M / kT, q["V"] ** 2 * M / kT))
    fl = np.array(fl)
    pu = np.array(pu)
    out["fluid_rho_u2_over_kT"] = {"x": float(fl[:, 0].mean()), "y": float(fl[:, 1].mean()),
                                   "samples": int(len(fl))}
    # disk velocity samples 50 steps apart are treated as independent for the interval
    pm = pu.mean()
    out["particle_M_U2_over_kT"] = {"mean": float(pm), "ci95": float(1.96 * pu.std() / np.sqrt(pu.size)),
                                    "samples": int(pu.size)}
    ctx.close()
    # per-domain launches of the FP64 path
    side = [torch.cuda.Stream() for _ in ws]
    ctxs = [lbm.Context(params(w, "f64"), stream=side[d].cuda_stream, particles=[w.particles])
            for d, w in enumerate(ws)]
    for c in ctxs:
        c.step(20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in ctxs:
        c.step(steps64)
    for c in ctxs:
        c.sync()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out["f64_per_domain"] = {"MLUPS": nodes * steps64 / t / 1e6, "steps": steps64,
                             "timing": "wall clock around the enqueue of every context and a sync of all"}
    for c in ctxs:
        c.close()
    return out


def busy_device(stream, cycles: int = 1_000_000):
    """Keep the stream's device busy (about half a millisecond) before a timed region, so
    that the host has enqueued the timed launches by the time the start event fires: the
    events then bracket device work only, not the host's launch latency."""
    import torch
    with torch.cuda.stream(stream):
        torch.cuda._sleep(cycles)


def _timed_steps(ctx, stream, steps):
    """Device ms of `steps` graph-replayed steps on the context stream (CUDA events)."""
    import torch
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    busy_device(stream)
    a0.record(stream)
    ctx.step(steps)
    a1.record(stream)
    a1.synchronize()
    ctx.sync()
    return a0.elapsed_time(a1)


def power_law_bench(lbm, workloads, stream, peak: float, steps: int = 400):
    """The power-law channel (4096 x 256, walls in y, body force, xi = 0.01, tau* clamped to
    [0.51, 2.0]) for n = 0.5, 0.75, 1.5 and each store: MLUPS of the graph-replayed step and
    the HBM fraction of the stream-collide pass (its tau* variant).  Timed from rest over a
    short window.  At n = 1.5 the clamp holds the fluid at nu = 1/300 everywhere and g = 1e-6
    would drive the developed flow past Ma 1, so that case runs at g = 2e-8."""
    out = {}
    for n in (0.5, 0.75, 1.5):
        w = workloads.power_law(n, g=2e-8 if n == 1.5 else 1e-6)
        nodes = w.nx * w.ny
        row = {"workload": f"power-law channel {w.nx}x{w.ny}: {w.note}"}
        for store in ("f64", "f32s", "f16s", "bf16s"):
            scale = 4096.0 if store in ("f16s", "bf16s") else 1.0
            p = lbm.make_params(nx=w.nx, ny=w.ny, store=store, store_scale=scale, **w.params)
            ctx = lbm.Context(p, stream=stream.cuda_stream)
            ctx.autotune(5)
            ctx.step(50)
            ctx.sync()
            ms = _timed_steps(ctx, stream, steps)
            k1 = ctx.time_stream(50) / 50
            gbs = nodes * 2 * 9 * STORE_BYTES[store] / (k1 * 1e-3) / 1e9
            row[store] = {"MLUPS": nodes * steps / (ms * 1e-3) / 1e6, "kernel_ms": k1, "kernel_GBs": gbs,
                          "frac": gbs / peak, "steps": steps}
            ctx.close()
        out[f"n={n}"] = row
    return out


def flb_bench(lbm, workloads, stream, peak: float, steps: int = 2000, samples: int = 40):
    """The fluctuating-LB configuration (512 x 512 periodic, tau = 1, kT = 1e-5, one R = 5
    neutrally buoyant disk): MLUPS of the graph-replayed step, the HBM fraction of the
    stream-collide pass (its noise variant) and the fluid temperature <rho u^2>/kT."""
    w = workloads.flb()
    nodes = w.nx * w.ny
    p = lbm.make_params(nx=w.nx, ny=w.ny, store="f32s", max_particles=1, **w.params)
    ctx = lbm.Context(p, stream=stream.cuda_stream, particles=[w.particles])
    ctx.autotune(10)
    ctx.step(500)
    ctx.sync()
    ms = _timed_steps(ctx, stream, steps)
    k1 = ctx.time_stream(100) / 100
    gbs = nodes * 72 / (k1 * 1e-3) / 1e9
    kT = w.params["kT"]
    acc = np.zeros(2)
    for _ in range(samples):
        ctx.step(50)
        rho, ux, uy = ctx.moments()
        acc += ((rho * ux * ux).mean() / kT, (rho * uy * uy).mean() / kT)
    out = {"workload": f"flb {w.nx}x{w.ny}: {w.note}", "nodes": nodes, "steps": steps,
           "MLUPS": nodes * steps / (ms * 1e-3) / 1e6, "us_per_step": ms * 1e3 / steps,
           "kernel_ms": k1, "kernel_GBs": gbs, "frac": gbs / peak, "launch": list(ctx.launch()),
           "fluid_rho_u2_over_kT": (acc / samples).tolist()}
    ctx.close()
    return out


# ---- error against the FP64 oracle ------------------------------------------------------------
# The GPU side runs a fresh context from a workload's start for a few steps and keeps the host
# state; the oracle leg (below, with the CPU baseline) runs the oracle over the same steps and
# reports relative L2 errors over fluid nodes of rho - rho0, u and the shifted populations
# f - omega_i rho0 (the parts that carry the dynamics), and the largest particle-state difference.
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def gpu_snapshot(lbm, stream, w, store, steps):
    scale = 4096.0 if store in ("f16s", "bf16s") else 1.0
    p = lbm.make_params(nx=w.nx, ny=w.ny, store=store, store_scale=scale,
                        max_particles=len(w.particles), **w.params)
    ctx = lbm.Context(p, stream=stream.cuda_stream, solids=[w.solid] if w.solid is not None else None,
                      particles=[w.particles] if w.particles else None)
    ctx.step(steps)
    snap = {"f": ctx.populations(), "mom": ctx.moments(), "parts": ctx.particles(), "steps": steps}
    ctx.close()
    return snap


def state_errors(ref, snap, solid, rho0=1.0):
    fluid = np.ones(snap["f"].shape[1:], bool) if solid is None else (np.asarray(solid) == 0)

    def rel(a, b):
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))
    rest = (W9 * rho0)[:, None]
    r0, ux0, uy0 = (m[fluid] for m in ref["mom"])
    r1, ux1, uy1 = (m[fluid] for m in snap["mom"])
    out = {"steps": snap["steps"],
           "drho": rel(r1 - rho0, r0 - rho0),
           "u": rel(np.stack([ux1, uy1]), np.stack([ux0, uy0])),
           "fneq": rel(snap["f"][:, fluid] - rest, ref["f"][:, fluid] - rest)}
    if ref["parts"]:
        out["particle"] = max(abs(a[k] - b[k]) for a, b in zip(ref["parts"], snap["parts"])
                              for k in ("x", "y", "U", "V", "Omega"))
    return out


def oracle_reference(w, steps):
    """Part of the oracle leg: the FP64 oracle from the workload's start over `steps` steps."""
    from oracle import oracle
    oracle.build()
    keys = {f[0] for f in oracle.Params._fields_}
    p = oracle.make_params(nx=w.nx, ny=w.ny, **{k: v for k, v in w.params.items() if k in keys})
    d = oracle.Domain(p, solid=w.solid, particles=w.particles)
    d.step(steps)
    return {"f": d.populations(), "mom": d.moments(), "parts": d.particles()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--store", default="f32s", choices=list(STORE_BYTES))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--profile-steps", type=int, default=500)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-channel", action="store_true")
    ap.add_argument("--no-combined", action="store_true")
    ap.add_argument("--no-grains", action="store_true")
    ap.add_argument("--no-power-law", action="store_true")
    ap.add_argument("--no-flb", action="store_true")
    ap.add_argument("--no-errors", action="store_true",
                    help="skip the error against the FP64 oracle (part of the oracle leg)")
    ap.add_argument("--channel-steps", type=int, default=16000)
    ap.add_argument("--ensemble-steps", type=int, default=4000)
    ap.add_argument("--launch", default=None,
                    help="stream-collide kernel,block,stages (e.g. 1,128,0); skips the autotuner")
    ap.add_argument("--print-hash", action="store_true",
                    help="print the hash of the CUDA sources (the key of the profile's traffic figure) and exit")
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=1024)
    args = ap.parse_args()
    if args.print_hash:
        print(csrc_hash())
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2006_12910_gb300 import lbm

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()

    w = porous_workload(args.nx, args.ny)
    nodes = w.nx * w.ny
    fluid = int((w.solid == 0).sum())
    base = {k: v for k, v in w.params.items()}
    scale = 4096.0 if args.store in ("f16s", "bf16s") else 1.0

    def make_ctx(store):
        p = lbm.make_params(nx=w.nx, ny=w.ny, store=store, max_particles=len(w.particles), store_scale=scale, **base)
        return lbm.Context(p, stream=stream.cuda_stream, solids=[w.solid], particles=[w.particles])

    ctx = make_ctx(args.store)
    if args.launch:
        ctx.set_launch(*[int(v) for v in args.launch.split(",")])
    elif not args.no_autotune:
        ctx.autotune(20)
    # with particles: FAR and NEAR stream-collide passes, the particle force launch, the
    # rasterisation + marks launch and the Eq. MP2 launch
    kernels_per_step = 5 if w.particles else 1

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- device-timed region: W warm-up steps, then exactly K steps ----------------------
    # set-up of the step graphs for the timed count (one graph replays all K steps), as
    # a caller that repeats a step count does once
    if args.steps <= lbm.PREPARE_MAX_STEPS:
        ctx.prepare_steps(args.steps)
    ctx.step(args.warmup)
    ctx.sync()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
    smi_index = vis.split(",")[dev] if vis else str(dev)
    clocks = ClockSampler(smi_index)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    busy_device(stream)
    e0.record(stream)
    ctx.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    ctx.sync()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, device="cuda")
    value = job_mlups(nodes, args.steps, ms, world)

    # ---- per-kernel device time ----------------------------------------------------------------
    # The dominant kernel's launch duration: CUDA events on the context stream (the stream the
    # kernel is launched on) around back-to-back stream-collide passes over every work item.
    # profile_steps adds events around each launch of a step run in sequence (no overlap).
    n_ts = 200
    k1_ms = ctx.time_stream(n_ts) / n_ts
    kf, kl, kk, nl = ctx.profile_steps(args.profile_steps)
    S = STORE_BYTES[args.store]
    alg_bytes = fluid * 2 * 9 * S  # read 9 + write 9 populations per fluid node update
    peak, peak_kind = _peaks()
    achieved = alg_bytes / (k1_ms * 1e-3) / 1e9
    launch = ctx.launch()
    k1_name = "k_stream_staged" if launch[0] == 2 else "k_stream_collide"
    traffic, traffic_note = recorded_traffic(k1_name, args.store) if (w.nx, w.ny) == (2048, 1024) else \
        (None, "profile covers the 2048x1024 workload only")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": traffic_note, "kernel": k1_name, "peak_source": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "kernel_ms": k1_ms,
                "kernel_timing": f"CUDA events around {n_ts} back-to-back passes over every work item on the context stream",
                "kernel_ms_in_sequence": kk / args.profile_steps,
                "kernel_share": kk / max(kf + kl + kk, 1e-9),
                "particle_kernel_ms": kf / args.profile_steps,
                "particle_side_ms": kl / args.profile_steps,
                "step_overlap": "far stream-collide items run concurrently with the particle launches",
                # the whole step against the same bound: fluid-node updates per second x bytes per update
                "step_frac": fluid * args.steps / (ms * 1e-3) * 2 * 9 * S / 1e9 / peak}

    # ---- end to end through the C ABI with host buffers ------------------------------------
    # Upload the initial state from pinned host memory, then every step: advance and read
    # the particle state back to the host; finally read the moment fields back.
    e2e = None
    if rank == 0 or world > 1:
        # End to end through the C ABI with host buffers: upload of the FP64 state from
        # pinned memory, K steps whose particle states are written to a pinned host
        # trajectory buffer at every step (lbm_record_particles) and read by the host after
        # each call of `chunk` steps, the moments read back at the end.
        ctx2 = make_ctx(args.store)
        f0 = torch.empty((9, w.ny, w.nx), dtype=torch.float64, pin_memory=True)
        f0.numpy()[:] = ctx2.populations()
        K2 = args.e2e_steps
        chunk = min(args.steps, K2, lbm.PREPARE_MAX_STEPS)
        npart = len(w.particles)
        rec = torch.empty((chunk, ctx2.particle_slots, 6), dtype=torch.float64, pin_memory=True)
        ctx2.record_particles(rec)
        ctx2.prepare_steps(chunk)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2.set_populations(f0.numpy())
        done, umax = 0, 0.0
        while done < K2:
            n = min(chunk, K2 - done)
            ctx2.step(n)
            ctx2.sync()
            r = rec.numpy()
            umax = max(umax, float(np.abs(r[:, :npart, 2:4]).max()))  # every step's particle velocities
            done += n
        rho, ux, uy = ctx2.moments()
        t = time.perf_counter() - t0
        ctx2.record_particles(None)
        h2d = 9 * nodes * 8 / K2
        d2h = npart * 48 + 3 * nodes * 8 / K2
        e2e = {"value": world * nodes * K2 / t / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": K2, "max_particle_speed": umax,
               "what": (f"lbm_set_populations(pinned FP64) + K/{chunk} x [lbm_step({chunk}) with every step's "
                        "particle states written to pinned host memory (lbm_record_particles) + lbm_sync + host "
                        "read of the records] + lbm_moments")}
        # the same with a blocking particle read after every single step
        K3 = min(K2, 500)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2.set_populations(f0.numpy())
        for _ in range(K3):
            ctx2.step(1)
            ctx2.particles_array()
        ctx2.moments()
        t3 = time.perf_counter() - t0
        e2e["blocking_read_each_step"] = {
            "value": world * nodes * K3 / t3 / 1e6, "unit": UNIT, "steps": K3,
            "what": "lbm_set_populations + K x [lbm_step(1) + lbm_particles] + lbm_moments"}
        ctx2.close()

    # ---- other storage kinds on the same workload (short) ----------------------------------
    variants = {}
    if not args.no_variants and rank == 0:
        for store in ("f16s", "f64"):
            if store == args.store:
                continue
            scale = 4096.0 if store in ("f16s", "bf16s") else 1.0
            c3 = make_ctx(store)
            if not args.no_autotune:
                c3.autotune(10)
            n3 = 2000 if store != "f64" else 500
            c3.step(50)
            c3.sync()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            busy_device(stream)
            a0.record(stream)
            c3.step(n3)
            a1.record(stream)
            a1.synchronize()
            c3.sync()
            m3 = a0.elapsed_time(a1)
            k3 = c3.time_stream(100) / 100
            b3 = fluid * 2 * 9 * STORE_BYTES[store]
            variants[store] = {"MLUPS": nodes * n3 / (m3 * 1e-3) / 1e6, "kernel_ms": k3,
                               "kernel_GBs": b3 / (k3 * 1e-3) / 1e9,
                               "frac": b3 / (k3 * 1e-3) / 1e9 / peak}
            if store == "f64":
                # FP64 arithmetic roofline: the collision's FP64 flops per fluid node (an FMA
                # counts 2; the one division per node not counted) against the device's FP64
                # FMA rate measured now by the library's probe.
                fp64_peak = lbm.fp64_fma_rate(stream.cuda_stream)
                achieved_gf = fluid * FP64_FLOPS_PER_NODE / (k3 * 1e-3) / 1e9
                variants[store]["alu"] = {"bound": "fp64", "flops_per_node": FP64_FLOPS_PER_NODE,
                                          "achieved_gflops": achieved_gf, "peak_gflops": fp64_peak,
                                          "frac": achieved_gf / fp64_peak,
                                          "hbm_floor_ms": b3 / (peak * 1e9) * 1e3,
                                          "alu_floor_ms": fluid * FP64_FLOPS_PER_NODE / (fp64_peak * 1e9) * 1e3}
            c3.close()

    ens = None
    if rank == 0 and not args.no_ensemble:
        from paper_2006_12910_gb300 import workloads as _wl
        ens = ensemble_bench(lbm, _wl, stream, args.ensemble_steps, max(100, args.ensemble_steps // 20), 20)

    chan = None
    if rank == 0 and not args.no_channel:
        from paper_2006_12910_gb300 import workloads as _wl
        chan = channel_bench(lbm, _wl, stream, args.channel_steps)

    grains = None
    if rank == 0 and not args.no_grains:
        from paper_2006_12910_gb300 import workloads as _wl
        grains = grains_bench(lbm, _wl, stream, 4000, peak)

    comb = None
    if rank == 0 and not args.no_combined:
        from paper_2006_12910_gb300 import workloads as _wl
        comb = combined_bench(lbm, _wl, stream, 200, peak)

    pl = None
    if rank == 0 and not args.no_power_law:
        from paper_2006_12910_gb300 import workloads as _wl
        pl = power_law_bench(lbm, _wl, stream, peak)

    flbk = None
    if rank == 0 and not args.no_flb:
        from paper_2006_12910_gb300 import workloads as _wl
        flbk = flb_bench(lbm, _wl, stream, peak)

    # GPU states for the error against the oracle: (label, workload, store, steps)
    snaps = []
    do_err = rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_errors
    if do_err:
        from paper_2006_12910_gb300 import workloads as _wl
        specs = [("headline", w, args.store, 20)]
        specs += [(f"variant:{st}", w, st, 20) for st in variants]
        if grains is not None:
            specs.append(("grains", _wl.grains(), "f32s", 10))
        if chan is not None:
            specs.append(("channel", _wl.confined_channel(), "f32s", 10))
        if comb is not None:
            specs.append(("combined", _wl.combined(), "f32s", 10))
        if flbk is not None:
            specs += [("flb", _wl.flb(), st, 10) for st in ("f32s", "f16s")]
        if pl is not None:
            for n in (0.5, 0.75, 1.5):
                # an x-periodic 64-wide copy of the 256-high channel: the flow is x-invariant
                wn = _wl.power_law(n, nx=64, ny=256, g=2e-8 if n == 1.5 else 1e-6)
                specs += [(f"power_law:n={n}", wn, st, 500) for st in ("f64", "f32s", "f16s", "bf16s")]
        for label, wk, st, k in specs:
            snaps.append((label, wk, st, gpu_snapshot(lbm, stream, wk, st, k)))

    cpu = None
    errors = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # ---- the oracle leg: CPU baseline and error against the oracle -----------------------
        v, n, t, cores = cpu_oracle_mlups(w, budget_s=15.0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} timesteps of the full 2048x1024 porous workload, FP64 oracle, OpenMP static"}
        v1, n1, t1, _ = cpu_oracle_mlups(w, budget_s=6.0, threads=1)
        cpu["single_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} timesteps of the same workload on one thread"}
        from paper_2006_12910_gb300 import workloads as _wl
        wf = _wl.porous(args.nx, args.ny)
        wf.particles = []
        v2, n2, t2, _ = cpu_oracle_mlups(wf, budget_s=8.0)
        cpu["without_particles"] = {"value": v2, "unit": UNIT, "cores": cores,
                                    "sample": f"{n2} timesteps of the porous workload with its particles "
                                              "removed (the oracle scans the whole lattice once per particle "
                                              "for the forces)"}
        refs = {}
        for label, wk, st, snap in snaps:
            key = (wk.name, wk.nx, wk.ny, snap["steps"])
            if key not in refs:
                refs[key] = oracle_reference(wk, snap["steps"])
            errors.setdefault(label, {})[st] = state_errors(refs[key], snap, wk.solid,
                                                            wk.params.get("rho0", 1.0))
        snaps.clear()
        refs.clear()
        for label, per in errors.items():
            if label.startswith("variant:"):
                variants[label.split(":", 1)[1]]["error_vs_oracle"] = per[label.split(":", 1)[1]]
            elif label == "grains" and grains is not None:
                grains["error_vs_oracle"] = per["f32s"]
            elif label == "channel" and chan is not None:
                chan["error_vs_oracle"] = per["f32s"]
            elif label == "combined" and comb is not None:
                comb["error_vs_oracle"] = per["f32s"]
            elif label == "flb" and flbk is not None:
                flbk["error_vs_oracle"] = per
            elif label.startswith("power_law:") and pl is not None:
                pl[label.split(":", 1)[1]]["error_vs_oracle"] = dict(
                    per, note="64x256 x-periodic copy of the channel, 500 steps from rest")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.store == "f64" else "f32", "data": "synthetic",
                "config": {"workload": workload_name(w),
                           "nodes": nodes, "fluid_nodes": fluid, "store": args.store,
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                           "l2": "no flush; per-step footprint (2 arenas) exceeds the 129 MB L2",
                           "launch": {"kernel": k1_name, "block": launch[1], "stages": launch[2],
                                      "grid": launch[3],
                                      "graphs": ("one prepared graph of the timed step count"
                                                 if args.steps <= lbm.PREPARE_MAX_STEPS
                                                 else "graphs of 2^j steps, one per binary digit of the count")}},
                "fluid_node_mlups": value * fluid / nodes,
                "clocks": clk, "gpu_launches": args.steps * kernels_per_step,
                "roofline": roofline, "e2e": e2e,
                "error_vs_oracle": errors.get("headline", {}).get(args.store),
                "variants": variants, "ensemble": ens, "channel": chan, "grains": grains, "combined": comb,
                "power_law": pl, "flb": flbk, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
