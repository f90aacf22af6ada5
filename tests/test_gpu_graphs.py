"""Step graphs: lbm_step(n) replays either one prepared graph of exactly n steps
(lbm_prepare_steps) or one graph per binary digit of n.  Every kernel of the
step is deterministic, so the two replays of the same steps must give the
same populations and particle states bit for bit, and both must match the
oracle on the porous workload with particles (the overlapped chains of
particle and stream-collide launches, drained at each graph's end)."""
import numpy as np
import pytest

from gpu_helpers import assert_close, compare_state, gpu_params, oracle_params
from paper_2006_12910_gb300 import lbm, workloads
from oracle import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _ctx(w, f0):
    ctx = lbm.Context(gpu_params(w.params | dict(nx=w.nx, ny=w.ny), "f32s", len(w.particles)), solids=[w.solid],
                      particles=[w.particles])
    ctx.set_populations(f0)
    return ctx


def test_prepared_graphs_replay_the_binary_graphs_bit_for_bit(errlog):
    w = workloads.porous(384, 192, n_obstacles=600, n_particles=120)
    assert len(w.particles) >= 2
    f0 = workloads.random_populations(w.nx, w.ny, seed=77, amp=0.005, solid=w.solid)
    a, b = _ctx(w, f0), _ctx(w, f0)
    for n in (20, 7, 3, 64, 65, 1):
        a.prepare_steps(n)
    # six counts were prepared: the two oldest (20 and 7) are no longer among
    # the LBM_PREPARE_SLOTS = 4 slots and fall back to the binary graphs
    counts = [20, 7, 7, 3, 65, 1, 20, 64, 7]
    for n in counts:
        a.step(n)
        b.step(n)
    fa, fb = a.populations(), b.populations()
    pa, pb = a.particles(), b.particles()
    assert a.step_count == b.step_count == sum(counts)
    assert np.array_equal(fa, fb)
    assert pa == pb
    ref = oracle.Domain(oracle_params(w.params | dict(nx=w.nx, ny=w.ny)), solid=w.solid, particles=w.particles,
                        f0=f0)
    ref.step(sum(counts))
    errs, tols = compare_state(ref, a, "f32s", w.solid)
    pr = ref.particles()
    perr = max(abs(x[k] - y[k]) for x, y in zip(pr, pa) for k in ("x", "y", "U", "V", "Omega"))
    errlog(steps=sum(counts), particle=perr, **errs)
    assert_close(errs, tols, "prepared graphs")
    assert perr < 1e-6
    a.close()
    b.close()


def test_prepare_rejects_counts_out_of_range():
    w = workloads.porous(256, 128, n_obstacles=100, n_particles=10)
    ctx = _ctx(w, workloads.random_populations(w.nx, w.ny, seed=5, amp=0.005, solid=w.solid))
    for n in (0, -3, lbm.PREPARE_MAX_STEPS + 1):
        with pytest.raises(lbm.LbmError):
            ctx.prepare_steps(n)
    ctx.prepare_steps(lbm.PREPARE_MAX_STEPS)
    ctx.step(2)
    ctx.sync()
    ctx.close()


def test_recorded_trajectories_equal_the_states_read_step_by_step():
    torch = pytest.importorskip("torch")
    w = workloads.porous(384, 192, n_obstacles=600, n_particles=120)
    f0 = workloads.random_populations(w.nx, w.ny, seed=78, amp=0.005, solid=w.solid)
    a, b = _ctx(w, f0), _ctx(w, f0)
    ns, cap = a.particle_slots, 8
    buf = torch.full((cap, ns, 6), float("nan"), dtype=torch.float64, pin_memory=True)
    a.record_particles(buf)
    a.prepare_steps(20)
    a.step(3)
    a.step(20)  # steps 4 .. 23: records of steps 16 .. 23 remain, at slots (t mod 8)
    a.sync()
    rec = buf.numpy().copy()
    seen = {}
    for t in range(1, 24):
        b.step(1)
        seen[t] = b.particles_array()
    for t in range(16, 24):
        want = seen[t][:, [0, 1, 4, 5, 6, 7]]  # x, y, U, V, Omega, theta
        assert np.array_equal(rec[t % cap, :len(want)], want), t
    assert np.isnan(rec[:, len(w.particles):]).all()  # slots beyond the particle count stay untouched
    # stop recording: later steps leave the buffer alone
    a.record_particles(None)
    before = buf.numpy().copy()
    a.step(5)
    a.sync()
    assert np.array_equal(buf.numpy(), before, equal_nan=True)
    a.close()
    b.close()


def test_record_rejects_pageable_memory_and_bad_capacity():
    torch = pytest.importorskip("torch")
    w = workloads.porous(256, 128, n_obstacles=100, n_particles=10)
    ctx = _ctx(w, workloads.random_populations(w.nx, w.ny, seed=6, amp=0.005, solid=w.solid))
    pageable = torch.zeros((4, ctx.particle_slots, 6), dtype=torch.float64)
    with pytest.raises(lbm.LbmError):
        ctx.record_particles(pageable)
    pinned = torch.zeros((4, ctx.particle_slots, 6), dtype=torch.float64, pin_memory=True)
    with pytest.raises(lbm.LbmError):
        ctx.record_particles(pinned, capacity=0)
    ctx.record_particles(pinned)
    ctx.step(4)
    ctx.sync()
    assert np.abs(pinned.numpy()[:, :1]).sum() > 0
    ctx.close()
