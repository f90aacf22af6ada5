"""lbm_checks_noalloc: the global sums over caller-owned device buffers, with no
device allocation inside the library, must agree with lbm_checks on a context.

It is meant for callers that cannot allocate device memory (code running during
stream capture, stepping loops that cannot afford the synchronisation of
cudaMalloc / cudaFree, frameworks whose own pool owns the GPU).  Here the
caller's buffers are torch tensors laid out as the library lays out
populations; two calls in a row, on two different states, are compared with
the context's own checks, so stale scratch from the first call would show.
"""
import numpy as np
import pytest

from paper_2006_12910_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

WEIGHTS = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("store", ["f64", "f32s", "f16s", "bf16s"])
def test_noalloc_checks_match_context_checks_twice(torch_cuda, store):
    torch = torch_cuda
    nx, ny, pitch = 150, 70, 160
    scale = 4096.0 if store in ("f16s", "bf16s") else 1.0  # the scaled half kinds store (f - w rho0) * scale
    solid = workloads.disk_mask(nx, ny, [(40.3, 33.1, 9.2), (110.0, 20.5, 6.4)])
    params = lbm.make_params(nx=nx, ny=ny, periodic_x=1, periodic_y=0, walls_y=1, tau=0.8, gx=3e-5, store=store,
                             store_scale=scale)
    ctx = lbm.Context(params, solids=[solid])
    ctx.set_populations(workloads.random_populations(nx, ny, seed=4242, amp=0.02, solid=solid))
    dtype = {"f64": torch.float64, "f32s": torch.float32, "f16s": torch.float16, "bf16s": torch.bfloat16}[store]
    solid_t = torch.zeros((ny, pitch), dtype=torch.uint8, device="cuda")
    solid_t[:, :nx] = torch.from_numpy(solid.astype(np.uint8)).cuda()
    stream = torch.cuda.Stream()  # a torch stream object is accepted as the stream argument
    for call in range(2):
        ctx.step(7 + 5 * call)
        ref = ctx.checks()
        f = ctx.populations()
        # the stored values (exactly representable: they come from the store's own kind)
        vals = f if store == "f64" else (f - WEIGHTS[:, None, None]) * (solid == 0) * scale
        buf = torch.zeros((9, ny, pitch), dtype=dtype, device="cuda")
        buf[:, :, :nx] = torch.from_numpy(vals).to(device="cuda", dtype=dtype)
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = lbm.checks_noalloc(buf, store, nx, ny, pitch, 1.0, scale, solid_t, out, stream=stream)
        assert rc == 0
        stream.synchronize()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - ref[0]) <= 1e-12 * ref[0], (call, got, ref)
        assert np.abs(got[1:] - ref[1:]).max() <= 1e-12 * ref[0], (call, got, ref)
    ctx.close()


def test_noalloc_rejects_oversized_and_bad_arguments(torch_cuda):
    torch = torch_cuda
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    buf = torch.zeros(9 * 8 * 8, dtype=torch.float32, device="cuda")
    too_many = lbm.NOALLOC_MAX_ROWS + 1
    assert lbm.checks_noalloc(buf, "f32s", 8, too_many, 8, 1.0, 1.0, None, out) == -1
    assert lbm.checks_noalloc(buf, "f32s", 8, 8, 4, 1.0, 1.0, None, out) == -1   # pitch < nx
    assert lbm.checks_noalloc(None, "f32s", 8, 8, 8, 1.0, 1.0, None, out) == -1
    assert lbm.checks_noalloc(buf, "f16s", 8, 8, 8, 1.0, 0.0, None, out) == -1   # no scale
    assert lbm.checks_noalloc(buf, "f32s", 8, 8, 8, 1.0, 1.0, None, out) == 0
    torch.cuda.synchronize()
    assert abs(out[0].item() - 64.0) < 1e-12  # rest state of 8x8 fluid nodes: mass = 64 rho0
