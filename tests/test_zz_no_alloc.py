"""lbm_step_noalloc, the entry point for callers that cannot allocate device memory.

Some callers may not call cudaMalloc: their device memory all comes from their
own pool, or an allocation's implicit synchronisation would stall their loop.
lbm_step_noalloc takes every buffer
from the caller and keeps its only scratch in a fixed device array. These tests
check it against the regular path (a lattice from lbm_create_ex advanced by
lbm_step with fused diagnostics) on the same state, for two calls in a row, and
check that an oversized lattice is refused with a clear message.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu

REL = 1e-12  # the FP64 parity tolerance of the other GPU tests


def _interior(buf, nx, ny, pitch, plane):
    """(9, ny, nx) view of a pitched FP64 population buffer."""
    return buf.reshape(9, plane)[:, : pitch * ny].reshape(9, ny, pitch)[:, :, :nx]


@pytest.mark.parametrize("model,nx,ny", [(3, 96, 40), (0, 37, 23), (2, 300, 70), (4, 64, 33)])
def test_noalloc_matches_regular_step_twice(model, nx, ny):
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    theta, tau = 0.37, 0.7
    pitch, plane, nbytes = capi.lbm_layout(nx, ny, capi.LBM_F64)
    f0 = flows.random_populations(nx, ny, seed=31 + model)
    stream = torch.cuda.current_stream()
    with Lattice(nx, ny, theta, tau, model, "f64", stream=stream) as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        raw = lat._buffers.view(torch.float64).view(2, 9 * plane)  # the lattice's ping-pong buffers
        src = raw[0].clone()  # state at t = 0, in the library's buffer convention
        dst = torch.full_like(src, float("nan"))
        diag = torch.full((5,), float("nan"), dtype=torch.float64, device=src.device)
        lat.set_diagnostics_interval(1)
        for call in range(2):
            lat.step(1)  # regular path: buffer (call + 1) % 2 now holds the state at t = call + 1
            ref_diag, t, status = lat.step_diagnostics()
            assert t == call and status == capi.LBM_OK
            capi.lbm_step_noalloc(nx, ny, theta, tau, model, src.data_ptr(), dst.data_ptr(), diag.data_ptr(),
                                  stream.cuda_stream)
            torch.cuda.synchronize()
            want = _interior(raw[(call + 1) % 2], nx, ny, pitch, plane).cpu().numpy()
            got = _interior(dst, nx, ny, pitch, plane).cpu().numpy()
            np.testing.assert_allclose(got, want, rtol=REL, atol=0)
            np.testing.assert_allclose(diag.cpu().numpy(), ref_diag, rtol=REL, atol=1e-13)
            src, dst = dst, src


def test_noalloc_large_lattice_grows_rows_per_thread():
    """A 4096 x 4096 lattice needs 16384 blocks at 4 rows per thread, more than the
    scratch holds, so the entry point doubles the rows per thread (to 8): the path
    of the large benchmark lattices. Two calls in a row against the regular path,
    compared on the device element by element at the same tolerance."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    nx = ny = 4096
    model, theta, tau = 3, 1.0 / 3.0, 0.52
    pitch, plane, nbytes = capi.lbm_layout(nx, ny, capi.LBM_F64)
    rho, ux, uy = flows.shear_wave(nx, ny, 0.1, 0.01)
    stream = torch.cuda.current_stream()
    with Lattice(nx, ny, theta, tau, model, "f64", stream=stream) as lat:
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        lat.step(4)  # a state off equilibrium; an even count leaves it in buffer 0
        raw = lat._buffers.view(torch.float64).view(2, 9 * plane)
        src = raw[0].clone()
        dst = torch.full_like(src, float("nan"))
        diag = torch.full((5,), float("nan"), dtype=torch.float64, device=src.device)
        lat.set_diagnostics_interval(1)
        for call in range(2):
            lat.step(1)
            ref_diag, _, status = lat.step_diagnostics()
            assert status == capi.LBM_OK
            capi.lbm_step_noalloc(nx, ny, theta, tau, model, src.data_ptr(), dst.data_ptr(), diag.data_ptr(),
                                  stream.cuda_stream)
            torch.cuda.synchronize()
            want = _interior(raw[(call + 1) % 2], nx, ny, pitch, plane)
            got = _interior(dst, nx, ny, pitch, plane)
            err = ((got - want).abs() / want.abs()).max().item()
            assert err <= REL, f"call {call}: max rel err {err:.3e}"
            np.testing.assert_allclose(diag.cpu().numpy(), ref_diag, rtol=REL, atol=1e-9)
            src, dst = dst, src


def test_noalloc_rejects_overlapping_buffers():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    nx, ny = 32, 16
    _, _, nbytes = capi.lbm_layout(nx, ny, capi.LBM_F64)
    buf = torch.zeros(2 * nbytes // 8 + 16, dtype=torch.float64, device="cuda")
    base = buf.data_ptr()
    # rejected on the host before any launch: the buffers are never touched
    for src, dst, diag in [(base, base + 8 * 64, base + 2 * nbytes),       # d_dst starts inside d_src
                           (base, base + nbytes, base + 8 * 10),           # d_diag5 inside d_src
                           (base, base + nbytes, base + nbytes + 8 * 3)]:  # d_diag5 inside d_dst
        with pytest.raises(capi.LBMError) as e:
            capi.lbm_step_noalloc(nx, ny, 1 / 3, 0.6, 3, src, dst, diag)
        assert e.value.status == capi.LBM_EINVAL and "overlap" in str(e.value)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    tiny = torch.zeros(16, dtype=torch.float64, device="cuda")
    other = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.LBMError) as e:
        # rejected on the host before any launch: the buffers are never touched
        capi.lbm_step_noalloc(16384, 16384, 1 / 3, 0.6, 3, tiny.data_ptr(), other.data_ptr(), tiny.data_ptr())
    assert e.value.status == capi.LBM_EINVAL
    assert "thread blocks" in str(e.value)
