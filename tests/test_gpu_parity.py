"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

FP64 bar (element by element, every population): |gpu - oracle| <= 1e-12 |oracle|
after 100 steps on the same seeded inputs. Sizes span several 32 x 8 thread
blocks with ragged tails, single rows/columns and a single node. At the full
benchmark size the oracle checks sampled nodes one by one: the GPU state at t
gives the pre-collision populations of a node; the oracle collides them and the
result must appear, streamed by c_i, in the GPU state at t + 1.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
REL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    capi.load()
    yield
    torch.cuda.synchronize()


def gpu_run(f0, theta, tau, model, steps, prec="f64"):
    _, ny, nx = f0.shape
    with Lattice(nx, ny, theta, tau, model, prec) as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(steps)
        lat.sync()
        return lat.state().cpu().numpy()


def assert_rel(gpu, ref, rel, what=""):
    err = np.abs(gpu - ref) / np.abs(ref)
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= rel, f"{what}: max rel err {err.max():.3e} at {worst}"


SIZES = [(37, 23), (64, 64), (100, 3), (1, 5), (5, 1), (1, 1), (33, 9)]


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("model", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("theta", [0.25, 1.0 / 3.0, 0.4])
def test_random_state_parity_f64(oracle, nx, ny, model, theta):
    """Generic non-equilibrium populations, 100 steps, tau = 0.8."""
    f0 = flows.random_populations(nx, ny, seed=1000 + nx * 7 + ny + model, spread=0.2)
    ref = oracle.run(f0, theta, 0.8, model, 100)
    got = gpu_run(f0, theta, 0.8, model, 100)
    assert_rel(got, ref, REL_F64, f"{nx}x{ny} model {model} theta {theta:.3f}")


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4, 5])
def test_taylor_green_parity_f64(oracle, model):
    """Taylor-Green at 64^2, theta = 1/3, nu = 0.01, u0 = 0.05, through lbm_init and lbm_moments."""
    n, theta, nu, u0 = 64, 1.0 / 3.0, 0.01, 0.05
    tau = oracle.tau_from_nu(nu, theta)
    rho, ux, uy = flows.taylor_green(n, n, u0, theta)
    ref = oracle.run(oracle.init(rho, ux, uy, theta), theta, tau, model, 100)
    with Lattice(n, n, theta, tau, model) as lat:
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        f_init = lat.state().cpu().numpy()
        lat.step(100)
        got = lat.state().cpu().numpy()
        r, u, v = (a.cpu().numpy() for a in lat.moments())
    assert_rel(f_init, oracle.init(rho, ux, uy, theta), 1e-15, "init")
    assert_rel(got, ref, REL_F64, f"TG model {model}")
    r0, u0_, v0 = oracle.moments(ref)
    assert_rel(r, r0, 1e-13, "rho")
    np.testing.assert_allclose(u, u0_, rtol=0, atol=1e-13 * u0)
    np.testing.assert_allclose(v, v0, rtol=0, atol=1e-13 * u0)


@pytest.mark.parametrize("U", [0.0, 0.1, 0.2])
@pytest.mark.parametrize("theta", [0.25, 1.0 / 3.0, 0.4])
def test_shear_wave_parity_f64(oracle, U, theta):
    """Advected shear wave (u_y = 0.01 sin(2 pi x/nx), u_x = U), nu = 0.005, all four models."""
    nx, ny = 96, 10
    tau = oracle.tau_from_nu(0.005, theta)
    rho, ux, uy = flows.shear_wave(nx, ny, U=U, amp=0.01)
    f0 = oracle.init(rho, ux, uy, theta)
    for model in range(4):
        ref = oracle.run(f0, theta, tau, model, 100)
        if not np.isfinite(ref).all():
            continue  # unstable model at this (theta, U): nothing to compare
        got = gpu_run(f0, theta, tau, model, 100)
        assert_rel(got, ref, REL_F64, f"shear U={U} theta={theta:.3f} model {model}")


def test_zero_steps_and_time(oracle):
    f0 = flows.random_populations(20, 12, seed=5)
    with Lattice(20, 12, 0.35, 0.7, "complete") as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(0)
        assert lat.time == 0
        np.testing.assert_array_equal(lat.state().cpu().numpy(), f0)
        lat.step(3)
        assert lat.time == 3


def test_diagnostics_parity(oracle):
    """lbm_diagnostics and the fused in-step reduction against the oracle's compensated sums."""
    f0 = flows.random_populations(70, 45, seed=9)
    theta, tau = 0.37, 0.75
    with Lattice(70, 45, theta, tau, "complete") as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        d0 = np.array(lat.diagnostics())
        np.testing.assert_allclose(d0, oracle.diagnostics(f0), rtol=1e-13, atol=1e-13)
        lat.set_diagnostics_interval(5)
        lat.step(12)  # fused passes at t = 0, 5, 10
        out, t, status = lat.step_diagnostics()
        assert t == 10 and status == capi.LBM_OK
        ref10 = oracle.run(f0, theta, tau, 3, 10)
        np.testing.assert_allclose(out, oracle.diagnostics(ref10), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(lat.diagnostics(), oracle.diagnostics(oracle.run(f0, theta, tau, 3, 12)),
                                   rtol=1e-12, atol=1e-13)


def test_nonfinite_is_reported(oracle):
    """A NaN planted on the host is found by both diagnostics paths (LBM_ENONFINITE)."""
    f0 = flows.random_populations(40, 17, seed=3)
    f0[4, 6, 11] = np.nan
    with Lattice(40, 17, 1 / 3, 0.8, "partial") as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        d, status = capi.lbm_diagnostics(lat.ctx, raise_nonfinite=False)
        assert status == capi.LBM_ENONFINITE and d[4] == 1
        np.testing.assert_allclose(d, oracle.diagnostics(f0), rtol=1e-13)
        lat.set_diagnostics_interval(1)
        lat.step(1)
        with pytest.raises(capi.LBMError) as e:
            lat.sync()
        assert e.value.status == capi.LBM_ENONFINITE


def test_state_errors():
    with Lattice(8, 8, 1 / 3, 0.6, "lbgk") as lat:
        with pytest.raises(capi.LBMError) as e:
            lat.step(1)
        assert e.value.status == capi.LBM_ESTATE
        with pytest.raises(capi.LBMError) as e:
            capi.lbm_step(lat.ctx, -1)
        assert e.value.status == capi.LBM_EINVAL


def test_library_owned_buffers_match_torch_buffers(oracle):
    f0 = flows.random_populations(50, 20, seed=21)
    ref = gpu_run(f0, 0.3, 0.9, 3, 20)
    with Lattice(50, 20, 0.3, 0.9, "complete", torch_buffers=False) as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(20)
        np.testing.assert_array_equal(lat.state().cpu().numpy(), ref)


def test_set_stream_orders_new_work_after_old():
    """Steps queued on one stream, then the lattice rebound to a second stream: work on the
    second stream (reading the state back) sees every earlier step and diagnostics sum."""
    n, steps = 1024, 60
    rho, ux, uy = flows.shear_wave(n, n, U=0.1, amp=0.01)
    ref_state = None
    for rebind in (False, True):
        first, second = torch.cuda.Stream(), torch.cuda.Stream()
        with Lattice(n, n, 1 / 3, 0.52, "complete", stream=first) as lat:
            lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
            lat.set_diagnostics_interval(1)
            lat.step(steps)  # asynchronous on `first`
            if rebind:
                lat.set_stream(second)
            got = lat.state()  # runs on the lattice's current stream
            diag, t, status = lat.step_diagnostics()
        torch.cuda.synchronize()
        if ref_state is None:
            ref_state, ref_diag = got.cpu().numpy(), diag
        else:
            np.testing.assert_array_equal(got.cpu().numpy(), ref_state)
            np.testing.assert_array_equal(diag, ref_diag)
            assert t == steps - 1 and status == capi.LBM_OK


def test_inputs_from_the_current_stream_reach_a_lattice_on_its_own_stream():
    """A lattice bound to a side stream takes fields that torch is still producing on
    its current stream (queued behind a long matmul chain): init and set_state order
    the lattice's stream after that work, so the result equals the same run with
    every input ready."""
    n, steps = 512, 5
    rho, ux, uy = flows.shear_wave(n, n, U=0.1, amp=0.01)
    host = [torch.from_numpy(a) for a in (rho, ux, uy)]
    with Lattice(n, n, 1 / 3, 0.52, "complete") as ref:
        ref.init(*(h.cuda() for h in host))
        ref.step(steps)
        want = ref.state().cpu()
    side = torch.cuda.Stream()
    with Lattice(n, n, 1 / 3, 0.52, "complete", stream=side) as lat:
        for setter in ("init", "set_state"):
            torch.cuda.synchronize()
            busy = torch.randn(2048, 2048, device="cuda")
            for _ in range(30):
                busy = torch.tanh(busy @ busy)
            zero = busy[0, 0] * 0.0  # ready only after the chain
            if setter == "init":
                lat.init(*(h.cuda() + zero for h in host))
            else:
                with Lattice(n, n, 1 / 3, 0.52, "complete") as tmp:
                    tmp.init(*(h.cuda() for h in host))
                    f_eq = tmp.state()
                lat.set_state(f_eq + zero)
            lat.step(steps)
            np.testing.assert_array_equal(lat.state().cpu().numpy(), want.numpy())


def test_run_host_matches_device_path(oracle):
    """lbm_run_host (host buffers in and out) equals init + step + moments on the device."""
    n, theta, tau = 48, 1 / 3, 0.56
    rho, ux, uy = flows.taylor_green(n, n, 0.04, theta)
    with Lattice(n, n, theta, tau, "complete") as lat:
        out = [np.empty((n, n)) for _ in range(3)]
        diag = capi.lbm_run_host(lat.ctx, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data, 30,
                                 out[0].ctypes.data, out[1].ctypes.data, out[2].ctypes.data, want_diag=True)
        ref = oracle.run(oracle.init(rho, ux, uy, theta), theta, tau, 3, 30)
        for got, want in zip(out, oracle.moments(ref)):
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(diag, oracle.diagnostics(ref), rtol=1e-12, atol=1e-13)


def _one_step_sample_check(oracle, lat, theta, tau, model, nsamp, seed, rel):
    """Sampled one-step parity on a lattice of any size (no full-grid oracle run)."""
    nx, ny = lat.nx, lat.ny
    g = flows.rng(seed)
    xs = torch.from_numpy(g.integers(0, nx, nsamp)).cuda()
    ys = torch.from_numpy(g.integers(0, ny, nsamp)).cuda()
    f_t = lat.state()
    pre = f_t[:, ys, xs].cpu().numpy().T  # (nsamp, 9) pre-collision populations at t
    del f_t
    lat.step(1)
    f_t1 = lat.state()
    cx, cy = torch.tensor(CX).cuda(), torch.tensor(CY).cuda()
    xd = (xs[:, None] + cx[None, :]) % nx
    yd = (ys[:, None] + cy[None, :]) % ny
    post = f_t1[torch.arange(9).cuda()[None, :], yd, xd].cpu().numpy()  # f*_i(x, t) streamed to x + c_i
    del f_t1
    for k in range(nsamp):
        want = oracle.collide_node(pre[k], theta, tau, model)
        err = np.abs(post[k] - want) / np.abs(want)
        assert err.max() <= rel, f"node ({int(xs[k])}, {int(ys[k])}): rel err {err.max():.3e}"


@pytest.mark.parametrize("model", [0, 3])
def test_full_size_sampled_parity_f64(oracle, model):
    """4096^2 advected shear wave (U = 0.1, theta = 1/3, nu = 0.005) after 20 fused steps with
    diagnostics every step, as the benchmark runs it: 512 sampled nodes, one step, 1e-13."""
    n, theta = 4096, 1.0 / 3.0
    tau = oracle.tau_from_nu(0.005, theta)
    rho, ux, uy = flows.shear_wave(n, n, U=0.1, amp=0.01)
    with Lattice(n, n, theta, tau, model) as lat:
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        lat.set_diagnostics_interval(1)
        lat.step(20)
        d, t, status = lat.step_diagnostics()
        assert t == 19 and status == capi.LBM_OK
        assert d[0] == pytest.approx(n * n, rel=1e-13)            # mass conserved
        assert d[1] == pytest.approx(0.1 * n * n, rel=1e-12)      # momentum conserved (models 0, 3)
        _one_step_sample_check(oracle, lat, theta, tau, model, 512, 77 + model, 1e-13)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_checkpoint_resume(prec):
    """lbm_get_state / lbm_set_state as checkpoint and resume: a run split at t = 7 and resumed
    in a new lattice equals the uninterrupted run (the FP32 form after its own first rounding)."""
    n, theta, tau = 48, 1 / 3, 0.6
    rho, ux, uy = flows.taylor_green(n, n, 0.05, theta)
    fields = [torch.from_numpy(a).cuda() for a in (rho, ux, uy)]
    with Lattice(n, n, theta, tau, "complete", prec) as a:
        a.init(*fields)
        a.step(7)
        ckpt = a.state()
        a.step(13)
        want = a.state().cpu().numpy()
    with Lattice(n, n, theta, tau, "complete", prec) as b:
        b.set_state(ckpt)
        assert b.time == 0
        b.step(13)
        got = b.state().cpu().numpy()
    np.testing.assert_array_equal(got, want)


def test_vjp_and_batch_argument_errors():
    with Lattice(16, 16, 1 / 3, 0.6, "complete", "f16") as lat:
        z = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
        with pytest.raises(capi.LBMError) as e:
            capi.lbm_vjp(lat.ctx, 4, 2, z.data_ptr(), z.data_ptr(), z.data_ptr())
        assert e.value.status == capi.LBM_EINVAL
    with Lattice(16, 16, 1 / 3, 0.6, "lbgk_poly", "f64") as lat:
        with pytest.raises(capi.LBMError) as e:  # the polynomial-equilibrium LBGK has no adjoint
            capi.lbm_vjp(lat.ctx, 4, 2, z.data_ptr(), z.data_ptr(), z.data_ptr())
        assert e.value.status == capi.LBM_EINVAL and "LBGK_POLY" in str(e.value)
    with Lattice(16, 16, 1 / 3, 0.6, "complete", "f64") as lat:
        with pytest.raises(capi.LBMError):
            capi.lbm_vjp(lat.ctx, 4, 0, z.data_ptr(), z.data_ptr(), z.data_ptr())
        with pytest.raises(capi.LBMError):
            capi.lbm_set_launch_ex(lat.ctx, 0, 48, 4, 4)  # bx not a multiple of 32
        with pytest.raises(capi.LBMError):
            capi.lbm_set_launch_ex(lat.ctx, 2, 32, 4, 4)  # unknown kind


@pytest.mark.parametrize("model", [0, 3])
def test_full_size_sampled_parity_f64df(oracle, model):
    """The benchmark workload in the double-float form (FP64 storage): 20 fused steps with diagnostics
    every step, then 512 sampled nodes over one step against the oracle's collision, 2e-13 relative
    (one step of double-float rounding, about 2^-47 per operation)."""
    n, theta = 4096, 1.0 / 3.0
    tau = oracle.tau_from_nu(0.005, theta)
    rho, ux, uy = flows.shear_wave(n, n, U=0.1, amp=0.01)
    with Lattice(n, n, theta, tau, model, "f64df") as lat:
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        lat.set_diagnostics_interval(1)
        lat.step(20)
        d, t, status = lat.step_diagnostics()
        assert t == 19 and status == capi.LBM_OK
        assert d[0] == pytest.approx(n * n, rel=1e-13)
        assert d[1] == pytest.approx(0.1 * n * n, rel=1e-12)
        _one_step_sample_check(oracle, lat, theta, tau, model, 512, 91 + model, 2e-13)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_full_size_sampled_shifted_forms(oracle, prec):
    """The benchmark workload in the shifted forms (default launch, diagnostics every step): 512
    sampled nodes over one step against the oracle's FP64 collision of the same pre-collision values.
    Bound per population: storage rounding of the stored deviation (2^-24 FP32, 2^-11 FP16) plus a few
    FP32 ulps of the O(deviation) arithmetic, as k 2^-p max|f - rest| with k = 16 (FP32), 1.5 (FP16).
    FP32 runs two steps a launch by default: its first 20 steps are 10 such launches, the sampled
    step a single one, and the whole state after the 21 steps equals, bit for bit, 21 single steps
    of the persistent pipeline."""
    n, theta = 4096, 1.0 / 3.0
    tau = oracle.tau_from_nu(0.005, theta)
    rho, ux, uy = flows.shear_wave(n, n, U=0.1, amp=0.01)
    w0, w1 = 1 - theta, theta / 2
    rest = np.array([w0, w1, w0, w1, w0, w1, w1, w1, w1]) * np.array([w0, w0, w1, w0, w1, w1, w1, w1, w1])
    with Lattice(n, n, theta, tau, "complete", prec) as lat:
        assert capi.lbm_get_launch_ex(lat.ctx)[0] == (2 if prec == "f32" else 1)  # as benchmarked
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        lat.set_diagnostics_interval(1)
        lat.step(20)
        nx, ny = lat.nx, lat.ny
        g = flows.rng(55)
        xs = torch.from_numpy(g.integers(0, nx, 512)).cuda()
        ys = torch.from_numpy(g.integers(0, ny, 512)).cuda()
        pre = lat.state()[:, ys, xs].cpu().numpy().T
        lat.step(1)
        f1 = lat.state()
        cx, cy = torch.tensor(CX).cuda(), torch.tensor(CY).cuda()
        post = f1[torch.arange(9).cuda()[None, :], (ys[:, None] + cy[None, :]) % ny,
                  (xs[:, None] + cx[None, :]) % nx].cpu().numpy()
    if prec == "f32":
        with Lattice(n, n, theta, tau, "complete", prec) as one:
            capi.lbm_set_launch_ex(one.ctx, 1, 64, 1, 4)
            one.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
            one.set_diagnostics_interval(1)
            one.step(21)
            assert torch.equal(one.state(), f1)
    del f1
    k, p = (16, 24) if prec == "f32" else (1.5, 11)
    for j in range(512):
        want = oracle.collide_node(pre[j], theta, tau, 3)
        d = max(np.abs(pre[j] - rest).max(), np.abs(want - rest).max())
        assert np.abs(post[j] - want).max() <= k * 2.0 ** -p * d, f"node {j}"


@pytest.mark.parametrize("nx,ny,rows", [(37, 23, 5), (128, 16, 4), (130, 9, 3), (257, 12, 7), (1, 5, 2), (3, 4, 4),
                                        (45, 19, 8), (600, 33, 16)])
@pytest.mark.parametrize("model", [0, 3, 4, 5])
def test_fp64_pipeline_parity(oracle, nx, ny, rows, model):
    """FP64 through the bulk-copy pipeline (launch kind 1: 128-column tiles, one node a consumer
    thread): full and partial strips, narrow lattices whose rows share a ring slot, odd widths
    whose last main copy runs into the row padding, ragged row blocks; 100 steps against the
    oracle at the FP64 bar, and one fused diagnostics pass against the oracle's sums."""
    theta, tau = 0.35, 0.8
    f0 = flows.random_populations(nx, ny, seed=4100 + nx + 3 * ny + model, spread=0.2)
    with Lattice(nx, ny, theta, tau, model, "f64") as lat:
        capi.lbm_set_launch_ex(lat.ctx, 1, 0, 0, rows)
        assert capi.lbm_get_launch_ex(lat.ctx)[0] == 1
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(99)
        prev = lat.state().cpu().numpy()
        lat.set_diagnostics_interval(1)
        lat.step(1)
        d, t, status = lat.step_diagnostics()
        got = lat.state().cpu().numpy()
    ref = oracle.run(f0, theta, tau, model, 100)
    assert_rel(got, ref, REL_F64, f"pipeline {nx}x{ny} rows {rows} model {model}")
    assert t == 99 and status == 0
    np.testing.assert_allclose(d, oracle.diagnostics(prev), rtol=1e-12, atol=1e-13)


def test_fp64_pipeline_rejects_persistent_grid():
    with Lattice(64, 8, 1 / 3, 0.8, "complete", "f64") as lat:
        with pytest.raises(capi.LBMError) as e:
            capi.lbm_set_launch_ex(lat.ctx, 1, 2, 0, 8)
        assert e.value.status == capi.LBM_EINVAL


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_largest_lattice_sampled_parity(oracle, prec):
    """A 16384^2 lattice: each population buffer holds 2.4e9 elements (plane offsets beyond 2^31),
    stepped with the default launch of the form; 512 sampled nodes over one step against the
    oracle's collision (FP64 at 1e-13 relative; FP16 within its storage rounding as above)."""
    n, theta = 16384, 1.0 / 3.0
    tau = oracle.tau_from_nu(0.005, theta)
    rho, ux, uy = flows.shear_wave(n, n, U=0.1, amp=0.01)
    with Lattice(n, n, theta, tau, "complete", prec) as lat:
        assert 9 * lat.nx * lat.ny > 2 ** 31
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        del rho, ux, uy
        lat.set_diagnostics_interval(1)
        lat.step(2)
        d, t, status = lat.step_diagnostics()
        assert t == 1 and status == capi.LBM_OK and d[4] == 0
        assert d[0] == pytest.approx(n * n, rel=1e-12 if prec == "f64" else 1e-5)
        if prec == "f64":
            _one_step_sample_check(oracle, lat, theta, tau, 3, 512, 99, 1e-13)
            return
        theta_w = (1 - theta, theta / 2)
        rest = np.array([theta_w[0], theta_w[1], theta_w[0], theta_w[1], theta_w[0]] + [theta_w[1]] * 4) * \
            np.array([theta_w[0], theta_w[0], theta_w[1], theta_w[0], theta_w[1]] + [theta_w[1]] * 4)
        g = flows.rng(98)
        xs = torch.from_numpy(g.integers(0, n, 512)).cuda()
        ys = torch.from_numpy(g.integers(0, n, 512)).cuda()
        pre = lat.state()[:, ys, xs].cpu().numpy().T
        lat.step(1)
        cx, cy = torch.tensor(CX).cuda(), torch.tensor(CY).cuda()
        post = lat.state()[torch.arange(9).cuda()[None, :], (ys[:, None] + cy[None, :]) % n,
                           (xs[:, None] + cx[None, :]) % n].cpu().numpy()
    for j in range(512):
        want = oracle.collide_node(pre[j], theta, tau, 3)
        dev = max(np.abs(pre[j] - rest).max(), np.abs(want - rest).max())
        assert np.abs(post[j] - want).max() <= 1.5 * 2.0 ** -11 * dev, f"node {j}"
