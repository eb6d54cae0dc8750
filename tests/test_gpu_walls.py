"""Fullway bounce-back walls (lbm_set_walls) through the C ABI against the FP64 oracle
with the same wall mask, and the isothermal shocktube of Sec. 5.2 built on them.

Bars: FP64 element by element |gpu - oracle| <= 1e-12 |oracle|; the shifted forms
within the linear rounding bound of tests/test_gpu_forms.py; the adjoint's
directional derivative against the oracle's complex step to 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, experiments, flows
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu

REL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    capi.load()
    yield
    torch.cuda.synchronize()


def random_walls(nx, ny, seed, frac=0.12):
    g = flows.rng(seed)
    w = (g.uniform(size=(ny, nx)) < frac).astype(np.uint8)
    w[:, 0] = 1  # a wall column, so that walls meet the periodic wrap too
    return w


def gpu_run(f0, theta, tau, model, steps, walls, prec="f64"):
    _, ny, nx = f0.shape
    with Lattice(nx, ny, theta, tau, model, prec) as lat:
        assert lat.set_walls(walls) == int((np.asarray(walls) != 0).sum())
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(steps)
        lat.sync()
        return lat.state().cpu().numpy()


def assert_rel(gpu, ref, rel, what=""):
    err = np.abs(gpu - ref) / np.abs(ref)
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= rel, f"{what}: max rel err {err.max():.3e} at {worst}"


@pytest.mark.parametrize("nx,ny", [(37, 23), (64, 17), (5, 1), (130, 3)])
@pytest.mark.parametrize("model", [0, 1, 2, 3, 4])
def test_walls_parity_f64(oracle, nx, ny, model):
    theta, tau = 0.37, 0.75
    walls = random_walls(nx, ny, 90 + nx + model)
    f0 = flows.random_populations(nx, ny, seed=2000 + nx + model, spread=0.2)
    ref = oracle.run(f0, theta, tau, model, 60, walls=walls)
    got = gpu_run(f0, theta, tau, model, 60, walls)
    assert_rel(got, ref, REL_F64, f"{nx}x{ny} model {model}")


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("nx,ny", [(48, 20), (45, 7)])
def test_walls_shifted_forms(oracle, prec, nx, ny):
    """Bounce-back permutes stored deviations bit for bit; the error stays within the forms' bound.
    nx = 48 takes the pipeline kernel (FP32), 45 the column kernel."""
    theta, tau, steps = 1.0 / 3.0, 0.7, 100
    walls = random_walls(nx, ny, 7 + nx)
    f0 = oracle.init(*flows.taylor_green(nx, ny, 0.05, theta), theta)
    w0, w1 = 1 - theta, theta / 2
    rest = np.array([w0, w1, w0, w1, w0, w1, w1, w1, w1]) * np.array([w0, w0, w1, w0, w1, w1, w1, w1, w1])
    d = np.abs(f0 - rest[:, None, None]).max()
    ref = oracle.run(f0, theta, tau, 3, steps, walls=walls)
    got = gpu_run(f0, theta, tau, 3, steps, walls, prec)
    bound = steps * (2.0 ** -24 * 16 * d if prec == "f32" else 2.0 ** -11 * d)
    assert np.abs(got - ref).max() <= bound


def test_closed_box_mass_and_diagnostics(oracle):
    """Walls on all sides: fused FP64 diagnostics equal the oracle's, and mass stays constant."""
    nx, ny, theta = 40, 30, 0.4
    walls = np.zeros((ny, nx), dtype=np.uint8)
    walls[0, :] = walls[-1, :] = walls[:, 0] = walls[:, -1] = 1
    f0 = flows.random_populations(nx, ny, seed=77, spread=0.2)
    m0 = oracle.diagnostics(f0)[0]
    with Lattice(nx, ny, theta, 0.6, 3, "f64") as lat:
        lat.set_walls(walls)
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.set_diagnostics_interval(1)
        lat.step(50)
        d, t, status = lat.step_diagnostics()
        assert t == 49 and status == capi.LBM_OK
        ref = oracle.diagnostics(oracle.run(f0, theta, 0.6, 3, 49, walls=walls))
        np.testing.assert_allclose(d[:4], ref[:4], rtol=1e-12, atol=1e-12)
        assert d[0] == pytest.approx(m0, rel=1e-13)
        assert lat.diagnostics()[0] == pytest.approx(m0, rel=1e-13)


def test_removing_walls_restores_the_periodic_step(oracle):
    nx, ny, theta, tau = 24, 9, 0.35, 0.8
    f0 = flows.random_populations(nx, ny, seed=78, spread=0.2)
    with Lattice(nx, ny, theta, tau, 2, "f64") as lat:
        assert lat.set_walls(random_walls(nx, ny, 3)) > 0
        assert lat.set_walls(None) == 0
        assert lat.set_walls(np.zeros((ny, nx))) == 0
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(20)
        got = lat.state().cpu().numpy()
    assert_rel(got, oracle.run(f0, theta, tau, 2, 20), REL_F64, "walls removed")
    with Lattice(nx, ny, theta, tau, 2, "f64") as lat, pytest.raises(ValueError):
        lat.set_walls(np.zeros((ny + 1, nx)))


@pytest.mark.parametrize("model", [0, 3, 4])
def test_vjp_with_walls_matches_oracle_complex_step(oracle, model):
    n, theta, steps, k = 18, 0.4, 25, 6
    tau = oracle.tau_from_nu(0.02, theta)
    walls = random_walls(n, n, 40 + model, frac=0.08)
    g = flows.rng(300 + model)
    rho, ux, uy = flows.random_modes(n, seed=300 + model, kmax=3, amp=0.03)
    fields = (rho + 0.01 * g.standard_normal((n, n)), ux, uy)
    v = [g.standard_normal((n, n)) * 1e-2 for _ in range(3)]
    w = [g.standard_normal((n, n)) for _ in range(3)]
    dev = [torch.from_numpy(a).cuda() for a in fields]
    gw = [torch.from_numpy(a).cuda() for a in w]
    out = [torch.empty_like(dev[0]) for _ in range(3)]
    with Lattice(n, n, theta, tau, model, "f64") as lat:
        lat.set_walls(walls)
        capi.lbm_vjp(lat.ctx, steps, k, *[t.data_ptr() for t in dev], *[t.data_ptr() for t in gw],
                     *[t.data_ptr() for t in out])
        lat.sync()
    grads = [t.cpu().numpy() for t in out]
    h = 1e-30
    f = oracle.run_cplx(oracle.init_cplx(*[a + 1j * h * d for a, d in zip(fields, v)], theta), theta, tau, model,
                        steps, walls=walls)
    want = sum((wk * mk).sum() for wk, mk in zip(w, oracle.moments_cplx(f))).imag / h
    got = sum(float((gk * vk).sum()) for gk, vk in zip(grads, v))
    assert got == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("model", [1, 2, 3, 4])
@pytest.mark.parametrize("theta,nu", [(0.4, 1e-12), (0.55, 1e-9)])
def test_shocktube_parity_with_oracle(oracle, model, theta, nu):
    """The paper's shocktube set-up (800 x 1, walls at both ends, 400 steps) on the GPU path equals
    the oracle's run of the same set-up."""
    rho, ux, uy, walls = experiments.shocktube_fields(800)
    tau = oracle.tau_from_nu(nu, theta)
    f0 = oracle.init(rho, ux, uy, theta)
    ref = oracle.run(f0, theta, tau, model, 400, walls=walls)
    got = gpu_run(f0, theta, tau, model, 400, walls)
    assert_rel(got, ref, 1e-10, f"shocktube model {model} theta {theta}")
