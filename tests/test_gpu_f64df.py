"""Storage form LBM_F64_DF: FP64 populations, collision in double-float arithmetic
(pairs of FP32 values, error-free transformations) on the FP32 pipes, against the
FP64 oracle.

Bar: |gpu - oracle| <= 1e-12 |oracle| element by element after 100 steps on the
same seeded inputs, as for the FP64 form. Derivation of the margin: one
double-float operation rounds with relative error about 2^-47 (1e-14) of its
operands' magnitude instead of FP64's 2^-53; with populations and moments of
order one, the error a step adds to each population is a few 1e-14 and grows
at most linearly over 100 steps (measured: 2.6e-13 at 100 steps, against
1.6e-14 for the FP64 kernels).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    capi.load()
    yield
    torch.cuda.synchronize()


def run(f0, theta, tau, model, steps, walls=None):
    _, ny, nx = f0.shape
    with Lattice(nx, ny, theta, tau, model, "f64df") as lat:
        if walls is not None:
            lat.set_walls(walls)
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(steps)
        lat.sync()
        return lat.state().cpu().numpy()


def assert_rel(got, ref, rel, what=""):
    err = np.abs(got - ref) / np.abs(ref)
    assert err.max() <= rel, f"{what}: max rel err {err.max():.3e}"


@pytest.mark.parametrize("nx,ny", [(37, 23), (64, 64), (1, 5), (130, 3)])
@pytest.mark.parametrize("model", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("theta", [0.25, 1.0 / 3.0, 0.4])
def test_random_state_parity(oracle, nx, ny, model, theta):
    f0 = flows.random_populations(nx, ny, seed=1000 + nx * 7 + ny + model, spread=0.2)
    assert_rel(run(f0, theta, 0.8, model, 100), oracle.run(f0, theta, 0.8, model, 100), REL,
               f"{nx}x{ny} model {model} theta {theta:.3f}")


@pytest.mark.parametrize("model", [0, 1, 3])
def test_taylor_green_1000_steps(oracle, model):
    """The first benchmark flow over its full 1000 steps: 1e-11 relative (linear growth of the 100-step bar)."""
    n, theta, nu, u0 = 64, 1.0 / 3.0, 0.01, 0.05
    tau = oracle.tau_from_nu(nu, theta)
    f0 = oracle.init(*flows.taylor_green(n, n, u0, theta), theta)
    assert_rel(run(f0, theta, tau, model, 1000), oracle.run(f0, theta, tau, model, 1000), 10 * REL, f"model {model}")


def test_fused_diagnostics_and_nonfinite(oracle):
    f0 = flows.random_populations(70, 45, seed=9)
    theta, tau = 0.37, 0.75
    with Lattice(70, 45, theta, tau, "complete", "f64df") as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.set_diagnostics_interval(5)
        lat.step(12)
        out, t, status = lat.step_diagnostics()
        assert t == 10 and status == capi.LBM_OK
        np.testing.assert_allclose(out, oracle.diagnostics(oracle.run(f0, theta, tau, 3, 10)), rtol=1e-12,
                                   atol=1e-12)
        bad = f0.copy()
        bad[4, 3, 5] = np.nan
        lat.set_state(torch.from_numpy(bad).cuda())
        lat.set_diagnostics_interval(1)
        lat.step(1)
        out, t, status = lat.step_diagnostics(raise_nonfinite=False)
        assert status == capi.LBM_ENONFINITE and out[4] >= 1


def test_walls(oracle):
    nx, ny = 40, 17
    walls = np.zeros((ny, nx), dtype=np.uint8)
    walls[:, 0] = walls[:, nx - 1] = 1
    walls[8, 20] = 1
    f0 = flows.random_populations(nx, ny, seed=33, spread=0.2)
    assert_rel(run(f0, 0.4, 0.7, 3, 60, walls), oracle.run(f0, 0.4, 0.7, 3, 60, walls=walls), REL, "walls")


def test_launch_limits_and_batches_refused():
    with Lattice(64, 32, 1 / 3, 0.6, "complete", "f64df") as lat:
        for shape in [(1, 0, 1, 32), (0, 512, 1, 8), (0, 128, 4, 8)]:
            with pytest.raises(capi.LBMError):
                capi.lbm_set_launch_ex(lat.ctx, *shape)
        capi.lbm_set_launch_ex(lat.ctx, 0, 128, 2, 8)
        assert capi.lbm_get_launch_ex(lat.ctx)[:4] == (0, 128, 2, 8)
    with pytest.raises(capi.LBMError):
        capi.lbm_batch_create([16], [16], [0.3], [0.6], 3, capi.LBM_F64_DF)
