"""Two steps per launch (launch kind 2, the shifted storage forms) through the C ABI.

The two-step kernel rounds step t's post-collision values to the storage type in
shared memory, as a single step stores them, so its results equal those of single
steps bit for bit. Checked against the bulk-copy pipeline (kind 1, one CTA per tile)
on random non-equilibrium states for every model, on lattices narrower than one tile,
exactly one tile wide, with a ragged last strip (even and odd widths, widths whose
wrapped columns are not chunk-aligned, a strip of one column), a single row and one row
fewer than the tile height; with even and odd step counts (an odd count ends with a
single step); and with walls, where lbm_step takes single steps. The fused diagnostics
of every step are compared at the FP32 block-sum bound, their time stamps exactly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu
THETA, TAU = 1.0 / 3.0, 0.8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    capi.load()
    yield
    torch.cuda.synchronize()


def _run(nx, ny, model, prec, f0, steps, launch, diag_every=0, chunks=(), walls=None):
    """State after `steps` steps taken in calls of the given sizes (default: one call),
    and the fused diagnostics of the last diagnosed step."""
    with Lattice(nx, ny, THETA, TAU, model, prec) as lat:
        capi.lbm_set_launch_ex(lat.ctx, *launch)
        if walls is not None:
            lat.set_walls(walls)
        lat.set_diagnostics_interval(diag_every)
        lat.set_state(f0)
        for n in (chunks or (steps,)):
            lat.step(n)
        diag = lat.step_diagnostics(raise_nonfinite=False)[:2] if diag_every else None
        return lat.state(), diag


SIZES = [(4, 3), (8, 1), (12, 5), (64, 64), (254, 9), (256, 40), (260, 33), (508, 17), (516, 8), (1024, 70),
         (1, 5), (2, 3), (3, 2), (37, 5), (255, 3), (257, 9), (509, 11), (511, 4), (66, 10), (130, 7)]


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_two_step_launch_equals_single_steps(nx, ny, prec):
    f0 = torch.from_numpy(flows.random_populations(nx, ny, seed=11 * nx + ny, spread=0.2)).cuda()
    for steps in (8, 7):
        one, _ = _run(nx, ny, "complete", prec, f0, steps, (1, 0, 1, 16))
        two, _ = _run(nx, ny, "complete", prec, f0, steps, (2, 0, 1, 16))
        assert torch.equal(one, two), f"{prec} {nx}x{ny}, {steps} steps: {(one - two).abs().max().item():.3e}"


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("model", ["lbgk", "oreg", "partial", "complete", "complete_neq", "lbgk_poly"])
def test_two_step_launch_every_model(model, prec):
    nx, ny = 136, 29
    f0 = torch.from_numpy(flows.random_populations(nx, ny, seed=3 + len(model), spread=0.15)).cuda()
    one, _ = _run(nx, ny, model, prec, f0, 12, (1, 0, 1, 8))
    for rows in (1, 8, 28, 29, 64):
        two, _ = _run(nx, ny, model, prec, f0, 12, (2, 0, 1, rows))
        assert torch.equal(one, two), f"{model}/{prec} rows {rows}"


@pytest.mark.parametrize("every", [1, 2, 3])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_two_step_diagnostics(prec, every):
    nx, ny = 512, 48
    f0 = torch.from_numpy(flows.random_populations(nx, ny, seed=77, spread=0.05)).cuda()
    for steps, chunks in ((9, ()), (10, (3, 4, 3)), (6, (1, 5))):
        one, d1 = _run(nx, ny, "complete", prec, f0, steps, (1, 0, 1, 16), every, chunks)
        two, d2 = _run(nx, ny, "complete", prec, f0, steps, (2, 0, 1, 16), every, chunks)
        assert torch.equal(one, two)
        assert d1[1] == d2[1] == (steps - 1) // every * every
        # the same values summed in FP32 within blocks of another shape: the derived FP32
        # block-sum bound is about 1e-7 of the mass here
        scale = nx * ny
        np.testing.assert_allclose(d2[0][:4], d1[0][:4], rtol=1e-6, atol=1e-6 * scale)
        assert d1[0][4] == d2[0][4] == 0


def test_two_step_launch_falls_back_with_walls():
    # walls act after every step, so lbm_step takes single steps
    nx, ny = 64, 16
    walls = np.zeros((ny, nx), dtype=np.uint8)
    walls[:, 0] = walls[:, -1] = 1
    f0 = torch.from_numpy(flows.random_populations(nx, ny, seed=5, spread=0.1)).cuda()
    one, _ = _run(nx, ny, "complete", "f32", f0, 6, (1, 0, 1, 4), walls=walls)
    two, _ = _run(nx, ny, "complete", "f32", f0, 6, (2, 0, 1, 4), walls=walls)
    assert torch.equal(one, two)


def test_two_step_launch_matches_the_oracle(oracle):
    # the FP32 form's bar against the oracle, through kind 2 (the exactness above makes
    # this the single-step bar)
    nx, ny, steps = 128, 40, 20
    rho, ux, uy = flows.taylor_green(nx, ny, 0.05, THETA)
    ref = oracle.run(oracle.init(rho, ux, uy, THETA), THETA, TAU, capi.LBM_OREG_COMPLETE, steps)
    with Lattice(nx, ny, THETA, TAU, "complete", "f32") as lat:
        capi.lbm_set_launch_ex(lat.ctx, 2, 0, 1, 16)
        assert capi.lbm_get_launch_ex(lat.ctx)[0] == 2
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        lat.step(steps)
        got = lat.state().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-6


def test_kind_two_is_refused_for_fp64_forms():
    for prec in ("f64", "f64df"):
        with Lattice(16, 8, THETA, TAU, "complete", prec) as lat:
            with pytest.raises(capi.LBMError, match="LBM_EINVAL"):
                capi.lbm_set_launch_ex(lat.ctx, 2, 0, 1, 16)
    with Lattice(16, 8, THETA, TAU, "complete", "f32") as lat:
        with pytest.raises(capi.LBMError, match="LBM_EINVAL"):
            capi.lbm_set_launch_ex(lat.ctx, 2, 64, 1, 16)  # one CTA per tile only


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_two_step_launch_long_run(prec):
    """600 steps of a Taylor-Green flow in calls of uneven length, diagnostics every 7 steps: the
    two-step launches stay equal to single steps bit for bit over a long run."""
    nx, ny = 260, 130
    fields = [torch.from_numpy(a).cuda() for a in flows.taylor_green(nx, ny, 0.08, THETA)]
    out = []
    for launch in ((1, 0, 1, 16), (2, 0, 1, 16)):
        with Lattice(nx, ny, THETA, 0.53, "complete", prec) as lat:
            capi.lbm_set_launch_ex(lat.ctx, *launch)
            lat.set_diagnostics_interval(7)
            lat.init(*fields)
            for n in (1, 2, 3, 97, 200, 297):
                lat.step(n)
            out.append((lat.state(), lat.step_diagnostics()[1]))
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] == 595
