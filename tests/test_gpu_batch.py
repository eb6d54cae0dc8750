"""Batched form: independent lattices of uneven size, theta and tau in one launch.

Each domain of a batch must be bit-identical to a single lattice run of the
same storage form (the per-node arithmetic is shared), in both execution modes,
and the FP64 batch must match the oracle at 1e-12 per node.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows, tune
from paper_2602_21242_gb300.batch import Batch
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu

DOMAINS = [(37, 23, 0.30, 0.70), (64, 64, 0.25, 0.80), (100, 3, 0.40, 0.60), (1, 5, 1 / 3, 0.90),
           (48, 31, 0.35, 0.75), (130, 9, 0.28, 0.65)]


def states(seed, domains=DOMAINS):
    return [flows.random_populations(nx, ny, seed=seed + k, spread=0.15) for k, (nx, ny, _, _) in enumerate(domains)]


def single_run(f0, nx, ny, theta, tau, model, prec, steps, kind=None):
    with Lattice(nx, ny, theta, tau, model, prec) as lat:
        if kind == 1:
            capi.lbm_set_launch_ex(lat.ctx, 1, 0, 1, 32)
        elif kind == 0:
            capi.lbm_set_launch_ex(lat.ctx, 0, 64, 4, 8)
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(steps)
        return lat.state().cpu().numpy()


def make_batch(model, prec, mode, domains=DOMAINS):
    return Batch([d[0] for d in domains], [d[1] for d in domains], [d[2] for d in domains],
                 [d[3] for d in domains], model, prec, mode=mode)


@pytest.mark.parametrize("mode", ["graph", "persistent"])
@pytest.mark.parametrize("prec,kind,nc", [("f64", 0, 0), ("f32", 0, 0), ("f32", 1, 0), ("f32", 1, 32),
                                           ("f16", 0, 0), ("f16", 1, 0), ("f16", 1, 64), ("f32", 2, 0),
                                           ("f16", 2, 0)])
@pytest.mark.parametrize("model", [0, 3])
def test_batch_bit_identical_to_single_lattices(model, prec, kind, nc, mode):
    """Kind 0 tiles run the column routine, kind 1 tiles the bulk-copy pipeline (any width, including
    1 x 5 and odd widths, tiles of 2 nc columns), kind 2 two steps a launch (graph mode; the odd 13th
    step and the persistent mode take single steps); each matches a single lattice stepped with the
    same launch kind (kind 2 with kind 1, which it equals bit for bit)."""
    f0 = states(100 + model)
    steps = 13
    with make_batch(model, prec, mode) as b:
        if kind == 0:
            b.set_launch(0, 64, 4, 2)
        else:
            b.set_launch(kind, nc, 1, 8)
        assert b.launch()[0] == kind
        for k, f in enumerate(f0):
            b.set_state(k, f)
        b.step(steps)
        b.sync()
        got = [b.state(k).cpu().numpy() for k in range(b.n)]
    for k, (nx, ny, theta, tau) in enumerate(DOMAINS):
        want = single_run(f0[k], nx, ny, theta, tau, model, prec, steps,
                          kind=min(kind, 1) if prec != "f64" else None)
        np.testing.assert_array_equal(got[k], want, err_msg=f"domain {k} ({nx}x{ny})")


@pytest.mark.parametrize("model", [1, 2, 3, 4, 5])
def test_batch_f64_oracle_parity(oracle, model):
    f0 = states(200 + model)
    with make_batch(model, "f64", "graph") as b:
        for k, f in enumerate(f0):
            b.set_state(k, f)
        b.step(50)
        for k, (nx, ny, theta, tau) in enumerate(DOMAINS):
            ref = oracle.run(f0[k], theta, tau, model, 50)
            got = b.state(k).cpu().numpy()
            err = np.max(np.abs(got - ref) / np.abs(ref).max(axis=0))
            assert err <= 1e-12, f"domain {k}: {err:.3e}"


def test_batch_graph_recapture_and_parity_changes(oracle):
    """Odd step counts flip the buffer parity; each call still advances every domain."""
    f0 = states(300)
    with make_batch(3, "f64", "graph") as b:
        for k, f in enumerate(f0):
            b.set_state(k, f)
        for n in (3, 5, 3, 0, 1):
            b.step(n)
        b.sync()
        assert capi.lbm_batch_info(b.handle)[2] == 12
        for k, (nx, ny, theta, tau) in enumerate(DOMAINS):
            ref = oracle.run(f0[k], theta, tau, 3, 12)
            np.testing.assert_allclose(b.state(k).cpu().numpy(), ref, rtol=1e-12)


def test_batch_init_moments_and_diagnostics(oracle):
    doms = [(40, 40, 1 / 3, 0.56), (64, 32, 0.3, 0.6), (33, 17, 0.38, 0.7)]
    rho, ux, uy = zip(*[flows.taylor_green(nx, ny, 0.05, th) for nx, ny, th, _ in doms])
    with make_batch(3, "f64", "graph", doms) as b:
        b.init(rho, ux, uy)
        b.set_diagnostics_interval(4)
        b.step(9)  # fused passes at t = 0, 4, 8
        fused, t, status = b.step_diagnostics()
        now = b.diagnostics()
        mom = b.moments()
        for k, (nx, ny, th, tau) in enumerate(doms):
            f8 = oracle.run(oracle.init(rho[k], ux[k], uy[k], th), th, tau, 3, 8)
            f9 = oracle.run(f8, th, tau, 3, 1)
            np.testing.assert_allclose(fused[k], oracle.diagnostics(f8), rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(now[k], oracle.diagnostics(f9), rtol=1e-12, atol=1e-12)
            for got, want in zip(mom[k], oracle.moments(f9)):
                np.testing.assert_allclose(got.cpu().numpy(), want, rtol=1e-12, atol=1e-14)
    assert t == 8 and status == capi.LBM_OK


def test_batch_launch_validation():
    # defaults: FP32 two steps a launch, FP16 the single-step pipeline, on 32-row tiles
    for prec, kind in (("f32", 2), ("f16", 1)):
        with make_batch(3, prec, "graph") as b:
            assert b.launch()[:4] == (kind, 0, 1, 32)
    with make_batch(3, "f32", "graph") as b:
        for bad in [(1, 256, 1, 8), (1, 48, 1, 8), (1, 0, 1, 0), (2, 32, 1, 8), (3, 0, 1, 8)]:
            with pytest.raises(capi.LBMError):
                b.set_launch(*bad)
    with make_batch(3, "f64", "graph") as b, pytest.raises(capi.LBMError):
        b.set_launch(1, 0, 1, 8)


def test_batch_rejects_bad_domains():
    with pytest.raises(capi.LBMError) as e:
        Batch([16, 0], [16, 16], [0.3, 0.3], [0.6, 0.6], "complete", "f32")
    assert e.value.status == capi.LBM_EINVAL
    with pytest.raises(capi.LBMError):
        Batch([16], [16], [0.3], [0.5], "complete", "f32")


def test_tuners(tmp_path):
    path = str(tmp_path / "tune.json")
    with Lattice(256, 256, 1 / 3, 0.56, "complete", "f32") as lat:
        shape, ms = tune.tune_lattice(lat, candidates=[(64, 2, 4), (128, 4, 8), (1, 0, 1, 16)], steps=4, path=path)
        assert shape in [(0, 64, 2, 4), (0, 128, 4, 8), (1, 0, 1, 16)] and ms > 0
        assert capi.lbm_get_launch_ex(lat.ctx)[0] == shape[0]
        assert capi.lbm_get_launch_ex(lat.ctx)[3] == shape[3]
        again, cached = tune.tune_lattice(lat, path=path)
        assert again == shape and cached is None
    with make_batch(3, "f32", "graph") as b:
        shape, ms = tune.tune_batch(b, candidates=[(32, 4, 4), (64, 2, 8), (1, 0, 1, 16)], steps=4, path=path)
        assert shape in [(0, 32, 4, 4), (0, 64, 2, 8), (1, 0, 1, 16)]
        assert b.launch()[:4] == shape


@pytest.mark.parametrize("every", [1, 3])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_batch_two_step_launch_diagnostics(prec, every):
    """Two steps a launch in graph mode: every domain's state equals the kind 1 batch's bit for bit
    after even and odd step counts, and the fused diagnostics of each domain agree within the FP32
    block-sum bound (about 1e-7 of the mass here) at the same time stamp."""
    doms = [(136, 40, 0.3, 0.7), (257, 33, 1 / 3, 0.6), (64, 64, 0.38, 0.8), (1, 7, 0.3, 0.9)]
    f0 = states(400, doms)
    out = {}
    for kind in (1, 2):
        with make_batch(3, prec, "graph", doms) as b:
            b.set_launch(kind, 0, 1, 16)
            b.set_diagnostics_interval(every)
            for k, f in enumerate(f0):
                b.set_state(k, f)
            for n in (4, 3, 6):
                b.step(n)
            fused, t, status = b.step_diagnostics()
            out[kind] = ([b.state(k).cpu().numpy() for k in range(b.n)], fused, t)
    for k in range(len(doms)):
        np.testing.assert_array_equal(out[2][0][k], out[1][0][k], err_msg=f"domain {k}")
        scale = doms[k][0] * doms[k][1]
        np.testing.assert_allclose(out[2][1][k][:4], out[1][1][k][:4], rtol=1e-6, atol=1e-6 * scale)
        assert out[2][1][k][4] == out[1][1][k][4] == 0
    assert out[1][2] == out[2][2] == (13 - 1) // every * every


@pytest.mark.parametrize("mode", ["graph", "persistent"])
def test_batch_two_step_long_run(mode):
    """Two steps a launch over 200 steps in calls of uneven length (odd calls end in a single step,
    which flips the buffer parity the next call starts from): every domain equals the kind 1 batch bit
    for bit."""
    doms = [(136, 40, 0.3, 0.7), (257, 33, 1 / 3, 0.6), (64, 64, 0.38, 0.8), (3, 7, 0.3, 0.9), (511, 19, 0.26, 0.55)]
    f0 = states(500, doms)
    got = {}
    for kind in (1, 2):
        with make_batch(3, "f32", mode, doms) as b:
            b.set_launch(kind, 0, 1, 16)
            for k, f in enumerate(f0):
                b.set_state(k, f)
            for n in (7, 100, 1, 92):
                b.step(n)
            b.sync()
            got[kind] = [b.state(k).cpu().numpy() for k in range(b.n)]
    for k in range(len(doms)):
        np.testing.assert_array_equal(got[2][k], got[1][k], err_msg=f"domain {k}")
