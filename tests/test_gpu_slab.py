"""Slab split along y on the GPU through the C ABI (lbm_halo_bytes, lbm_halo_pack,
lbm_halo_unpack): one lattice held as K slabs of one process, each an ordinary context
stepped by the same kernels, trading the populations that cross its faces after every
step (Eq. 1's streaming between slabs).

* The slabs put together equal the unsplit lattice bit for bit in every storage form
  (the per-node arithmetic does not depend on the node's place), for ragged splits,
  one-row slabs and a lattice spanning several tiles.
* FP64: equal to the oracle's single-lattice run within the FP64 bar (1e-12 relative).
* The summed diagnostics (lbm_diagnostics and the fused ones of the next step) equal
  the whole lattice's within FP64 summation error.
* A slab that is its own neighbour (one slab, or one rank without torch.distributed)
  is the periodic lattice itself.
* Host-side refusals: NULL and misaligned face buffers, a pack that does not follow
  exactly one step, an unpack without its pack.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows
from paper_2602_21242_gb300.lattice import Lattice
from paper_2602_21242_gb300.slab import (SlabLattice, init_slabs, set_state_slabs, slab_rows, slabs_diagnostics,
                                         step_slabs)

pytestmark = pytest.mark.gpu
THETA, TAU = 1.0 / 3.0, 0.8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    capi.load()
    yield
    torch.cuda.synchronize()


def _split_run(nx, ny, k, model, prec, f0, steps, diag_every=0):
    slabs = [SlabLattice(nx, ny, THETA, TAU, model, prec, nslabs=k, index=j) for j in range(k)]
    try:
        for s in slabs:
            s.set_diagnostics_interval(diag_every)
        set_state_slabs(slabs, f0)
        step_slabs(slabs, steps)
        whole = torch.cat([s.state() for s in slabs], dim=1)
        diag = slabs_diagnostics(slabs)
        fused = None
        if diag_every:
            parts = [s.lattice.step_diagnostics()[:2] for s in slabs]
            assert len({t for _, t in parts}) == 1
            fused = [sum(p[0][j] for p in parts) for j in range(5)], parts[0][1]
        return whole, diag, fused
    finally:
        for s in slabs:
            s.close()


def _whole_run(nx, ny, model, prec, f0, steps, diag_every=0):
    with Lattice(nx, ny, THETA, TAU, model, prec) as lat:
        lat.set_diagnostics_interval(diag_every)
        lat.set_state(f0)
        lat.step(steps)
        fused = lat.step_diagnostics()[:2] if diag_every else None
        return lat.state(), lat.diagnostics(), fused


CASES = [(48, 37, 3), (48, 37, 2), (33, 5, 5), (40, 3, 3), (256, 200, 2), (30, 16, 1)]


@pytest.mark.parametrize("prec", ["f64", "f64df", "f32", "f16"])
@pytest.mark.parametrize("nx,ny,k", CASES)
def test_slabs_equal_the_whole_lattice_bitwise(nx, ny, k, prec):
    f0 = torch.from_numpy(flows.random_populations(nx, ny, seed=7 * nx + ny + k, spread=0.2)).cuda()
    steps = 40 if nx * ny < 20000 else 100
    split, _, _ = _split_run(nx, ny, k, "complete", prec, f0, steps)
    whole, _, _ = _whole_run(nx, ny, "complete", prec, f0, steps)
    assert torch.equal(split, whole), f"{prec} {nx}x{ny}/{k}: max diff {(split - whole).abs().max().item():.3e}"


@pytest.mark.parametrize("model", ["lbgk", "oreg", "partial", "complete", "complete_neq", "lbgk_poly"])
def test_slabs_match_the_oracle(oracle, model):
    nx, ny, k, steps = 40, 29, 3, 100
    f0 = flows.random_populations(nx, ny, seed=29 + len(model), spread=0.2)
    ref = oracle.run(f0, THETA, TAU, capi.MODELS[model], steps)
    split, diag, _ = _split_run(nx, ny, k, model, "f64", torch.from_numpy(f0).cuda(), steps)
    got = split.cpu().numpy()
    assert (np.abs(got - ref) / np.abs(ref)).max() <= 1e-12
    want = oracle.diagnostics(ref)
    assert diag[4] == 0
    np.testing.assert_allclose(diag[:4], want[:4], rtol=1e-12, atol=1e-12 * want[0])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_summed_diagnostics_equal_the_whole_lattice(prec):
    nx, ny, k, steps = 96, 64, 4, 10
    f0 = torch.from_numpy(flows.random_populations(nx, ny, seed=5, spread=0.05)).cuda()
    _, d_split, fused_split = _split_run(nx, ny, k, "complete", prec, f0, steps, diag_every=1)
    _, d_whole, fused_whole = _whole_run(nx, ny, "complete", prec, f0, steps, diag_every=1)
    scale = d_whole[0]
    # lbm_diagnostics: FP64 sums of the same stored values in another order. The shifted
    # forms' fused diagnostics sum in FP32 within a thread block: the derived bound of that
    # sum, h u sum |x_i| with h <= 32 roundings and |m0| <= 0.05 a node, is about 1e-7 of
    # the mass here; 1e-6 of it is taken for each side's difference.
    np.testing.assert_allclose(d_split[:4], d_whole[:4], rtol=1e-12, atol=1e-13 * scale)
    assert fused_split[1] == fused_whole[1] == steps - 1
    tol = 1e-12 if prec == "f64" else 1e-6
    np.testing.assert_allclose(fused_split[0][:4], fused_whole[0][:4], rtol=tol, atol=tol * scale)
    assert fused_split[0][4] == fused_whole[0][4] == 0


def test_one_rank_slab_is_the_periodic_lattice():
    import torch.distributed as dist

    if dist.is_initialized():
        pytest.skip("a process group is active")
    nx, ny = 64, 48
    rho, ux, uy = (torch.from_numpy(a).cuda() for a in flows.taylor_green(nx, ny, 0.05, THETA))
    with SlabLattice(nx, ny, THETA, TAU, "complete", "f64") as s, Lattice(nx, ny, THETA, TAU, "complete") as lat:
        assert (s.y0, s.y1, s.nslabs) == (0, ny, 1)
        s.init(rho, ux, uy)
        lat.init(rho, ux, uy)
        s.step(25)
        lat.step(25)
        assert torch.equal(s.state(), lat.state())
        assert s.diagnostics() == lat.diagnostics()


def test_init_from_whole_fields_equals_whole_init():
    nx, ny, k = 50, 23, 3
    fields = [torch.from_numpy(a).cuda() for a in flows.taylor_green(nx, ny, 0.05, THETA)]
    slabs = [SlabLattice(nx, ny, THETA, TAU, "partial", "f64", nslabs=k, index=j) for j in range(k)]
    try:
        init_slabs(slabs, *fields)
        step_slabs(slabs, 30)
        split = torch.cat([s.state() for s in slabs], dim=1)
        assert [(s.y0, s.y1) for s in slabs] == [slab_rows(ny, k, j) for j in range(k)]
    finally:
        for s in slabs:
            s.close()
    with Lattice(nx, ny, THETA, TAU, "partial") as lat:
        lat.init(*fields)
        lat.step(30)
        assert torch.equal(split, lat.state())


def test_halo_calls_refuse_bad_buffers():
    nx, ny = 16, 8
    with Lattice(nx, ny, THETA, TAU, "complete", "f64") as lat:
        nbytes = capi.lbm_halo_bytes(lat.ctx)
        assert nbytes == 3 * nx * 8
        buf = torch.zeros(4 * nbytes + 64, dtype=torch.uint8, device="cuda")
        p = buf.data_ptr()
        with pytest.raises(capi.LBMError, match="LBM_ESTATE"):
            capi.lbm_halo_pack(lat.ctx, p, p + nbytes)
        lat.init(*(torch.from_numpy(a).cuda() for a in flows.taylor_green(nx, ny, 0.05, THETA)))
        with pytest.raises(capi.LBMError, match="LBM_EINVAL"):
            capi.lbm_halo_pack(lat.ctx, 0, p)
        with pytest.raises(capi.LBMError, match="LBM_EINVAL"):
            capi.lbm_halo_unpack(lat.ctx, p + 4, p + nbytes)
        # the order: exactly one step, then pack, then unpack
        with pytest.raises(capi.LBMError, match="LBM_ESTATE"):
            capi.lbm_halo_pack(lat.ctx, p, p + nbytes)  # no step since init
        lat.step(2)
        with pytest.raises(capi.LBMError, match="LBM_ESTATE"):
            capi.lbm_halo_pack(lat.ctx, p, p + nbytes)  # two steps
        with pytest.raises(capi.LBMError, match="LBM_ESTATE"):
            capi.lbm_halo_unpack(lat.ctx, p, p + nbytes)  # no pack
        lat.set_state(lat.state())
        lat.step(1)
        capi.lbm_halo_pack(lat.ctx, p, p + nbytes)
        capi.lbm_halo_unpack(lat.ctx, p, p + nbytes)
        with pytest.raises(capi.LBMError, match="LBM_ESTATE"):
            capi.lbm_halo_unpack(lat.ctx, p, p + nbytes)  # already unpacked
        lat.sync()
    with Lattice(nx, ny, THETA, TAU, "complete", "f16") as lat16:
        assert capi.lbm_halo_bytes(lat16.ctx) == 3 * nx * 2
