"""Shifted-storage forms (FP32 and FP16 deviations from the rest state, FP32
arithmetic) against the FP64 oracle, at stated error bounds.

Bound derivation (absolute error per population after n steps, flows with
|f - rho_ref W| <= d): each step rounds every stored deviation once (half an ulp
of d: 2^-24 d in FP32, 2^-11 d in FP16) and the FP32 collision adds at most a few
ulps of its O(d) intermediate terms; errors in the conserved moments persist,
those in the other moments relax. A linear worst case over n steps is
n * (2^-24 * 16 d) for FP32 and n * (2^-11 d) for FP16 storage, the form of the
bounds asserted below with d the largest initial deviation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import flows
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu

STEPS = 100


def rest_state(theta):
    w0, w1 = 1 - theta, theta / 2
    wx = np.array([w0, w1, w0, w1, w0, w1, w1, w1, w1])
    wy = np.array([w0, w0, w1, w0, w1, w1, w1, w1, w1])
    return wx * wy


def bound(prec, d, steps=STEPS):
    return steps * (2.0 ** -24 * 16 * d if prec == "f32" else 2.0 ** -11 * d)


U32 = 2.0 ** -24


def rows_per_thread(lat, prec):
    """Most nodes (or node pairs) one thread of the step kernel accumulates into its FP32 diagnostics
    sums under the lattice's launch: `rows` for the column kernel and one CTA per tile; for a
    persistent grid a CTA may take every tile, so rows x tiles."""
    from paper_2602_21242_gb300 import capi
    kind, bx, _, rows = capi.lbm_get_launch_ex(lat.ctx)
    if kind == 1 and bx > 0:
        width = 256 if prec == "f32" else 512
        return rows * (-(-lat.nx // width)) * (-(-lat.ny // rows))
    return rows


def diag_sum_bound(state, theta, h_rows):
    """Derived bound on the error of the shifted forms' fused diagnostics of the pre-collision state
    `state` (9, ny, nx): FP32 sums inside a thread block, FP64 across blocks.

    For a floating-point sum whose longest chain of additions has h roundings, |fl(S) - S| is at
    most h u sum_i |x_i| to first order (u = 2^-24 for FP32). The chains here: a node's moment
    (m0: 4 additions; j: 3; twice the kinetic energy j.u: j, the FP32 reciprocal of rho and the
    products, 8), the thread's accumulation over its h_rows rows (two roundings a row for m0 and j,
    the pair's sum and the running sum; four for the energy's chained FMAs), the warp's xor
    butterfly (5) and thread 0's sum of up to 16 warp totals (15). The FP64 sum across blocks adds
    at most 2^-53 of the total. Returns the bounds for (mass, momentum x, momentum y, energy)."""
    dev = state - rest_state(theta)[:, None, None]
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])[:, None, None]
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])[:, None, None]
    m0, jx, jy = dev.sum(0), (cx * dev).sum(0), (cy * dev).sum(0)
    ke = 0.5 * (jx * jx + jy * jy) / state.sum(0)
    h = np.array([4 + 2 * h_rows + 20, 3 + 2 * h_rows + 20, 3 + 2 * h_rows + 20, 8 + 4 * h_rows + 20])
    sums = np.array([np.abs(m0).sum(), np.abs(jx).sum(), np.abs(jy).sum(), np.abs(ke).sum()])
    totals = np.abs(np.array([state.sum(), jx.sum(), jy.sum(), ke.sum()]))
    return h * U32 * sums + 2.0 ** -53 * totals


def run_form(f0, theta, tau, model, prec, steps=STEPS):
    _, ny, nx = f0.shape
    with Lattice(nx, ny, theta, tau, model, prec) as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(steps)
        lat.sync()
        return lat.state().cpu().numpy()


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("model", [0, 1, 2, 3, 4, 5])
def test_taylor_green_forms(oracle, prec, model):
    n, theta, nu, u0 = 64, 1.0 / 3.0, 0.01, 0.05
    tau = oracle.tau_from_nu(nu, theta)
    f0 = oracle.init(*flows.taylor_green(n, n, u0, theta), theta)
    d = np.abs(f0 - rest_state(theta)[:, None, None]).max()
    ref = oracle.run(f0, theta, tau, model, STEPS)
    got = run_form(f0, theta, tau, model, prec)
    err = np.abs(got - ref).max()
    assert err <= bound(prec, d), f"{prec} model {model}: max abs err {err:.3e} > bound {bound(prec, d):.3e}"
    # velocity error relative to the flow amplitude
    du = max(np.abs(a - b).max() for a, b in zip(oracle.moments(got)[1:], oracle.moments(ref)[1:]))
    assert du / u0 <= (2e-5 if prec == "f32" else 5e-2)


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("theta", [0.25, 0.4])
def test_advected_shear_wave_forms(oracle, prec, theta):
    nx, ny, U = 96, 10, 0.1
    tau = oracle.tau_from_nu(0.005, theta)
    f0 = oracle.init(*flows.shear_wave(nx, ny, U=U, amp=0.01), theta)
    d = np.abs(f0 - rest_state(theta)[:, None, None]).max()
    ref = oracle.run(f0, theta, tau, 3, STEPS)
    got = run_form(f0, theta, tau, 3, prec)
    err = np.abs(got - ref).max()
    assert err <= bound(prec, d), f"{prec} theta {theta}: max abs err {err:.3e} > bound {bound(prec, d):.3e}"


@pytest.mark.parametrize("nx,ny", [(45, 19), (46, 19), (2, 3), (130, 1)])
@pytest.mark.parametrize("model", [0, 3])
def test_random_state_f32(oracle, model, nx, ny):
    """Generic non-equilibrium populations (deviations up to ~0.2 rho w) in the FP32 form; odd
    widths take the one-node-per-thread kernel, even widths the node-pair kernel."""
    theta, tau = 0.35, 0.8
    f0 = flows.random_populations(nx, ny, seed=700 + model, spread=0.2)
    d = np.abs(f0 - rest_state(theta)[:, None, None]).max()
    ref = oracle.run(f0, theta, tau, model, STEPS)
    got = run_form(f0, theta, tau, model, "f32")
    err = np.abs(got - ref).max()
    assert err <= bound("f32", d), f"model {model}: max abs err {err:.3e} > bound {bound('f32', d):.3e}"


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_forms_diagnostics(oracle, prec):
    """FP64 global reductions of the shifted forms against the oracle's compensated sums of
    the same (rounded) state; total mass over 100 steps within what storage rounding allows
    (rounding a stored deviation does not conserve mass: relative drift ~ 1e-8 in FP32,
    ~1e-4 in FP16 for this flow)."""
    n, theta = 48, 1.0 / 3.0
    tau = oracle.tau_from_nu(0.01, theta)
    f0 = oracle.init(*flows.taylor_green(n, n, 0.05, theta), theta)
    with Lattice(n, n, theta, tau, "complete", prec) as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        s0 = lat.state().cpu().numpy()
        np.testing.assert_allclose(lat.diagnostics(), oracle.diagnostics(s0), rtol=1e-12, atol=1e-12)
        lat.set_diagnostics_interval(10)
        lat.step(STEPS)
        st = lat.state().cpu().numpy()
        lat.step(1)  # fused pass at t = STEPS
        fused, t, status = lat.step_diagnostics()
        h_rows = rows_per_thread(lat, prec)
    assert t == STEPS and status == 0
    ref = oracle.diagnostics(st)
    # fused sums (FP32 within a block for the shifted forms, FP64 across blocks): the derived bound
    err = np.abs(np.asarray(fused[:4]) - ref[:4])
    assert (err <= diag_sum_bound(st, theta, h_rows)).all(), (err, diag_sum_bound(st, theta, h_rows))
    drift = abs(ref[0] - oracle.diagnostics(f0)[0]) / ref[0]
    assert drift <= (1e-8 if prec == "f32" else 1e-4)


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("launch", [None, (1, 0, 1, 24), (0, 128, 4, 16)])
def test_fused_sums_against_fp64_sums_of_the_same_state(prec, launch):
    """Separates the two errors in the shifted forms' mass drift. The fused pass sums in FP32
    inside a block; lbm_diagnostics sums the same stored state in FP64 per node. Their
    difference is the reduction error alone and stays within the derived bound; the FP64 sums'
    change over the run is the storage rounding's drift (rounding a stored deviation does not
    conserve mass), reported by the FP64 path, not the reduction."""
    from paper_2602_21242_gb300 import capi
    n, theta, steps = 256, 0.3, 200
    rho, ux, uy = flows.shear_layer(n, n, U=0.1, width=n / 16)
    with Lattice(n, n, theta, 0.50333, "complete", prec) as lat:
        if launch is not None:
            capi.lbm_set_launch_ex(lat.ctx, *launch)
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        m_init = lat.diagnostics()[0]
        lat.step(steps - 1)
        st = lat.state().cpu().numpy()
        exact = lat.diagnostics()  # FP64 per-node sums of the stored state at t = steps - 1
        lat.set_diagnostics_interval(1)
        lat.step(1)  # fused pass over the same state
        fused, t, status = lat.step_diagnostics()
        h_rows = rows_per_thread(lat, prec)
    assert t == steps - 1 and status == 0
    err = np.abs(np.asarray(fused[:4]) - np.asarray(exact[:4]))
    assert (err <= diag_sum_bound(st, theta, h_rows)).all(), (err, diag_sum_bound(st, theta, h_rows))
    # the storage drift is what the FP64 sums see: each step rounds the nine stored deviations of
    # every node once, at most half an ulp each (2^-24 or 2^-11 of a deviation of at most d)
    d = np.abs(st - rest_state(theta)[:, None, None]).max()
    drift = abs(exact[0] - m_init) / (n * n)
    assert drift <= steps * 9 * (U32 if prec == "f32" else 2.0 ** -11) * d


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("nx,ny,rows,ctas", [(64, 40, 7, 0), (264, 17, 5, 0), (520, 9, 4, 0), (8, 5, 2, 0),
                                             (1024, 33, 64, 0), (1032, 65, 3, 1), (2048, 40, 4, 2)])
@pytest.mark.parametrize("model", [0, 3])
def test_pipeline_kernel_matches_column_kernel(prec, nx, ny, rows, ctas, model):
    """The bulk-copy pipeline (launch kind 1) and the column kernel share the per-node
    arithmetic: populations bit-identical, diagnostics equal to FP32 summation order.
    Sizes cover full and partial column strips, partial row blocks, the periodic edges, and
    both one CTA per tile (ctas = 0) and persistent grids (ctas CTAs per SM)."""
    theta, tau = 0.33, 0.7
    f0 = flows.random_populations(nx, ny, seed=900 + nx + ny, spread=0.1)
    out, h_rows = {}, {}
    for kind in (0, 1):
        with Lattice(nx, ny, theta, tau, model, prec) as lat:
            from paper_2602_21242_gb300 import capi
            if kind == 1:
                capi.lbm_set_launch_ex(lat.ctx, 1, ctas, 0, rows)
                assert capi.lbm_get_launch_ex(lat.ctx)[0] == 1
            else:
                capi.lbm_set_launch_ex(lat.ctx, 0, 128, 4, 16)
            lat.set_state(torch.from_numpy(f0).cuda())
            lat.step(5)
            prev = lat.state().cpu().numpy()
            lat.set_diagnostics_interval(1)
            lat.step(1)
            lat.sync()
            d, t, _ = lat.step_diagnostics()
            out[kind] = (lat.state().cpu().numpy(), np.array(d))
            h_rows[kind] = rows_per_thread(lat, prec)
    np.testing.assert_array_equal(out[1][0], out[0][0])
    # two FP32 summation orders of the same state: each within its derived bound of the exact sums
    both = diag_sum_bound(prev, theta, h_rows[0]) + diag_sum_bound(prev, theta, h_rows[1])
    assert (np.abs(out[1][1][:4] - out[0][1][:4]) <= both).all()


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("nx,ny,rows,ctas", [(45, 19, 8, 0), (3, 7, 4, 0), (1, 4, 2, 0), (257, 9, 5, 0),
                                             (513, 6, 4, 1), (100, 6, 3, 2), (250, 33, 16, 0)])
def test_pipeline_kernel_any_width(oracle, prec, nx, ny, rows, ctas):
    """The bulk-copy pipeline on widths that are not multiples of the 16-byte chunk: the main copy is
    rounded up into the row padding, the chunk left of column 0 is the aligned chunk holding column
    nx - 1, and a pair whose second node lies past the strip stores its first node only. Against the
    oracle within the forms' bound, and fused diagnostics against the oracle's."""
    theta, tau, steps = 0.33, 0.7, 40
    f0 = flows.random_populations(nx, ny, seed=950 + nx + ny, spread=0.1)
    d = np.abs(f0 - rest_state(theta)[:, None, None]).max()
    from paper_2602_21242_gb300 import capi
    with Lattice(nx, ny, theta, tau, 3, prec) as lat:
        capi.lbm_set_launch_ex(lat.ctx, 1, ctas, 0, rows)
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(steps - 1)
        prev = lat.state().cpu().numpy()
        lat.set_diagnostics_interval(1)
        lat.step(1)
        out, t, _ = lat.step_diagnostics()
        got = lat.state().cpu().numpy()
        h_rows = rows_per_thread(lat, prec)
    ref = oracle.run(f0, theta, tau, 3, steps)
    assert np.abs(got - ref).max() <= bound(prec, d, steps)
    # the fused pass reduces f(steps - 1): FP32 sums of deviations inside a block, FP64 across blocks
    assert t == steps - 1
    err = np.abs(np.asarray(out[:4]) - oracle.diagnostics(prev)[:4])
    assert (err <= diag_sum_bound(prev, theta, h_rows)).all(), (err, diag_sum_bound(prev, theta, h_rows))
    assert out[4] == 0


@pytest.mark.parametrize("prec,launch", [("f64", None), ("f64df", None), ("f32", (0, 128, 4, 16)),
                                         ("f32", (1, 0, 1, 8)), ("f32", (1, 64, 1, 8)), ("f16", (0, 128, 4, 16)),
                                         ("f16", (1, 0, 1, 8)), ("f16", (1, 64, 1, 8))])
def test_fused_diagnostics_skip_a_nonfinite_node(oracle, prec, launch):
    """One NaN population (at an odd column, so the second node of a pair in the shifted forms):
    the fused pass counts exactly that node and sums the others, in every storage form and
    launch kind, against the oracle's sums over the finite nodes of the same stored state."""
    from paper_2602_21242_gb300 import capi
    f0 = flows.random_populations(40, 17, seed=31, spread=0.1)
    f0[4, 6, 11] = np.nan
    with Lattice(40, 17, 1 / 3, 0.8, "complete", prec) as lat:
        if launch is not None:
            capi.lbm_set_launch_ex(lat.ctx, *launch)
        lat.set_state(torch.from_numpy(f0).cuda())
        stored = lat.state().cpu().numpy()
        lat.set_diagnostics_interval(1)
        lat.step(1)
        d, t, status = lat.step_diagnostics(raise_nonfinite=False)
    assert status == capi.LBM_ENONFINITE and t == 0
    want = oracle.diagnostics(stored)
    assert want[4] == 1 and d[4] == 1
    tol = {"f64": 1e-12, "f64df": 1e-11}.get(prec, 1e-5)
    np.testing.assert_allclose(d[:4], want[:4], rtol=tol, atol=tol)


@pytest.mark.parametrize("prec,n,want", [("f64", 4096, (0, 64, 2, 32)), ("f64df", 4096, (0, 64, 2, 32)),
                                         ("f32", 4096, (2, 0, 1, 24)), ("f32", 8192, (2, 0, 1, 48)),
                                         ("f32", 4097, (2, 0, 1, 24)),
                                         ("f16", 4096, (1, 0, 1, 24)), ("f16", 8192, (1, 0, 1, 48))])
def test_default_launch_shapes(prec, n, want):
    """The documented defaults: FP64 and double-float on the column kernel; FP32 two steps a launch
    on 24-row tiles (48 from 8192^2; any width); FP16 one CTA per tile with the height that fills the
    last wave of three CTAs per SM on GB300's 152 SMs (24 rows at 4096^2: 3.0 waves; 48 rows at
    8192^2: 6.0)."""
    from paper_2602_21242_gb300 import capi
    if prec == "f16" and torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the FP16 tile height depends on the SM count")
    with Lattice(n, n, 1 / 3, 0.6, "complete", prec) as lat:
        assert capi.lbm_get_launch_ex(lat.ctx) == want
