"""The FP64 form's integer-pipe binary64 products (and the sum routine beside them)
against the FP64 instructions, bit for bit, on the GPU: operand families that reach
every path of the routines (random bit patterns with zeros, subnormals, infinities
and NaNs; normal operands at every exponent distance; cancelling sums; exact ties;
products at the edges of the normal range; the lattice's magnitudes); and the FP64
collision of every model with its products on the integer pipes against the same
collision with every product on the FP64 pipe, on near-equilibrium and far-from-
equilibrium nodes, nodes at rest and nodes with zero populations."""
import numpy as np
import pytest

from paper_2602_21242_gb300 import capi, flows

pytestmark = pytest.mark.gpu


def _bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)


def _same(a, b):
    return (_bits(a) == _bits(b)) | (np.isnan(a) & np.isnan(b))


def _make(sign, e, frac):
    u = (sign.astype(np.uint64) << np.uint64(63)) | (e.astype(np.uint64) << np.uint64(52)) | (
        frac.astype(np.uint64) & np.uint64((1 << 52) - 1))
    return u.view(np.float64)


def _families(seed, n):
    g = np.random.default_rng(seed)
    r = lambda: g.integers(0, 2 ** 63, n, dtype=np.uint64) * np.uint64(2) + g.integers(0, 2, n, dtype=np.uint64)
    out = []
    # random bit patterns
    out.append((r().view(np.float64), r().view(np.float64)))
    # normal operands at every exponent distance
    ea = g.integers(1, 2047, n)
    eb = np.clip(ea - g.integers(0, 72, n), 1, 2046)
    out.append((_make(g.integers(0, 2, n), ea, r()), _make(g.integers(0, 2, n), eb, r())))
    # cancelling: b = -(a with low bits changed), same or next exponent
    ea = g.integers(2, 2042, n)
    fa = r()
    flip = r() & ((np.uint64(1) << g.integers(0, 53, n).astype(np.uint64)) - np.uint64(1))
    sa = g.integers(0, 2, n)
    out.append((_make(sa, ea, fa), _make(1 - sa, ea - g.integers(0, 2, n), fa ^ flip)))
    # ties: b at half an ulp of a or near it; short significands (exact products and ties)
    ea = g.integers(60, 1960, n)
    out.append((_make(g.integers(0, 2, n), ea, r()), _make(g.integers(0, 2, n), ea - g.integers(52, 56, n),
                                                           (r() >> np.uint64(48)) << np.uint64(36))))
    k = g.integers(1, 28, n).astype(np.uint64)
    ma = (r() >> (np.uint64(64) - k)) | np.uint64(1)
    mb = (r() >> (np.uint64(64) - k)) | np.uint64(1)
    sh = np.uint64(53) - k
    out.append((_make(g.integers(0, 2, n), g.integers(700, 1300, n), ma << sh),
                _make(g.integers(0, 2, n), g.integers(700, 1300, n), mb << sh)))
    # products at the bottom and the top of the normal range
    ea = g.integers(1, 2047, n)
    top = g.integers(0, 2, n)
    eb = np.clip(np.where(top == 1, 3069 - ea, 1024 - ea) + g.integers(-2, 3, n), 1, 2046)
    out.append((_make(g.integers(0, 2, n), ea, r()), _make(g.integers(0, 2, n), eb, r())))
    # the lattice's magnitudes
    a = (g.uniform(size=n) - 0.25) * g.choice([1.0, 0.5, 0.1, 0.01], n)
    b = (g.uniform(size=n) - 0.5) * g.choice([1.0, 0.5, 0.1, 0.01], n)
    b = np.where(g.uniform(size=n) < 0.2, -a + (g.uniform(size=n) - 0.5) * 1e-9, b)
    out.append((a, b))
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
                        np.finfo(np.float64).max, -np.finfo(np.float64).max, 0.5, 3.0, 1e-300, 1e300])
    sa, sb = np.meshgrid(special, special)
    out.append((sa.ravel(), sb.ravel()))
    return out


@pytest.mark.parametrize("op", [0, 1])
def test_integer_pipe_arithmetic_is_bit_identical(op):
    with np.errstate(all="ignore"):
        for fam, (a, b) in enumerate(_families(2602 + op, 200_000)):
            for x, y in ((a, b), (b, a)):
                emu, fp64 = capi.lbm_selftest_fp64_emu(op, x, y)
                host = x + y if op == 0 else x * y
                bad = ~_same(emu, fp64)
                assert not bad.any(), (f"op {op} family {fam}: {bad.sum()} mismatches, first a={x[bad][0]!r} "
                                       f"b={y[bad][0]!r} emu={emu[bad][0]!r} fp64={fp64[bad][0]!r}")
                assert _same(fp64, host).all(), f"op {op} family {fam}: the FP64 instruction differs from the host"


def _nodes(seed, n):
    """n x 9 populations: near and far from equilibrium, nodes at rest, zeros."""
    g = np.random.default_rng(seed)
    near = flows.random_populations(n, 1, seed=seed, spread=0.02).reshape(9, n).T
    far = flows.random_populations(n, 1, seed=seed + 1, spread=0.9).reshape(9, n).T
    rest = flows.random_populations(n, 1, seed=seed + 2, spread=0.0).reshape(9, n).T.copy()
    zeros = far.copy()
    zeros[g.uniform(size=zeros.shape) < 0.15] = 0.0
    sym = near.copy()
    sym[:, 3], sym[:, 4], sym[:, 7], sym[:, 8] = sym[:, 1], sym[:, 2], sym[:, 5], sym[:, 6]  # u = 0 exactly
    return np.concatenate([near, far, rest, zeros, sym])


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("model", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("theta,tau", [(1.0 / 3.0, 0.8), (0.25, 0.51), (0.4, 1.7)])
def test_collision_with_integer_pipe_products_is_bit_identical(model, theta, tau, mode):
    f = _nodes(100 + model, 20_000)
    emu, ref = capi.lbm_selftest_collide_f64(model, theta, tau, f, mode)
    bad = ~_same(emu, ref)
    assert not bad.any(), f"model {model}: {bad.any(axis=1).sum()} nodes differ, e.g. node {np.argmax(bad.any(axis=1))}"
    # and the collision conserves mass (and momentum, except the uncorrected model, whose
    # momentum defect is the compatibility error psi that the corrections remove) on the
    # near-equilibrium nodes
    post = emu[:20_000, :9]
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    np.testing.assert_allclose(post.sum(axis=1), f[:20_000].sum(axis=1), rtol=1e-14)
    if model != 1:
        np.testing.assert_allclose(post @ cx, f[:20_000] @ cx, atol=1e-15)


def test_selftest_arguments_are_checked():
    with pytest.raises(capi.LBMError):
        capi.lbm_selftest_fp64_emu(2, np.ones(2), np.ones(2))
    with pytest.raises(capi.LBMError):
        capi.lbm_selftest_collide_f64(6, 1 / 3, 0.8, np.ones((2, 9)))
    with pytest.raises(capi.LBMError):
        capi.lbm_selftest_collide_f64(3, 1 / 3, 0.5, np.ones((2, 9)))
    with pytest.raises(capi.LBMError):
        capi.lbm_selftest_collide_f64(3, 1 / 3, 0.8, np.ones((2, 9)), mode=3)
    e, r = capi.lbm_selftest_fp64_emu(0, np.array([]), np.array([]))
    assert e.size == r.size == 0


@pytest.mark.parametrize("launch", [None, (1, 0, 1, 8)])
@pytest.mark.parametrize("flow", ["shear_wave", "uy_zero", "rest", "partial_rest"])
@pytest.mark.parametrize("model", [0, 3, 5])
def test_fp64_step_with_zero_velocities_matches_the_oracle(oracle, flow, model, launch):
    """Velocities that are exactly zero (a component everywhere, a fluid at rest, a region
    at rest) send the FP64 collision's integer-pipe products to the FP64 instruction (a
    node redone, then whole warps on FP64 products): the column kernel and the bulk-copy
    pipeline both stay within the FP64 bar of the oracle after 30 steps."""
    import torch
    from paper_2602_21242_gb300.lattice import Lattice
    nx, ny, theta, tau, steps = 160, 48, 1.0 / 3.0, 0.8, 30
    U, amp = {"shear_wave": (0.1, 0.01), "uy_zero": (0.1, 0.0), "rest": (0.0, 0.0), "partial_rest": (0.05, 0.02)}[flow]
    rho, ux, uy = flows.shear_wave(nx, ny, U, amp)
    if flow == "partial_rest":  # the right half at rest
        ux[:, nx // 2:] = 0.0
        uy[:, nx // 2:] = 0.0
    ref = oracle.run(oracle.init(rho, ux, uy, theta), theta, tau, model, steps)
    with Lattice(nx, ny, theta, tau, model, "f64") as lat:
        if launch is not None:
            capi.lbm_set_launch_ex(lat.ctx, *launch)
        lat.set_diagnostics_interval(1)
        lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
        lat.step(steps)
        got = lat.state().cpu().numpy()
        diag = lat.step_diagnostics()[0]
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    assert err.max() <= 1e-12, f"{flow} model {model}: max relative error {err.max():.3e}"
    assert diag[4] == 0 and np.isfinite(diag[:4]).all()


@pytest.mark.parametrize("model", [0, 3, 4])
def test_fp64_result_does_not_depend_on_which_warps_switch_products(model):
    """Every product mode gives the same bits, so the FP64 state after a flow whose warps switch
    modes at different rows (a region at rest beside a moving one, zeros on lines) is the same
    bit for bit under every launch shape and both FP64 kernels."""
    import torch
    from paper_2602_21242_gb300.lattice import Lattice
    nx, ny, theta, tau, steps = 300, 70, 1.0 / 3.0, 0.7, 12
    rho, ux, uy = flows.shear_wave(nx, ny, 0.05, 0.02)
    ux[:, : nx // 3] = 0.0  # a third at rest
    uy[:, : nx // 3] = 0.0
    uy[ny // 2, :] = 0.0
    out = []
    for launch in ((0, 64, 2, 32), (0, 32, 4, 8), (0, 128, 1, 3), (0, 32, 1, 64), (1, 0, 1, 5), (1, 0, 1, 16)):
        with Lattice(nx, ny, theta, tau, model, "f64") as lat:
            capi.lbm_set_launch_ex(lat.ctx, *launch)
            lat.set_diagnostics_interval(1)
            lat.init(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
            lat.step(steps)
            out.append((launch, lat.state().cpu().numpy()))
    ref = out[0][1]
    for launch, got in out[1:]:
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), f"launch {launch} differs from {out[0][0]}"
