"""Hand-written adjoint (lbm_vjp) against the oracle's complex-step gradient and
against central differences of the GPU forward.

Loss L = sum_x g_rho rho(x, n) + g_ux u_x(x, n) + g_uy u_y(x, n) for random
cotangent fields g; its gradient with respect to (rho0, u0) is what lbm_vjp
returns. Directional derivatives along random directions v are compared.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows
from paper_2602_21242_gb300.lattice import Lattice, run

pytestmark = pytest.mark.gpu


def problem(n, seed, theta):
    g = flows.rng(seed)
    rho, ux, uy = flows.random_modes(n, seed=seed, kmax=3, amp=0.03)
    rho = rho + 0.01 * g.standard_normal((n, n))
    v = [g.standard_normal((n, n)) * 1e-2 for _ in range(3)]
    w = [g.standard_normal((n, n)) for _ in range(3)]
    return (rho, ux, uy), v, w


def gpu_vjp(fields, w, theta, tau, model, steps, k, prec="f64", nx=None, ny=None):
    ny, nx = fields[0].shape
    dev = [torch.from_numpy(a).cuda() for a in fields]
    gw = [torch.from_numpy(a).cuda() for a in w]
    out = [torch.empty_like(dev[0]) for _ in range(3)]
    with Lattice(nx, ny, theta, tau, model, prec) as lat:
        capi.lbm_vjp(lat.ctx, steps, k, *[t.data_ptr() for t in dev], *[t.data_ptr() for t in gw],
                     *[t.data_ptr() for t in out])
        lat.sync()
    return [t.cpu().numpy() for t in out]


def oracle_dd(oracle, fields, v, w, theta, tau, model, steps):
    h = 1e-30
    args = [a + 1j * h * d for a, d in zip(fields, v)]
    f = oracle.run_cplx(oracle.init_cplx(*args, theta), theta, tau, model, steps)
    m = oracle.moments_cplx(f)
    return sum((wk * mk).sum() for wk, mk in zip(w, m)).imag / h


def dot(grads, v):
    return sum(float((gk * vk).sum()) for gk, vk in zip(grads, v))


@pytest.mark.parametrize("prec", ["f64", "f64df"])
@pytest.mark.parametrize("model", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("theta", [1.0 / 3.0, 0.4])
def test_vjp_matches_oracle_complex_step(oracle, model, theta, prec):
    """FP64 and the double-float form (FP64 storage and adjoint fields in double-float pairs)."""
    n, steps, k = 20, 30, 7  # segments of 7, 7, 7, 7, 2 steps
    tau = oracle.tau_from_nu(0.02, theta)
    fields, v, w = problem(n, 11 + model, theta)
    grads = gpu_vjp(fields, w, theta, tau, model, steps, k, prec)
    want = oracle_dd(oracle, fields, v, w, theta, tau, model, steps)
    assert dot(grads, v) == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("model", [0, 3, 4])
def test_vjp_every_component_small_grid(oracle, model):
    """Full gradient on a 4 x 3 grid, each input component by its own complex step."""
    nx, ny, theta, steps = 4, 3, 0.35, 9
    tau = 0.7
    g = flows.rng(5)
    fields = (1 + 0.05 * g.standard_normal((ny, nx)), 0.05 * g.standard_normal((ny, nx)),
              0.05 * g.standard_normal((ny, nx)))
    w = [g.standard_normal((ny, nx)) for _ in range(3)]
    grads = gpu_vjp(fields, w, theta, tau, model, steps, 4)
    for c in range(3):
        for idx in np.ndindex(ny, nx):
            v = [np.zeros((ny, nx)) for _ in range(3)]
            v[c][idx] = 1.0
            want = oracle_dd(oracle, fields, v, w, theta, tau, model, steps)
            assert grads[c][idx] == pytest.approx(want, rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("model", [0, 3])
def test_vjp_matches_gpu_central_difference(model):
    """Central differences of the GPU forward itself (FP64), relative 1e-6."""
    n, theta, steps = 32, 1.0 / 3.0, 40
    tau = 0.56
    fields, v, w = problem(n, 23, theta)
    grads = gpu_vjp(fields, w, theta, tau, model, steps, 10)

    def loss(eps):
        with Lattice(n, n, theta, tau, model) as lat:
            lat.init(*(torch.from_numpy(a + eps * d).cuda() for a, d in zip(fields, v)))
            lat.step(steps)
            m = [t.cpu().numpy() for t in lat.moments()]
        return sum((wk * mk).sum() for wk, mk in zip(w, m))

    e = 1e-5
    fd = (loss(e) - loss(-e)) / (2 * e)
    assert dot(grads, v) == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("n", [32, 31])
@pytest.mark.parametrize("model", [0, 3])
def test_vjp_f32_against_f64(oracle, n, model):
    """The FP32 form's adjoint (FP32 arithmetic) against the FP64 adjoint on the same problem, even and
    odd widths."""
    theta, steps = 1.0 / 3.0, 40
    tau = 0.56
    fields, v, w = problem(n, 29, theta)
    g64 = gpu_vjp(fields, w, theta, tau, model, steps, 10, "f64")
    g32 = gpu_vjp(fields, w, theta, tau, model, steps, 10, "f32")
    for a, b in zip(g32, g64):
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b)


def test_autograd_function_uses_the_adjoint(oracle):
    """torch.autograd through run() equals the complex-step gradient of a misfit loss
    L = 1/2 sum (rho_T - rho_target)^2 (the differentiation workload's loss)."""
    n, theta, steps = 24, 1.0 / 3.0, 25
    tau = 0.53
    fields, v, _ = problem(n, 37, theta)
    target = flows.random_modes(n, seed=38, kmax=3, amp=0.03)
    ref_rho = oracle.moments(oracle.run(oracle.init(*target, theta), theta, tau, 3, steps))[0]
    x = [torch.from_numpy(a).cuda().requires_grad_(True) for a in fields]
    with Lattice(n, n, theta, tau, "complete") as lat:
        rho, ux, uy = run(lat, *x, steps, ckpt_every=6)
        loss = 0.5 * ((rho - torch.from_numpy(ref_rho).cuda()) ** 2).sum()
        loss.backward()
    grads = [t.grad.cpu().numpy() for t in x]
    h = 1e-30
    args = [a + 1j * h * d for a, d in zip(fields, v)]
    f = oracle.run_cplx(oracle.init_cplx(*args, theta), theta, tau, 3, steps)
    r = oracle.moments_cplx(f)[0]
    want = (0.5 * (r - ref_rho) ** 2).sum().imag / h
    assert dot(grads, v) == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("prec", ["f64", "f64df", "f32"])
@pytest.mark.parametrize("n_steps,k", [(23, 5), (20, 5), (7, 50)])
def test_vjp_reusing_the_forward_pass(prec, n_steps, k):
    """lbm_vjp_forward + lbm_vjp_ex(LBM_VJP_REUSE_FORWARD) gives the same cotangents as lbm_vjp
    (bit for bit: the same states, the same adjoint steps), leaves the same final state, and is
    refused (LBM_ESTATE, nothing done) once the lattice changed after the forward pass."""
    n, theta, tau, model = 24, 1 / 3, 0.6, 3
    fields, _, w = problem(n, 7, theta)
    dev = [torch.from_numpy(a).cuda() for a in fields]
    gw = [torch.from_numpy(a).cuda() for a in w]
    ptrs = [t.data_ptr() for t in dev] + [t.data_ptr() for t in gw]
    ref = [torch.empty_like(dev[0]) for _ in range(3)]
    got = [torch.empty_like(dev[0]) for _ in range(3)]
    with Lattice(n, n, theta, tau, model, prec) as lat:
        capi.lbm_vjp(lat.ctx, n_steps, k, *ptrs, *[t.data_ptr() for t in ref])
        state_ref = lat.state().cpu().numpy()
        capi.lbm_vjp_forward(lat.ctx, n_steps, k, *ptrs[:3])
        np.testing.assert_array_equal(lat.state().cpu().numpy(), state_ref)
        capi.lbm_vjp_ex(lat.ctx, n_steps, k, *ptrs, *[t.data_ptr() for t in got], flags=capi.LBM_VJP_REUSE_FORWARD)
        lat.sync()
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        # the backward pass consumed the forward pass; another call, or a changed lattice, is refused
        for change in (None, "step"):
            if change == "step":
                capi.lbm_vjp_forward(lat.ctx, n_steps, k, *ptrs[:3])
                lat.step(1)
            with pytest.raises(capi.LBMError) as e:
                capi.lbm_vjp_ex(lat.ctx, n_steps, k, *ptrs, *[t.data_ptr() for t in got],
                                flags=capi.LBM_VJP_REUSE_FORWARD)
            assert e.value.status == capi.LBM_ESTATE
        capi.lbm_vjp_forward(lat.ctx, n_steps, k, *ptrs[:3])
        with pytest.raises(capi.LBMError) as e:  # other n
            capi.lbm_vjp_ex(lat.ctx, n_steps + 1, k, *ptrs, *[t.data_ptr() for t in got],
                            flags=capi.LBM_VJP_REUSE_FORWARD)
        assert e.value.status == capi.LBM_ESTATE
        with pytest.raises(capi.LBMError) as e:
            capi.lbm_vjp_ex(lat.ctx, n_steps, k, *ptrs, *[t.data_ptr() for t in got], flags=2)
        assert e.value.status == capi.LBM_EINVAL
