"""Torch-facing wrapper of one lattice: torch supplies device memory and the
stream, liblbm.so does every step of the computation.

Example::

    lat = Lattice(256, 256, theta=1/3, tau=0.53, model="complete")
    lat.init(rho, ux, uy)          # float64 CUDA tensors of shape (ny, nx)
    lat.step(100)
    rho, ux, uy = lat.moments()
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi


def tau_from_nu(nu: float, theta: float) -> float:
    """Relaxation time for lattice viscosity nu: nu = theta (tau - 1/2)."""
    return nu / theta + 0.5


def _dev_f64(t: torch.Tensor, shape, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.to(torch.float64).contiguous()


class Lattice:
    """One doubly periodic D2Q9 lattice advanced by the fused CUDA step (Eq. 1)."""

    def __init__(self, nx: int, ny: int, theta: float, tau: float, model="complete", prec="f64",
                 device=None, stream: torch.cuda.Stream | None = None, torch_buffers: bool = True):
        self.nx, self.ny = int(nx), int(ny)
        self.theta, self.tau = float(theta), float(tau)
        self.model = capi.MODELS[model] if isinstance(model, str) else int(model)
        self.prec = capi.PRECS[prec] if isinstance(prec, str) else int(prec)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        _, _, nbytes = capi.lbm_layout(self.nx, self.ny, self.prec)
        self._buffers = None
        ptr = 0
        with torch.cuda.device(self.device):
            if torch_buffers:
                # torch's caching allocator hands out 512-byte aligned blocks
                self._buffers = torch.empty(2 * nbytes, dtype=torch.uint8, device=self.device)
                ptr = self._buffers.data_ptr()
            self._ctx = capi.lbm_create_ex(self.nx, self.ny, self.theta, self.tau, self.model, self.prec,
                                           self.stream.cuda_stream, ptr)

    # -- lifecycle
    def close(self) -> None:
        if getattr(self, "_ctx", None):
            with torch.cuda.device(self.device):
                capi.lbm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def ctx(self):
        return self._ctx

    def _after_current(self) -> None:
        """Order the lattice's stream after the work queued so far on torch's current
        stream, which produced the tensors handed to the next call (a no-op when the
        lattice runs on the current stream)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _fields(self):
        return torch.empty((3, self.ny, self.nx), dtype=torch.float64, device=self.device)

    # -- state
    def init(self, rho, ux, uy) -> None:
        shape = (self.ny, self.nx)
        rho, ux, uy = (_dev_f64(t, shape, n) for t, n in ((rho, "rho"), (ux, "ux"), (uy, "uy")))
        with torch.cuda.device(self.device):
            self._after_current()
            capi.lbm_init(self._ctx, rho.data_ptr(), ux.data_ptr(), uy.data_ptr())
            self._keep = (rho, ux, uy)  # alive until the stream has consumed them
            self.stream.synchronize()
            self._keep = None

    def set_state(self, f: torch.Tensor) -> None:
        f = _dev_f64(f, (9, self.ny, self.nx), "f")
        with torch.cuda.device(self.device):
            self._after_current()
            capi.lbm_set_state(self._ctx, f.data_ptr())
            self.stream.synchronize()

    def state(self) -> torch.Tensor:
        out = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            capi.lbm_get_state(self._ctx, out.data_ptr())
            self.stream.synchronize()
        return out

    # -- stepping
    def step(self, n: int = 1) -> None:
        with torch.cuda.device(self.device):
            capi.lbm_step(self._ctx, int(n))

    def set_stream(self, stream: torch.cuda.Stream) -> None:
        """Run later calls on `stream`; the library orders them after the work already queued."""
        with torch.cuda.device(self.device):
            capi.lbm_set_stream(self._ctx, stream.cuda_stream)
        self.stream = stream

    def set_diagnostics_interval(self, every: int) -> None:
        capi.lbm_set_diagnostics_interval(self._ctx, int(every))

    def set_walls(self, mask) -> int:
        """Fullway bounce-back wall nodes, (ny, nx) host mask (numpy or CPU tensor; nonzero = wall),
        None = doubly periodic. Returns the number of wall nodes."""
        if mask is not None:
            if isinstance(mask, torch.Tensor):
                mask = mask.detach().cpu().numpy()
            if tuple(np.shape(mask)) != (self.ny, self.nx):
                raise ValueError(f"wall mask must have shape {(self.ny, self.nx)}")
        with torch.cuda.device(self.device):
            return capi.lbm_set_walls(self._ctx, mask)

    def step_diagnostics(self, raise_nonfinite: bool = True):
        with torch.cuda.device(self.device):
            return capi.lbm_step_diagnostics(self._ctx, raise_nonfinite)

    def sync(self) -> None:
        with torch.cuda.device(self.device):
            capi.lbm_sync(self._ctx)

    @property
    def time(self) -> int:
        return capi.lbm_time(self._ctx)

    # -- observables
    def moments(self):
        out = self._fields()
        with torch.cuda.device(self.device):
            capi.lbm_moments(self._ctx, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
            self.stream.synchronize()
        return out[0], out[1], out[2]

    def diagnostics(self, raise_nonfinite: bool = True):
        with torch.cuda.device(self.device):
            return capi.lbm_diagnostics(self._ctx, raise_nonfinite)[0]


class _Run(torch.autograd.Function):
    """(rho0, u0) -> (rho, u) after n steps; backward through lbm_vjp (hand-written adjoint)."""

    @staticmethod
    def forward(fctx, rho0, ux0, uy0, lattice, n, ckpt_every):
        shape = (lattice.ny, lattice.nx)
        r0, u0, v0 = (_dev_f64(t.detach(), shape, nm) for t, nm in ((rho0, "rho0"), (ux0, "ux0"), (uy0, "uy0")))
        if lattice.prec == capi.LBM_F16_SHIFT:  # no adjoint for this form: a plain run
            lattice.init(r0, u0, v0)
            lattice.step(n)
        else:  # the adjoint's forward pass, whose checkpoints the backward pass reuses
            with torch.cuda.device(lattice.device):
                lattice._after_current()
                capi.lbm_vjp_forward(lattice.ctx, n, ckpt_every, r0.data_ptr(), u0.data_ptr(), v0.data_ptr())
        rho, ux, uy = lattice.moments()
        fctx.save_for_backward(r0, u0, v0)
        fctx.lattice, fctx.n, fctx.k = lattice, n, ckpt_every
        return rho.clone(), ux.clone(), uy.clone()

    @staticmethod
    def backward(fctx, g_rho, g_ux, g_uy):
        r0, u0, v0 = fctx.saved_tensors
        lat = fctx.lattice
        grads = [torch.empty_like(r0) for _ in range(3)]
        gs = [g.contiguous().to(torch.float64) if g is not None else None for g in (g_rho, g_ux, g_uy)]
        args = (lat.ctx, fctx.n, fctx.k, r0.data_ptr(), u0.data_ptr(), v0.data_ptr(),
                *[g.data_ptr() if g is not None else 0 for g in gs], *[g.data_ptr() for g in grads])
        with torch.cuda.device(lat.device):
            lat._after_current()  # the incoming gradients and the outputs' allocations
            try:  # the forward pass's checkpoints, unless the lattice changed since
                capi.lbm_vjp_ex(*args, flags=capi.LBM_VJP_REUSE_FORWARD)
            except capi.LBMError as e:
                if e.status != capi.LBM_ESTATE:
                    raise
                capi.lbm_vjp(*args)
            lat.stream.synchronize()
        return grads[0], grads[1], grads[2], None, None, None


def run(lattice: Lattice, rho0, ux0, uy0, n: int, ckpt_every: int = 50):
    """Differentiable run: returns (rho, u_x, u_y) after n steps from f^eq(rho0, u0); gradients
    with respect to rho0, ux0, uy0 come from the library's adjoint (lbm_vjp)."""
    return _Run.apply(rho0, ux0, uy0, lattice, int(n), int(ckpt_every))
