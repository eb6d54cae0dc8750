"""Torch-facing wrapper of the batched form: many independent periodic lattices
of uneven size, theta and tau, advanced together by liblbm.so."""
from __future__ import annotations

import numpy as np
import torch

from . import capi


class Batch:
    """Independent D2Q9 lattices sharing a collision model and storage form."""

    def __init__(self, nx, ny, theta, tau, model="complete", prec="f32", device=None,
                 stream: torch.cuda.Stream | None = None, mode: str = "graph"):
        self.nx = [int(v) for v in nx]
        self.ny = [int(v) for v in ny]
        self.n = len(self.nx)
        self.theta = [float(v) for v in theta]
        self.tau = [float(v) for v in tau]
        self.model = capi.MODELS[model] if isinstance(model, str) else int(model)
        self.prec = capi.PRECS[prec] if isinstance(prec, str) else int(prec)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.sizes = [a * b for a, b in zip(self.nx, self.ny)]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        with torch.cuda.device(self.device):
            self._b = capi.lbm_batch_create(self.nx, self.ny, self.theta, self.tau, self.model, self.prec,
                                            self.stream.cuda_stream)
        self.set_mode(mode)

    @property
    def handle(self):
        return self._b

    @property
    def total_nodes(self) -> int:
        return int(self.offsets[-1])

    def close(self) -> None:
        if getattr(self, "_b", None):
            with torch.cuda.device(self.device):
                capi.lbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_mode(self, mode: str) -> None:
        capi.lbm_batch_set_mode(self._b, {"graph": capi.LBM_BATCH_GRAPH,
                                          "persistent": capi.LBM_BATCH_PERSISTENT}[mode])

    def set_launch(self, *shape) -> None:
        """(bx, by, rows) for launch kind 0, or (kind, bx, by, rows)."""
        kind, bx, by, rows = (0, *shape) if len(shape) == 3 else shape
        with torch.cuda.device(self.device):
            capi.lbm_batch_set_launch_ex(self._b, kind, bx, by, rows)

    def launch(self):
        """(kind, bx, by, rows, ntiles)."""
        return capi.lbm_batch_get_launch_ex(self._b)

    def set_diagnostics_interval(self, every: int) -> None:
        capi.lbm_batch_set_diagnostics_interval(self._b, every)

    def _after_current(self) -> None:
        """Order the batch's stream after the work queued so far on torch's current stream,
        which produced the tensors handed to the next call (a no-op when the batch runs on
        the current stream)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _packed(self, fields):
        out = []
        for name, parts in zip(("rho", "ux", "uy"), fields):
            flat = torch.cat([torch.as_tensor(p, dtype=torch.float64).reshape(-1) for p in parts])
            if flat.numel() != self.total_nodes:
                raise ValueError(f"{name}: expected {self.total_nodes} values")
            out.append(flat.to(self.device).contiguous())
        return out

    def init(self, rho, ux, uy) -> None:
        """rho, ux, uy: sequences of per-domain (ny_k, nx_k) arrays or tensors."""
        r, u, v = self._packed((rho, ux, uy))
        with torch.cuda.device(self.device):
            self._after_current()
            capi.lbm_batch_init(self._b, r.data_ptr(), u.data_ptr(), v.data_ptr())
            self.stream.synchronize()

    def set_state(self, k: int, f) -> None:
        f = torch.as_tensor(f, dtype=torch.float64).to(self.device).contiguous()
        if tuple(f.shape) != (9, self.ny[k], self.nx[k]):
            raise ValueError("state must have shape (9, ny_k, nx_k)")
        with torch.cuda.device(self.device):
            self._after_current()
            capi.lbm_batch_set_state(self._b, k, f.data_ptr())
            self.stream.synchronize()

    def state(self, k: int) -> torch.Tensor:
        out = torch.empty((9, self.ny[k], self.nx[k]), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            capi.lbm_batch_get_state(self._b, k, out.data_ptr())
            self.stream.synchronize()
        return out

    def step(self, n: int = 1) -> None:
        with torch.cuda.device(self.device):
            capi.lbm_batch_step(self._b, int(n))

    def sync(self) -> None:
        with torch.cuda.device(self.device):
            capi.lbm_batch_sync(self._b)

    def moments(self):
        out = torch.empty((3, self.total_nodes), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            capi.lbm_batch_moments(self._b, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
            self.stream.synchronize()
        res = []
        for k in range(self.n):
            a, b = int(self.offsets[k]), int(self.offsets[k + 1])
            res.append(tuple(out[j, a:b].reshape(self.ny[k], self.nx[k]) for j in range(3)))
        return res

    def diagnostics(self, raise_nonfinite: bool = True):
        with torch.cuda.device(self.device):
            return capi.lbm_batch_diagnostics(self._b, self.n, raise_nonfinite)[0]

    def step_diagnostics(self, raise_nonfinite: bool = True):
        with torch.cuda.device(self.device):
            return capi.lbm_batch_step_diagnostics(self._b, self.n, raise_nonfinite)
