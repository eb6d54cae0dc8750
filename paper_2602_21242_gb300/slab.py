"""Slab split of one periodic D2Q9 lattice along y (Eq. 1's streaming across the
faces between slabs).

Each slab is an ordinary context of nx x (y1 - y0) nodes holding rows [y0, y1)
of the nx x ny lattice, stepped by the same fused kernels as a whole lattice.
After every step each slab trades, with the slab below and the slab above,
the 3 nx populations per face that cross it (lbm_halo_pack / lbm_halo_unpack:
i = 2, 5, 6 upward, 4, 7, 8 downward); no row is duplicated or stepped twice.
Across ranks the trade is one point-to-point send and receive per face
(torch.distributed: NCCL between GPUs, gloo on CPU); the only collective is the
sum of the five global diagnostics when they are asked for. Within one process, `step_slabs` advances several
slabs in lock step and hands each the other slabs' face buffers directly.

Example (one rank per GPU, launched by torchrun)::

    dist.init_process_group("nccl")
    s = SlabLattice(4096, 4096, theta=1/3, tau=0.515, model="complete")
    s.init(rho, ux, uy)          # the whole lattice's (ny, nx) fields, or only rows [s.y0, s.y1)
    s.step(100)
    mass, jx, jy, energy, bad = s.diagnostics()   # the whole lattice's
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import capi
from .lattice import Lattice

# Populations that cross a face (c_y = +1 upward, c_y = -1 downward), in the order
# of the face buffers.
UP_POPS = (2, 5, 6)
DOWN_POPS = (4, 7, 8)


def slab_rows(ny: int, nslabs: int, k: int) -> tuple[int, int]:
    """Rows [y0, y1) of slab k when ny rows are split into nslabs slabs as evenly as
    possible (the first ny % nslabs slabs take one row more)."""
    if not 1 <= nslabs <= ny:
        raise ValueError(f"cannot split {ny} rows into {nslabs} slabs of at least one row")
    if not 0 <= k < nslabs:
        raise ValueError(f"slab index {k} outside [0, {nslabs})")
    base, extra = divmod(ny, nslabs)
    y0 = k * base + min(k, extra)
    return y0, y0 + base + (1 if k < extra else 0)


def neighbours(k: int, nslabs: int) -> tuple[int, int]:
    """(slab below, slab above) of slab k on the periodic lattice."""
    return (k - 1) % nslabs, (k + 1) % nslabs


def _peer(group, r: int) -> int:
    return r if group is None else dist.get_global_rank(group, r)


def halo_exchange(send_up: torch.Tensor, send_down: torch.Tensor, recv_below: torch.Tensor,
                  recv_above: torch.Tensor, group=None) -> None:
    """One step's trade of face buffers between the ranks of `group`, rank r holding slab r:
    send_up goes to the rank above and arrives there as its recv_below; send_down goes to the
    rank below and arrives as its recv_above. Blocking for the host with gloo; with NCCL the
    transfers are ordered after the current stream's work and before its later work.

    The four operations are issued in the same order on every rank (send up, send down,
    receive from below, receive from above), which pairs them correctly also where the
    backend matches messages between two ranks by order rather than by tag (two ranks,
    where the rank above and the rank below are the same)."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        recv_below.copy_(send_up)
        recv_above.copy_(send_down)
        return
    rank = dist.get_rank(group)
    below, above = (_peer(group, r) for r in neighbours(rank, world))
    ops = [dist.P2POp(dist.isend, send_up, above, group, tag=0),
           dist.P2POp(dist.isend, send_down, below, group, tag=1),
           dist.P2POp(dist.irecv, recv_below, below, group, tag=0),
           dist.P2POp(dist.irecv, recv_above, above, group, tag=1)]
    for work in dist.batch_isend_irecv(ops):
        work.wait()


def global_diagnostics(out5, device, group=None) -> list:
    """Sum the five diagnostics (mass, momentum x, y, kinetic energy, non-finite nodes) of
    every rank's slab; every rank receives the whole lattice's."""
    t = torch.tensor([float(v) for v in out5], dtype=torch.float64, device=device)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.tolist()


class SlabLattice:
    """Rows [y0, y1) of an nx x ny doubly periodic lattice in a context of their own.

    With `nslabs` and `index` unset, the slabs are the ranks of `group` (the default
    process group if torch.distributed is initialised, else one slab); `step` trades
    the face buffers with the neighbouring ranks after each step. With `nslabs` and
    `index` set, the slab is one of several in this process, advanced together by
    `step_slabs`.
    """

    def __init__(self, nx: int, ny: int, theta: float, tau: float, model="complete", prec="f64", *,
                 group=None, nslabs: int | None = None, index: int | None = None, device=None):
        if (nslabs is None) != (index is None):
            raise ValueError("give both nslabs and index, or neither")
        self.local = nslabs is not None
        self.group = group
        if self.local:
            self.nslabs, self.index = int(nslabs), int(index)
        elif dist.is_initialized():
            self.nslabs, self.index = dist.get_world_size(group), dist.get_rank(group)
        else:
            self.nslabs, self.index = 1, 0
        self.nx, self.ny = int(nx), int(ny)
        self.y0, self.y1 = slab_rows(self.ny, self.nslabs, self.index)
        self.lattice = Lattice(self.nx, self.y1 - self.y0, theta, tau, model, prec, device=device)
        nbytes = capi.lbm_halo_bytes(self.lattice.ctx)
        # send up, send down, receive from below, receive from above (each 512-byte aligned)
        stride = (nbytes + 511) // 512 * 512
        self._faces = torch.empty(4 * stride, dtype=torch.uint8, device=self.lattice.device)
        self.send_up, self.send_down, self.recv_below, self.recv_above = (
            self._faces[k * stride:k * stride + nbytes] for k in range(4))

    # -- lifecycle
    def close(self) -> None:
        self.lattice.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def ctx(self):
        return self.lattice.ctx

    @property
    def stream(self):
        return self.lattice.stream

    def _rows(self, t: torch.Tensor, name: str) -> torch.Tensor:
        """The slab's rows of a whole-lattice field (last two dims (ny, nx)); a field that
        already has the slab's shape is taken as is."""
        if t.shape[-2] == self.ny and self.y1 - self.y0 != self.ny:
            return t[..., self.y0:self.y1, :]
        if t.shape[-2] != self.y1 - self.y0:
            raise ValueError(f"{name} must have {self.ny} rows (whole lattice) or {self.y1 - self.y0} (this slab)")
        return t

    # -- state
    def init(self, rho, ux, uy) -> None:
        """Guided equilibrium (Eq. 10) of the given fields (the slab's rows need nothing from
        its neighbours until the first step)."""
        self.lattice.init(*(self._rows(t, n) for t, n in ((rho, "rho"), (ux, "ux"), (uy, "uy"))))

    def set_state(self, f: torch.Tensor) -> None:
        self.lattice.set_state(self._rows(f, "f"))

    def state(self) -> torch.Tensor:
        """Populations f(x, t) of the slab's rows, (9, y1 - y0, nx)."""
        return self.lattice.state()

    def moments(self):
        return self.lattice.moments()

    # -- stepping
    def step(self, n: int = 1) -> None:
        if self.local:
            raise RuntimeError("a slab of several in one process is advanced by step_slabs")
        for _ in range(int(n)):
            self.lattice.step(1)
            self.exchange()

    def exchange(self) -> None:
        """Pack the faces, trade them with the neighbouring ranks, unpack what arrived."""
        if self.local:
            raise RuntimeError("a slab of several in one process trades its faces in step_slabs")
        with torch.cuda.device(self.lattice.device), torch.cuda.stream(self.lattice.stream):
            capi.lbm_halo_pack(self.ctx, self.send_up.data_ptr(), self.send_down.data_ptr())
            halo_exchange(self.send_up, self.send_down, self.recv_below, self.recv_above, self.group)
            capi.lbm_halo_unpack(self.ctx, self.recv_below.data_ptr(), self.recv_above.data_ptr())

    def set_diagnostics_interval(self, every: int) -> None:
        self.lattice.set_diagnostics_interval(every)

    # -- the whole lattice's diagnostics
    def diagnostics(self, raise_nonfinite: bool = True):
        out = self.lattice.diagnostics(raise_nonfinite=False)
        return self._global(out, raise_nonfinite)

    def step_diagnostics(self, raise_nonfinite: bool = True):
        out, t, _ = self.lattice.step_diagnostics(raise_nonfinite=False)
        return self._global(out, raise_nonfinite), t

    def _global(self, out5, raise_nonfinite: bool):
        g = out5 if self.local else global_diagnostics(out5, self.lattice.device, self.group)
        if raise_nonfinite and g[4] > 0:
            raise capi.LBMError(capi.LBM_ENONFINITE, f"{g[4]:.0f} node(s) hold non-finite populations")
        return g


def _ring(slabs) -> None:
    if not slabs:
        raise ValueError("no slabs")
    k = len(slabs)
    if sorted(s.index for s in slabs) != list(range(k)) or any(not s.local or s.nslabs != k for s in slabs):
        raise ValueError("step_slabs takes every slab of one split, each built with nslabs and index")
    if any(s.lattice.stream != slabs[0].lattice.stream or s.lattice.device != slabs[0].lattice.device
           for s in slabs):
        raise ValueError("the slabs of one process must share a device and a stream")


def exchange_slabs(slabs) -> None:
    """The face trade of every slab of one process: all pack, then each unpacks its
    neighbours' buffers (one stream orders the two phases)."""
    _ring(slabs)
    by_index = sorted(slabs, key=lambda s: s.index)
    with torch.cuda.device(by_index[0].lattice.device):
        for s in by_index:
            capi.lbm_halo_pack(s.ctx, s.send_up.data_ptr(), s.send_down.data_ptr())
        for s in by_index:
            below, above = (by_index[j] for j in neighbours(s.index, len(by_index)))
            capi.lbm_halo_unpack(s.ctx, below.send_up.data_ptr(), above.send_down.data_ptr())


def init_slabs(slabs, rho, ux, uy) -> None:
    """Initialise every slab of one process from the whole lattice's fields."""
    _ring(slabs)
    for s in slabs:
        s.init(rho, ux, uy)


def set_state_slabs(slabs, f: torch.Tensor) -> None:
    _ring(slabs)
    for s in slabs:
        s.set_state(f)


def step_slabs(slabs, n: int = 1) -> None:
    """Advance every slab of one process n steps in lock step, trading faces after each."""
    _ring(slabs)
    for _ in range(int(n)):
        for s in slabs:
            s.lattice.step(1)
        exchange_slabs(slabs)


def slabs_diagnostics(slabs, raise_nonfinite: bool = True):
    """The whole lattice's diagnostics (lbm_diagnostics) summed over the slabs of one process."""
    _ring(slabs)
    tot = [0.0] * 5
    for s in slabs:
        for j, v in enumerate(s.lattice.diagnostics(raise_nonfinite=False)):
            tot[j] += v
    if raise_nonfinite and tot[4] > 0:
        raise capi.LBMError(capi.LBM_ENONFINITE, f"{tot[4]:.0f} node(s) hold non-finite populations")
    return tot
