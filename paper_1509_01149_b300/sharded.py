"""K-sharded MPPI: one controller's samples split over the ranks of a torch.distributed group.

The K samples of one iteration are independent (the sampling loop of Algorithm 1), so each
rank rolls out a contiguous range of them and the ranks exchange one small partial each
(rho_r, k*_r, eta_r and the T*m weighted sums N_r, all relative to the rank's own minimum:
TM + 3 doubles, the layout of mppi_shard_partial_async).  One all-gather per iteration
gives every rank all R partials in rank order; each rank merges them the same way
(mppi_shard_update_async: Eq. App_PI with the min shift, FP64) and holds the same controls.

The exchange is the only collective on the data path.  With the NCCL backend the partials
stay on the device; with gloo they go through host memory.
"""
from __future__ import annotations

import math

import numpy as np

SHARD_ALIGN = 128      # shard boundaries: multiples of every rollout block's sample count


def shard_range(K: int, rank: int, world: int, align: int = SHARD_ALIGN) -> tuple[int, int]:
    """(k_begin, k_count) of `rank`: contiguous ranges in rank order covering [0, K), boundaries
    multiples of `align` (the last range ends at K), as even as `align` allows.  A rank may get
    an empty range when K has fewer than `world` aligned units."""
    if not (0 <= rank < world) or K < 1 or align < 1:
        raise ValueError("bad shard arguments")
    units = math.ceil(K / align)
    per, extra = divmod(units, world)
    u0 = rank * per + min(rank, extra)
    u1 = u0 + per + (1 if rank < extra else 0)
    k0, k1 = min(K, u0 * align), min(K, u1 * align)
    return k0, k1 - k0


def empty_partial(TM: int) -> np.ndarray:
    """The partial of a rank without samples: no finite cost, nothing to add."""
    p = np.zeros(TM + 3, dtype=np.float64)
    p[0] = np.inf
    p[1] = float(2 ** 31 - 1)
    return p


def exchange_partials(local, group=None):
    """All-gather one partial [TM + 3] (a torch tensor) from every rank; returns [R][TM + 3] in
    rank order, on the same device as `local`."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(out, local.contiguous(), group=group)
    return torch.stack(out)


class ShardedController:
    """This rank's part of one K-sharded controller: a Controller created with the full K whose
    shard is set to this rank's range.  step() runs the rank's rollout and partial, the
    all-gather and the merge + update on the controller's stream, then the shift."""

    def __init__(self, ctrl, rank: int, world: int, device, group=None):
        import torch
        import torch.distributed as dist
        self.ctrl, self.rank, self.world, self.group = ctrl, rank, world, group
        self.k_begin, self.k_count = shard_range(ctrl.K, rank, world)
        if self.k_count > 0:
            ctrl.set_shard(self.k_begin, self.k_count)
        self.TM = ctrl.T * ctrl.m
        self.device = torch.device(device)
        self.host_exchange = dist.get_backend(group) != "nccl"
        self.partial = torch.tensor(empty_partial(self.TM), dtype=torch.float64, device=self.device)
        self.u0 = torch.zeros(ctrl.m, dtype=torch.float32, device=self.device)

    def step(self, d_state: int, stream) -> "torch.Tensor":
        """One sharded iteration + shift from the device state at address d_state; returns u0
        (device, [m]), ready on `stream` (the controller's stream)."""
        import torch
        with torch.cuda.stream(stream):
            if self.k_count > 0:
                self.ctrl.shard_partial_async(d_state, self.partial.data_ptr())
            if self.host_exchange:
                stream.synchronize()
                allp = exchange_partials(self.partial.cpu(), self.group).to(self.device)
            else:
                allp = exchange_partials(self.partial, self.group)
            self.ctrl.shard_update_async(allp.data_ptr(), self.world, self.u0.data_ptr())
            self.ctrl.shift()
        self._all = allp            # keep the gathered partials alive until the stream has used them
        return self.u0
