"""A GGArray partitioned over the ranks of a process group (one GPU per
rank): the LFVectors of one logical array are split into contiguous
ranges, rank r holding LFVectors [l0_r, l1_r) as its own GGArray.

The paper's LFVectors are independent (Sec. IV: each block grows its own
LFVector), so insertion needs no exchange: each rank inserts into its own
LFVectors.  The global view is the prefix sum of the LFVector sizes (Sec.
IV), which needs one exchange: an all-gather of the L per-LFVector sizes.
From it every rank knows the global offsets, so

* flatten is distributed: rank r's LFVectors form the contiguous slice
  [offsets[l0_r], offsets[l1_r]) of the flattened array, and its local
  flatten is exactly that slice (LFVector-major order is kept);
* a read of global index g goes to the rank whose slice holds g; requests
  travel in one all-to-all, are read there as local global indices
  (g minus the rank's base), and the values come back in a second one.

Only collectives of the process group move data between ranks (NCCL on
GPUs, gloo on CPUs): no kernel reads a peer's memory.  The local part is
any object with the three calls below -- the library's GGArray on a GPU
(`GGArrayPart`), or a CPU model in tests.
"""

from __future__ import annotations

import torch
import torch.distributed as dist


def lfv_range(L: int, world: int, rank: int):
    """Contiguous LFVector range [l0, l1) of `rank` when L LFVectors are split
    over `world` ranks (the first L % world ranks get one more)."""
    q, r = divmod(L, world)
    l0 = rank * q + min(rank, r)
    return l0, l0 + q + (1 if rank < r else 0)


class GGArrayPart:
    """The local part on a GPU: a GGArray of this rank's LFVectors."""

    def __init__(self, g):
        self.g = g

    def lfv_sizes(self) -> torch.Tensor:
        _, rc, sizes, _ = self.g.sizes_caps()
        if rc != 0:
            from .gga import GGAError
            raise GGAError(rc, "local part")
        return sizes.to(torch.int64)

    def read_local(self, idx: torch.Tensor) -> torch.Tensor:
        return self.g.read(idx)

    def flatten_local(self) -> torch.Tensor:
        return self.g.flatten()


class PartitionedGGArray:
    def __init__(self, local, L: int, world: int, rank: int, group=None, device=None):
        self.local, self.L, self.world, self.rank, self.group = local, L, world, rank, group
        self.device = device if device is not None else torch.device("cpu")
        self.l0, self.l1 = lfv_range(L, world, rank)
        self.offsets = None          # [L + 1] global prefix sum of sizes, after sync()
        self.rank_base = None        # [world + 1] first global index of every rank's slice

    def sync(self):
        """The one exchange of the global view: all-gather of every rank's
        LFVector sizes (after insertions, before global indexing)."""
        sizes = self.local.lfv_sizes().to(self.device, torch.int64)
        assert sizes.numel() == self.l1 - self.l0
        parts = [torch.zeros(b - a, dtype=torch.int64, device=self.device)
                 for a, b in (lfv_range(self.L, self.world, r) for r in range(self.world))]
        if self.world > 1:
            # all_gather needs equal sizes: pad to the largest range.
            width = max(p.numel() for p in parts)
            pad = torch.zeros(width, dtype=torch.int64, device=self.device)
            pad[:sizes.numel()] = sizes
            gathered = [torch.empty(width, dtype=torch.int64, device=self.device) for _ in range(self.world)]
            dist.all_gather(gathered, pad, group=self.group)
            parts = [g[:p.numel()] for g, p in zip(gathered, parts)]
        else:
            parts = [sizes]
        all_sizes = torch.cat(parts)
        self.offsets = torch.zeros(self.L + 1, dtype=torch.int64, device=self.device)
        self.offsets[1:] = torch.cumsum(all_sizes, 0)
        bounds = [lfv_range(self.L, self.world, r)[0] for r in range(self.world)] + [self.L]
        self.rank_base = self.offsets[torch.tensor(bounds, device=self.device)]
        return self.offsets

    def global_size(self) -> int:
        return int(self.offsets[-1])

    def flatten(self):
        """This rank's slice of the flattened array: (first global index,
        elements), the elements being the local flatten."""
        n = int(self.rank_base[self.rank + 1] - self.rank_base[self.rank])
        return int(self.rank_base[self.rank]), self.local.flatten_local()[:n]

    def read(self, gidx: torch.Tensor) -> torch.Tensor:
        """Values at global indices gidx (int64, every index < global size),
        in gidx's order: routed to the owning ranks and back."""
        gidx = gidx.to(self.device, torch.int64)
        owner = torch.searchsorted(self.rank_base[1:], gidx, right=True)
        order = torch.argsort(owner, stable=True)
        send_idx = gidx[order] - self.rank_base[owner[order]]
        send_counts = torch.bincount(owner, minlength=self.world)
        recv_counts = torch.empty_like(send_counts)
        if self.world > 1:
            dist.all_to_all_single(recv_counts, send_counts, group=self.group)
        else:
            recv_counts.copy_(send_counts)
        sc, rc = send_counts.tolist(), recv_counts.tolist()
        recv_idx = torch.empty(sum(rc), dtype=torch.int64, device=self.device)
        if self.world > 1:
            dist.all_to_all_single(recv_idx, send_idx, rc, sc, group=self.group)
        else:
            recv_idx.copy_(send_idx)
        vals = self.local.read_local(recv_idx)
        back = torch.empty((sum(sc),) + tuple(vals.shape[1:]), dtype=vals.dtype, device=self.device)
        if self.world > 1:
            dist.all_to_all_single(back, vals.contiguous(), sc, rc, group=self.group)
        else:
            back.copy_(vals)
        out = torch.empty_like(back)
        out[order] = back
        return out
