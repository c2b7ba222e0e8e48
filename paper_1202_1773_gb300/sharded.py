"""Plane-sharded transforms across the ranks of a process group.

The planes of the shearlet transform are independent (Sec. 3.1): rank r
computes the coefficients of its own contiguous plane range from fft2(f),
which every rank recomputes, so the forward has no exchange.  The inverse of
Sec. 3.3 is a sum over planes, sum_i psi_hat_i * fft2(c_i), followed by one
ifft2: each rank sums its planes into a partial half spectrum
(ffst_inverse_partial), one sum-reduce over the group combines them on the
root, and the root finishes (ffst_inverse_finish).  One process per GPU; the
reduce is the only collective, M x (N/2 + 1) complex64 per inverse.
"""

from __future__ import annotations


def plane_range(num_planes: int, world: int, rank: int):
    """Contiguous plane range [p0, p1) of `rank` among `world` ranks; the
    ranges are disjoint, cover every plane and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    if num_planes < world:
        raise ValueError(f"{num_planes} planes cannot be split over {world} ranks")
    return num_planes * rank // world, num_planes * (rank + 1) // world


def reduce_finish(partial, finish, group=None, root: int = 0):
    """The exchange step of the sharded inverse: sum the ranks' partial half
    spectra `partial` (a complex tensor, overwritten) onto `root` and return
    finish(sum) there; None on the other ranks."""
    import torch
    import torch.distributed as dist

    buf = torch.view_as_real(partial) if partial.is_complex() else partial
    dist.reduce(buf, dst=root, op=dist.ReduceOp.SUM, group=group)
    rank = dist.get_rank(group) if group is not None else dist.get_rank()
    return finish(partial) if rank == root else None


class ShardedPlan:
    """A libffst plan restricted to this rank's planes.

    forward(img) returns the local stack [p1 - p0, rows, cols]; inverse(local)
    returns the image on `root` and None elsewhere (every rank must call it).
    """

    def __init__(self, rows: int, cols: int, scales: int = 0, group=None, root: int = 0, device=None, **opts):
        import torch.distributed as dist

        from . import Plan

        self.group = group
        self.root = root
        self.world = dist.get_world_size(group) if group is not None else dist.get_world_size()
        self.rank = dist.get_rank(group) if group is not None else dist.get_rank()
        self.plan = Plan(rows, cols, scales, device=device, **opts)
        self.p0, self.p1 = plane_range(self.plan.num_planes, self.world, self.rank)
        self.plan.set_planes(self.p0, self.p1)

    @property
    def shape(self):
        return self.plan.shape

    def forward(self, img, out=None):
        return self.plan.forward(img, out=out)

    def inverse(self, local, out=None, normalise: bool = True):
        spec = self.plan.inverse_partial(local)
        return reduce_finish(spec, lambda s: self.plan.inverse_finish(s, normalise, out=out), self.group, self.root)

    def close(self):
        self.plan.close()
