"""Band-sharded solve over several GPUs (one process per GPU).

The opacity bands of the multi-band scheme are independent transfer problems
(paper Sect. 1, multi-band opacity binning; Sect. 6 scales the 4-band 288^3
case over GPUs): each rank solves a contiguous slice of the bands on its own
GPU, and the band sums J = sum_b J_b, F = sum_b F_b, Q_rad = sum_b Q_b are
formed by one all-reduce of the five FP64 fields (the only exchange). The
emergent intensities I_top stay with the rank that solved their band.

The partition and the reduction are plain functions so that they can be
checked without a GPU (tests run them on gloo ranks with the CPU oracle as
the local solve); ShardedSolver puts them around the CUDA library's Solver.
"""
from __future__ import annotations


def band_partition(nbands: int, world: int, rank: int):
    """Contiguous slice [b0, b1) of the bands owned by `rank`: the first
    nbands % world ranks take one band more. A rank may own no band when
    world > nbands (it then contributes zeros to the reduction)."""
    if nbands < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad partition request: nbands={nbands}, world={world}, rank={rank}")
    base, extra = divmod(nbands, world)
    b0 = rank * base + min(rank, extra)
    return b0, b0 + base + (1 if rank < extra else 0)


def reduce_band_sums(J, F, Q, group=None):
    """Sum the ranks' partial band sums in place (J, F, Q: tensors of the
    same shape on every rank; CUDA tensors with NCCL, CPU tensors with
    gloo). One all-reduce per field; F carries its three components."""
    import torch.distributed as dist

    for t in (J, F, Q):
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


class ShardedSolver:
    """The bands [b0, b1) of an nbands problem on this rank's GPU.

    solve(chi, S) takes this rank's band slice ([b1-b0, nz, ny, nx], CUDA
    tensors) and returns J, F, Q_rad summed over all ranks' bands and this
    rank's I_top slice. Every rank must call solve (the reduction is
    collective); a rank with no band passes empty tensors."""

    def __init__(self, nx, ny, nz, nbands, group=None, **solver_opts):
        import torch
        import torch.distributed as dist

        from . import Solver

        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.b0, self.b1 = band_partition(nbands, self.world, self.rank)
        self.nx, self.ny, self.nz, self.nbands = nx, ny, nz, nbands
        self.local = Solver(nx, ny, nz, self.b1 - self.b0, **solver_opts) if self.b1 > self.b0 else None
        self.torch = torch

    def solve(self, chi, S, out=None, check=True, **kw):
        torch = self.torch
        dev = chi.device
        if self.local is not None:
            out = self.local.solve(chi, S, out=out, check=check, **kw)
        else:
            if out is None:
                out = dict(I_top=None, J=torch.zeros((self.nz, self.ny, self.nx), dtype=torch.float64, device=dev),
                           F=torch.zeros((3, self.nz, self.ny, self.nx), dtype=torch.float64, device=dev),
                           Q=torch.zeros((self.nz, self.ny, self.nx), dtype=torch.float64, device=dev))
            else:
                for k in ("J", "F", "Q"):
                    out[k].zero_()
        if self.world > 1:
            reduce_band_sums(out["J"], out["F"], out["Q"], self.group)
        return out
