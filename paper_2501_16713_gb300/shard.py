"""Phase sharding of the nonrigid SENSE operator over ranks (one GPU each).

The stacked SENSE equation ("Nonrigid SENSE Operators") sums over motion
states: A^H y = sum_j A_j^H y_j and E x = sum_j A_j^H A_j x + lambda x.  Rank r
holds a plan of its own states J_r only (their displacements, trajectories and
k-space data); after each phase sum the library calls the plan's reduction
hook (nrsense_plan_set_reduce), which all-reduces the N^3 image over the
ranks.  Every rank then holds the same vectors, so the CG / flexible-CG /
FISTA iterations and their FP64 reductions run unchanged and identically on
every rank; per normal-operator application one image (8 N^3 bytes) crosses
the ranks, nothing else.

This module holds the host logic: the partition of the states into
contiguous blocks of balanced sample counts, and a plan wrapper that builds
the rank's plan and registers a torch.distributed all-reduce (NCCL on GPUs)
as its hook.  The partition and the composition of partial sums are checked
on CPU with gloo ranks; on GPUs the hook runs inside the library's entry
points.
"""

from __future__ import annotations

from typing import Callable, Sequence


def phase_partition(counts: Sequence[int], world: int) -> list[list[int]]:
    """Split motion states 0..P-1 into `world` contiguous blocks of balanced
    sample counts: block r ends at the first state where the running total
    reaches (r + 1) / world of the whole, with at least one state per block
    while states last (P < world leaves the last world - P blocks empty).
    Every state is in exactly one block."""
    P = len(counts)
    if world < 1:
        raise ValueError("world must be >= 1")
    cs = [int(c) for c in counts]
    if any(c < 0 for c in cs):
        raise ValueError("sample counts must be >= 0")
    if P <= world:
        return [[j] if j < P else [] for j in range(world)]
    prefix = [0]
    for c in cs:
        prefix.append(prefix[-1] + c)
    total = prefix[-1]
    cuts = [0]
    for r in range(1, world):
        lo, hi = cuts[-1] + 1, P - (world - r)  # keep a state for every later block
        k = hi
        for kk in range(lo, hi + 1):
            if prefix[kk] * world >= total * r:
                k = kk
                break
        cuts.append(k)
    cuts.append(P)
    return [list(range(cuts[r], cuts[r + 1])) for r in range(world)]


def local_rows(counts: Sequence[int], phases: Sequence[int]) -> list[tuple[int, int]]:
    """Row ranges [start, end) of the given states in the phase-major k-space
    data of all states (states in order, M_j rows each)."""
    starts = [0]
    for c in counts:
        starts.append(starts[-1] + int(c))
    return [(starts[j], starts[j + 1]) for j in phases]


def sharded_normal(x, local_normal: Callable, all_reduce: Callable, lam: float = 0.0):
    """E x on a rank: its states' partial sum sum_{j in J_r} A_j^H A_j x,
    all-reduced over the ranks, plus lambda x (added once, after the sum) --
    the composition the library performs with a reduction hook."""
    part = local_normal(x)
    total = all_reduce(part)
    return total + lam * x if lam != 0.0 else total


def torch_all_reduce(group=None):
    """A reduction hook body for Plan.set_reduce: in-place SUM all-reduce of
    the staged image over `group` (torch.distributed, NCCL for CUDA tensors)."""
    import torch.distributed as dist

    def fn(buf, stream):
        import torch
        # a complex image is summed as its real and imaginary parts
        dist.all_reduce(torch.view_as_real(buf), group=group)

    return fn


class ShardedPlan:
    """The plan of one rank's motion states with the all-reduce hook set.

    shape, disp (P, 3, n0, n1, n2), coords (list of P (M_j, 3) tensors) and
    smaps describe the whole problem; the rank keeps the states of its block
    of phase_partition(M, world).  forward/adjoint take and return the rank's
    rows of the phase-major k-space data (local_rows); normal, solve_cg and
    the other solvers return the full (replicated) image."""

    def __init__(self, shape, disp, coords, smaps, rank: int, world: int,
                 reduce: Callable | None = None, **plan_kw):
        from .nrsense import Plan
        counts = [int(c.shape[0]) for c in coords]
        self.counts = counts
        self.phases = phase_partition(counts, world)[rank]
        if not self.phases:
            raise ValueError(f"rank {rank} holds no motion state (world {world} > states)")
        self.rows = local_rows(counts, self.phases)
        self.plan = Plan(shape, disp=disp[self.phases], coords=[coords[j] for j in self.phases],
                         smaps=smaps, n_phases=len(self.phases), **plan_kw)
        self.plan.set_reduce(reduce if reduce is not None else torch_all_reduce())

    def local_data(self, y_all):
        """The rank's rows of phase-major data of all states."""
        import torch
        return torch.cat([y_all[a:b] for a, b in self.rows]).contiguous()

    def __getattr__(self, name):
        if name == "plan":
            raise AttributeError(name)
        return getattr(self.plan, name)

    def close(self):
        self.plan.set_reduce(None)
        self.plan.close()
