"""One molecule's hot path split over ranks (one process per GPU).

B: the unique pairs (rows of B_u) are cut into contiguous ranges, one per rank; rank k computes
the full-width rows of its range (lrtei_assemble_Bu_rows).  Rows are independent, so there is no
collective; a caller that needs the whole B on one device gathers the ranks' rows itself.

J-builds (eq. coulapprox): the same ranges split the rows of F_u.  X = F_u^T vec(D) is the sum of
the ranks' partial X (one all-reduce of R x n^3 numbers); every rank applies the node sum to the
summed X and writes J for its own pairs; J is the sum of the ranks' J (a second all-reduce).

The orchestration takes the two halves and the all-reduce as callables, so that the same code runs
with the CUDA library's lrtei_jbuild_partial_x / lrtei_jbuild_apply_x and torch.distributed on GPUs
and, in the CPU tests, with other implementations of the halves on gloo ranks.
"""
from __future__ import annotations

from typing import Callable, List, Tuple

from . import lrtei


def pair_ranges(npair: int, world: int, align: int = 128) -> List[Tuple[int, int]]:
    """Contiguous ranges [r0, r1) covering [0, npair) once, one per rank, of about equal length, each
    boundary rounded to a multiple of `align` (the tensor-core GEMMs' row blocks) where possible."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cuts = [0]
    for k in range(1, world):
        c = round(k * npair / world / align) * align
        cuts.append(min(npair, max(cuts[-1], c)))
    cuts.append(npair)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def jbuild_sharded(partial_x: Callable, apply_x: Callable, allreduce: Callable, npair: int, rank: int, world: int):
    """J of one rank's share, summed over ranks: X_k = partial_x(r0, r1); X = allreduce(X_k);
    J_k = apply_x(X, r0, r1); J = allreduce(J_k)."""
    r0, r1 = pair_ranges(npair, world)[rank]
    X = allreduce(partial_x(r0, r1))
    return allreduce(apply_x(X, r0, r1))


def b_rows_sharded(assemble_rows: Callable, npair: int, rank: int, world: int):
    """(r0, r1, rows of B_u [r0, r1)) of one rank: no collective."""
    r0, r1 = pair_ranges(npair, world)[rank]
    return r0, r1, assemble_rows(r0, r1)


# ------------------------------------------------------------------ the CUDA library's halves

def gpu_halves(plan: "lrtei.Plan", D):
    """(partial_x, apply_x) of a plan and CUDA densities D (R x N_b x N_b)."""
    import torch
    R = D.shape[0]
    n3 = plan.info["n"] ** 3

    def partial_x(r0, r1):
        X = torch.empty((R, n3), dtype=torch.float64, device=D.device)
        lrtei.lrtei_jbuild_partial_x(plan.plan, D, R, r0, r1, X)
        return X

    def apply_x(X, r0, r1):
        J = torch.empty_like(D)
        lrtei.lrtei_jbuild_apply_x(plan.plan, X, R, r0, r1, J)
        return J

    return partial_x, apply_x


def gpu_b_rows(plan: "lrtei.Plan", form: str = "auto"):
    def assemble_rows(r0, r1):
        return plan.Bu_rows(r0, r1, form)
    return assemble_rows


def torch_allreduce(t):
    """Sum over the process group (no-op without one)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t)
    return t
