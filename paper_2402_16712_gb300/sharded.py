"""One fit split across the ranks of a torch.distributed group.

Algorithm 1's outer loop over the preserved coordinate jhat is independent per
jhat: each z_jhat needs only its own m pairs.  Rank r of a world of size w
scores the contiguous jhat range [r m / w, (r + 1) m / w) on its own GPU (every
jhat costs the same: all m - 1 pairs of its column), which is
`l1line_fit_subset`.  The one exchange is Algorithm 1's argmin over jhat: per
lambda, the smallest objective, ties to the smallest jhat (the strict
improvement test scanning jhat upward), then v* from the rank that owns jhat*.
It takes three small collectives: an all-reduce MIN over the objectives' bit
patterns (z >= 0, so the bits order like the values), an all-reduce MIN over
the jhat of the ranks that hold that objective, and an all-reduce SUM of v rows
that only the owner fills (adding zeros leaves its entries unchanged).

Collectives run on CUDA tensors for the nccl backend and on host tensors
otherwise (gloo).
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import l1line

_NO_JHAT = np.iinfo(np.int64).max


def shard_range(m: int, rank: int, world: int):
    """The contiguous jhat range [lo, hi) of `rank`: equal counts (every jhat
    costs the same), the first m % world ranks one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(m, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def combine(obj, jstar, v, group=None):
    """Global (obj, jstar, v) from every rank's best over its own jhat range.

    obj [nl] float64, jstar [nl] int (-1: this rank scored no jhat), v [nl, m];
    all on the collective's device.  Returns new tensors on that device."""
    import torch
    import torch.distributed as dist

    obj = obj.to(torch.float64)
    none = jstar < 0
    zbits = obj.view(torch.int64).clone()
    zbits[none] = _NO_JHAT
    dist.all_reduce(zbits, op=dist.ReduceOp.MIN, group=group)
    mine = (obj.view(torch.int64) == zbits) & ~none
    jb = torch.where(mine, jstar.to(torch.int64), torch.full_like(zbits, _NO_JHAT))
    dist.all_reduce(jb, op=dist.ReduceOp.MIN, group=group)
    owner = mine & (jstar.to(torch.int64) == jb)
    vs = torch.where(owner[:, None], v, torch.zeros_like(v))
    dist.all_reduce(vs, op=dist.ReduceOp.SUM, group=group)
    return zbits.view(torch.float64), jb.to(torch.int32), vs


def fit_sharded(X, lambdas, group=None, workspace: Optional[l1line.Workspace] = None,
                stream=None):
    """Algorithm 1 on X (a CUDA tensor on this rank's device, the same matrix
    on every rank) with the jhat loop split over the ranks of `group`.
    Returns (v [nl, m], obj [nl], jstar [nl]) on X's device, identical on
    every rank; without an initialised process group it is one plain fit."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        v, obj, js, _ = l1line.fit(X, lambdas, workspace=workspace, stream=stream)
        return v, obj, js
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    m = X.shape[1]
    lo, hi = shard_range(m, rank, world)
    nl = np.atleast_1d(np.asarray(lambdas, dtype=np.float64)).size
    if hi > lo:
        jl = torch.arange(lo, hi, dtype=torch.int32, device=X.device)
        v, obj, js, _ = l1line.fit_subset(X, lambdas, jl, workspace=workspace, stream=stream)
        js = js.to(torch.int64)
    else:  # more ranks than columns
        v = torch.zeros((nl, m), dtype=X.dtype, device=X.device)
        obj = torch.zeros(nl, dtype=torch.float64, device=X.device)
        js = torch.full((nl,), -1, dtype=torch.int64, device=X.device)
    if stream is not None:
        stream.synchronize()
    comm = X.device if dist.get_backend(group) == "nccl" else torch.device("cpu")
    zg, jg, vg = combine(obj.to(comm), js.to(comm), v.to(comm), group)
    return vg.to(X.device), zg.to(X.device), jg.to(X.device)
