"""Splitting one graph's edges between ranks, one GPU per rank.

The energy is a sum of independent edge terms (§QAOA algorithm: E is the sum
over edges of (1 - <Z_j Z_k>)/2, each term its own lightcone network), so a
graph shards by edges.  Each rank plans a contiguous edge range whose planned
algorithmic bytes are about equal to the other ranks' (the cost model of the
bucket kernels, which are bound by memory traffic), evaluates its partial
sums of E[B] and dE/dtheta[B, 2p] on its own GPU, and one FP64 all-reduce of
B * (1 + 2p) values gives every rank the totals.  That sum is the only
exchange of the path.

``ShardedEnergy`` is the torch-facing wrapper; ``edge_costs``, ``partition``
and ``reduce_partials`` are its host-side pieces.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as qb
from .energy import DTYPES, EnergyPlan


def edge_costs(n_vertices, edges, p, batch=1, dtype="c64", max_width=0, slice=False):
    """Algorithmic bytes per edge of one forward call, from a host-only plan
    (no device memory, no GPU needed)."""
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    opt = qb.qt_plan_options_default()
    opt.batch = int(batch)
    opt.dtype = DTYPES[dtype]
    opt.mode = qb.QT_MODE_PER_BUCKET
    opt.max_width = int(max_width)
    opt.slice = int(bool(slice))
    plan = qb.qt_plan_create(int(n_vertices), edges, int(p), opt)
    try:
        return qb.qt_plan_edge_bytes(plan, len(edges))
    finally:
        qb.qt_plan_free(plan)


def _greedy_ranges(costs, limit):
    """Cut before the edge that would take the running sum above `limit`."""
    ranges, start, acc = [], 0, 0.0
    for i, c in enumerate(costs):
        if i > start and acc + c > limit:
            ranges.append((start, i))
            start, acc = i, 0.0
        acc += c
    ranges.append((start, len(costs)))
    return ranges


def partition(costs, world):
    """Contiguous edge ranges [a_r, b_r), r = 0..world-1, covering every edge
    once in order, that minimise the largest range cost (bisection on the
    limit of a greedy cut, which is optimal for contiguous splits).  With
    fewer edges than ranks the last ranks get empty ranges."""
    costs = np.asarray(costs, dtype=np.float64)
    m = len(costs)
    world = int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    if m == 0:
        return [(0, 0)] * world
    lo, hi = float(costs.max()), float(costs.sum())
    for _ in range(100):
        if hi - lo <= 1e-12 * max(hi, 1.0):
            break
        mid = 0.5 * (lo + hi)
        if len(_greedy_ranges(costs, mid)) <= world:
            hi = mid
        else:
            lo = mid
    ranges = _greedy_ranges(costs, hi)
    # use every rank while there are edges to spare: split the costliest range
    while len(ranges) < world and any(b - a > 1 for a, b in ranges):
        k = max((i for i, (a, b) in enumerate(ranges) if b - a > 1), key=lambda i: costs[slice(*ranges[i])].sum())
        a, b = ranges[k]
        pre = np.cumsum(costs[a:b])
        cut = a + 1 + int(np.searchsorted(pre[:-1], pre[-1] / 2.0))
        cut = min(max(cut, a + 1), b - 1)
        ranges[k:k + 1] = [(a, cut), (cut, b)]
    while len(ranges) < world:
        ranges.append((m, m))
    return ranges


def reduce_partials(energy, grad=None, group=None):
    """Sum partial E[B] (and dE/dtheta[B, 2p]) over the ranks of `group`:
    one all_reduce of one packed FP64 tensor.  Returns the totals."""
    import torch.distributed as dist
    parts = [energy.reshape(-1)] + ([grad.reshape(-1)] if grad is not None else [])
    buf = torch.cat(parts).to(torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    e = buf[:energy.numel()].reshape(energy.shape)
    if grad is None:
        return e
    return e, buf[energy.numel():].reshape(grad.shape)


class ShardedEnergy:
    """E (and dE/dtheta) of one graph with its edges split over the ranks of
    a process group (torch.distributed; NCCL across GPUs).  Every rank calls
    ``energy`` with the same angles and gets the full totals."""

    def __init__(self, n_vertices, edges, p, batch=1, dtype="c64", group=None, device=None, costs=None,
                 max_width=0, slice=False, **plan_kw):
        import torch.distributed as dist
        dist_on = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if dist_on else 0
        self.world = dist.get_world_size(group) if dist_on else 1
        self.group = group
        self.p, self.batch = int(p), int(batch)
        self.device = torch.device(device if device is not None else f"cuda:{torch.cuda.current_device()}")
        if costs is None:
            costs = edge_costs(n_vertices, edges, p, batch, dtype, max_width, slice)
        self.ranges = partition(costs, self.world)
        a, b = self.ranges[self.rank]
        self.plan = None
        if b > a:
            self.plan = EnergyPlan(n_vertices, edges, p, batch=batch, dtype=dtype, edge_range=(a, b),
                                   max_width=max_width, slice=slice, device=self.device, **plan_kw)

    def energy(self, gamma, beta, grad=False):
        B, p = self.batch, self.p
        if self.plan is not None:
            res = self.plan.energy(gamma, beta, grad=grad)
            e, g = (res if grad else (res, None))
        else:
            e = torch.zeros(B, dtype=torch.float64, device=self.device)
            g = torch.zeros((B, 2 * p), dtype=torch.float64, device=self.device) if grad else None
        return reduce_partials(e, g, self.group)

    def check(self):
        if self.plan is not None:
            self.plan.check()
