"""Torch-facing helpers: device workspace, current stream, plan lifetime.

PyTorch provides the device memory (one uint8 workspace tensor per plan)
and the stream; every step of the contraction runs in the library's CUDA
kernels behind the C ABI.  There is no CPU path: without the built library
or a CUDA device these helpers raise.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as qb

DTYPES = {"c128": qb.QT_C128, "c64": qb.QT_C64, "c64x2": qb.QT_C64X2}
MODES = {"per_bucket": qb.QT_MODE_PER_BUCKET, "persistent": qb.QT_MODE_PERSISTENT}
QUEUE_ORDERS = {"round_robin": 0, "critical_path": 1, "simulated": 2}


def _stream_handle(device):
    return torch.cuda.current_stream(device).cuda_stream


class EnergyPlan:
    """All edge lightcones of one graph, planned once for `batch` angle sets.

    ``energy(gamma, beta)`` takes float64 CUDA tensors of shape [batch, p] and
    returns E[batch] (and per-edge <Z_j Z_k> if asked), asynchronously on the
    current stream.  ``energy_host`` takes numpy arrays and synchronises.
    """

    def __init__(self, n_vertices, edges, p, batch=1, dtype="c128", mode="persistent",
                 max_workspace=0, max_width=0, device="cuda:0", gradient=False, lane_items=0,
                 group_rows=0, edge_range=None, slice=False, chunk_tiles=0, order_trials=0, order_seed=0,
                 order_tau=1.0, checkpoint_bytes=0, chain_steps=False,
                 queue_order="simulated", chunk_tiles_by_rank=None, fuse_chains=3):
        self.n_vertices, self.p, self.batch = int(n_vertices), int(p), int(batch)
        self.edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        self.device = torch.device(device)
        self.edge_range = (0, len(self.edges)) if edge_range is None else tuple(int(x) for x in edge_range)
        self.options = dict(batch=batch, dtype=dtype, mode=mode, max_workspace=max_workspace,
                            max_width=max_width, gradient=gradient, lane_items=lane_items,
                            group_rows=group_rows, edge_range=self.edge_range, slice=slice,
                            chunk_tiles=chunk_tiles, order_trials=order_trials, order_seed=order_seed,
                            order_tau=order_tau,
                            checkpoint_bytes=checkpoint_bytes, chain_steps=chain_steps,
                            queue_order=queue_order, chunk_tiles_by_rank=chunk_tiles_by_rank,
                            fuse_chains=fuse_chains)
        opt = self._plan_options()
        self.plan = qb.qt_plan_create(self.n_vertices, self.edges, self.p, opt)
        self.ws_bytes = qb.qt_plan_workspace_size(self.plan)
        self.stats = qb.qt_plan_stats(self.plan)
        self.widths = qb.qt_plan_edge_widths(self.plan, self.n_edges)
        self.slices = qb.qt_plan_edge_slices(self.plan, self.n_edges)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def _plan_options(self, **override):
        """The plan options of this plan (qt_plan_options), with any field overridden."""
        o = dict(self.options, **override)
        opt = qb.qt_plan_options_default()
        opt.batch = self.batch
        opt.dtype = DTYPES[o["dtype"]]
        opt.mode = MODES[o["mode"]]
        opt.gradient = int(bool(o["gradient"]))
        opt.max_width = int(o["max_width"])
        opt.max_workspace = int(o["max_workspace"])
        opt.lane_items = int(o["lane_items"])
        opt.group_rows = int(o["group_rows"])
        opt.edge_begin, opt.edge_end = self.edge_range
        opt.slice = int(bool(o["slice"]))
        opt.chunk_tiles = int(o["chunk_tiles"])
        opt.order_trials = int(o["order_trials"])
        opt.order_seed = int(o["order_seed"])
        opt.order_tau = float(o["order_tau"])
        opt.checkpoint_bytes = int(o["checkpoint_bytes"])
        opt.chain_steps = int(bool(o["chain_steps"]))
        opt.queue_order = QUEUE_ORDERS[o["queue_order"]]
        for r, t in (o["chunk_tiles_by_rank"] or {}).items():  # {output rank: warp tiles per queue task}
            opt.chunk_tiles_by_rank[int(r)] = int(t)
        opt.fuse_chains = int(o["fuse_chains"])  # consumers fused into a step at most (0: none)
        return opt

    def bucket_bytes(self):
        """Algorithmic bytes of one evaluation counted bucket by bucket (every
        bucket's intermediate inputs read and its result written), as if no
        bucket were fused with its consumers: the figure a roofline divides.
        The chained steps of this plan store and read fewer bytes
        (``stats["alg_bytes"]``).  Plans the same orders on the host; no
        device memory."""
        if int(self.options["fuse_chains"]) == 0 or self.options["gradient"]:
            return self.stats["alg_bytes"]
        h = qb.qt_plan_create(self.n_vertices, self.edges, self.p, self._plan_options(fuse_chains=0))
        try:
            return qb.qt_plan_stats(h)["alg_bytes"]
        finally:
            qb.qt_plan_free(h)

    @property
    def n_edges(self):
        """Edges covered by this plan (its edge range)."""
        return self.edge_range[1] - self.edge_range[0]

    def energy(self, gamma, beta, edge_zz=False, grad=False, out=None):
        B, p = self.batch, self.p
        for t in (gamma, beta):
            if t.dtype != torch.float64 or t.device != self.device or tuple(t.shape) != (B, p):
                raise ValueError(f"angles must be float64 [{B}, {p}] on {self.device}")
        gamma, beta = gamma.contiguous(), beta.contiguous()
        energy = out if out is not None else torch.empty(B, dtype=torch.float64, device=self.device)
        zz = torch.empty((self.n_edges, B, 2), dtype=torch.float64, device=self.device) if edge_zz else None
        g = torch.empty((B, 2 * p), dtype=torch.float64, device=self.device) if grad else None
        qb.qt_plan_energy(self.plan, gamma.data_ptr(), beta.data_ptr(), energy.data_ptr(),
                          zz.data_ptr() if zz is not None else 0, g.data_ptr() if g is not None else 0,
                          self.workspace.data_ptr(), self.ws_bytes, _stream_handle(self.device))
        res = [energy]
        if edge_zz:
            res.append(zz)
        if grad:
            res.append(g)
        return res[0] if len(res) == 1 else tuple(res)

    def check(self):
        """Synchronise and raise if a device-side wait timed out."""
        qb.qt_plan_check(self.plan, _stream_handle(self.device))

    def trace(self, gamma, beta, grad=False):
        """Evaluate once with queue tracing on and return (trace, tasks):
        trace is a uint64 array [n_tasks, 4] of (claimed, ready, done) device
        clock readings in ns and (SM << 16 | warp); tasks the queue entries
        (``binding.qt_plan_tasks``).  Persistent plans only."""
        n = qb.qt_plan_trace_size(self.plan)
        buf = torch.zeros(max(n, 8), dtype=torch.uint8, device=self.device)
        qb.qt_plan_set_trace(self.plan, buf.data_ptr(), n)
        try:
            self.energy(gamma, beta, grad=grad)
            self.check()
        finally:
            qb.qt_plan_set_trace(self.plan, 0, 0)
        tr = buf[:n].cpu().numpy().view(np.uint64).reshape(-1, 4)
        return tr, qb.qt_plan_tasks(self.plan)

    def capture(self, edge_zz=False, grad=False):
        """Capture one evaluation of this plan as a CUDA graph (``CapturedEnergy``)."""
        return CapturedEnergy(self, edge_zz=edge_zz, grad=grad)

    def energy_host(self, gamma, beta, edge_zz=False, grad=False):
        B, p = self.batch, self.p
        ga = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(B, p))
        be = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(B, p))
        energy = np.empty(B)
        zz = np.empty((self.n_edges, B, 2)) if edge_zz else None
        g = np.empty((B, 2 * p)) if grad else None
        qb.qt_plan_energy_host(self.plan, ga, be, energy, zz, g, self.workspace.data_ptr(), self.ws_bytes,
                               _stream_handle(self.device))
        res = [energy] + ([zz] if edge_zz else []) + ([g] if grad else [])
        return res[0] if len(res) == 1 else tuple(res)

    def close(self):
        if getattr(self, "plan", None):
            qb.qt_plan_free(self.plan)
            self.plan = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CapturedEnergy:
    """One plan evaluation (angle table, leaf factors, the persistent bucket
    launch, the FP64 energy sum and, for gradient plans, the leaf-gradient
    kernels) captured once as a CUDA graph and replayed per call.

    The graph reads the angles from static device tensors and writes static
    outputs, so ``__call__`` copies the new angles in, replays the graph on
    the current stream and returns the static outputs (overwritten by the
    next replay; clone them to keep them).  A first direct call, outside the
    capture, binds the plan to its workspace (that call uploads the plan's
    descriptors and synchronises, which a capture cannot hold).
    """

    def __init__(self, plan, edge_zz=False, grad=False):
        self.plan = plan
        dev = plan.device
        B, p = plan.batch, plan.p
        self.gamma = torch.zeros((B, p), dtype=torch.float64, device=dev)
        self.beta = torch.zeros((B, p), dtype=torch.float64, device=dev)
        self.kw = dict(edge_zz=edge_zz, grad=grad)
        plan.energy(self.gamma, self.beta, **self.kw)
        plan.check()
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side, capture_error_mode="thread_local"):
                self.outputs = plan.energy(self.gamma, self.beta, **self.kw)
        torch.cuda.current_stream(dev).wait_stream(side)

    def replay(self):
        """Replay the captured evaluation on the static angle tensors."""
        self.graph.replay()
        return self.outputs

    def __call__(self, gamma, beta):
        self.gamma.copy_(gamma)
        self.beta.copy_(beta)
        return self.replay()


class QAOAEnergy(torch.autograd.Function):
    """E(gamma, beta) of a gradient plan as an autograd function.

    ``QAOAEnergy.apply(gamma, beta, plan)`` takes real float64 [B, p] CUDA
    tensors and returns E[B].  When either angle tensor requires a gradient,
    the forward call also runs the plan's adjoint bucket sweep (one call of
    the library computes E and dE/dgamma, dE/dbeta for all B angle sets) and
    keeps the gradient; backward scales it by grad_output.  Complex tensors
    never reach autograd.
    """

    @staticmethod
    def forward(ctx, gamma, beta, plan):
        p = plan.p
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            if not plan.options["gradient"]:
                raise qb.QTError(qb.QT_ESTATE, "angles require a gradient but the plan has no adjoint sweep")
            e, g = plan.energy(gamma.detach(), beta.detach(), grad=True)
            ctx.save_for_backward(g)
        else:
            e = plan.energy(gamma.detach(), beta.detach())
        ctx.p = p
        return e

    @staticmethod
    def backward(ctx, grad_energy):
        (g,) = ctx.saved_tensors
        go = grad_energy.reshape(-1, 1)
        return go * g[:, :ctx.p], go * g[:, ctx.p:], None


def qaoa_energy(plan, gamma, beta):
    """E[B] for angle tensors [B, p]; differentiable through ``QAOAEnergy``."""
    return QAOAEnergy.apply(gamma, beta, plan)


def autotune(n_vertices, edges, p, batch=1, dtype="c64", gradient=False, device="cuda:0", reps=3,
             lane_items=None, group_rows=(0, -1, 32), max_workspace=0, edge_range=None, gamma=None, beta=None,
             **plan_options):
    """Pick the warp-tile size and bucket grouping of a persistent plan by
    timing each candidate on the device (CUDA events around `reps` calls after
    two warm-ups).  Returns (best_options, {candidate: ms}).  Angles default
    to zeros (the work does not depend on their values).  Further keyword
    arguments (order_trials, chain_steps, ...) go to every candidate plan."""
    device = torch.device(device)
    if lane_items is None:
        lane_items = (16, 32, 64) if batch >= 16 else (8, 16, 32)
    g = torch.zeros((batch, p), dtype=torch.float64, device=device) if gamma is None else gamma
    b = torch.zeros((batch, p), dtype=torch.float64, device=device) if beta is None else beta
    timings = {}
    for li in lane_items:
        for gr in group_rows:
            plan = EnergyPlan(n_vertices, edges, p, batch=batch, dtype=dtype, mode="persistent",
                              gradient=gradient, device=device, lane_items=li, group_rows=gr,
                              max_workspace=max_workspace, edge_range=edge_range, **plan_options)
            for _ in range(2):
                plan.energy(g, b, grad=gradient)
            plan.check()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(reps):
                plan.energy(g, b, grad=gradient)
            t1.record()
            torch.cuda.synchronize(device)
            plan.check()
            timings[(li, gr)] = t0.elapsed_time(t1) / reps
            plan.close()
            del plan
            torch.cuda.empty_cache()
    li, gr = min(timings, key=timings.get)
    return dict(lane_items=li, group_rows=gr), timings


WIDTH_BANDS = ((18, 31), (14, 17), (0, 13))


def autotune_bands(n_vertices, edges, p, batch=1, dtype="c64", gradient=False, device="cuda:0", reps=3,
                   spans=(1, 2, 4), bands=WIDTH_BANDS, gamma=None, beta=None, **plan_options):
    """Per-width schedule: for each band of output ranks, the number of warp
    tiles one queue task takes (``chunk_tiles_by_rank``), picked by timing on
    the device with the other plan options fixed.  Bands are tuned one after
    another (the widest first, where most bytes move), each keeping the best
    choice of those before it; span 1 everywhere (the plan default) is the
    first candidate, so the result is never slower than it as timed.
    Returns ({rank: tiles}, {band: {"tiles_per_task": span, "ms_per_candidate": {span: ms}}})."""
    device = torch.device(device)
    g = torch.zeros((batch, p), dtype=torch.float64, device=device) if gamma is None else gamma
    b = torch.zeros((batch, p), dtype=torch.float64, device=device) if beta is None else beta

    def time_choice(choice):
        plan = EnergyPlan(n_vertices, edges, p, batch=batch, dtype=dtype, mode="persistent", gradient=gradient,
                          device=device, chunk_tiles_by_rank=choice, **plan_options)
        for _ in range(2):
            plan.energy(g, b, grad=gradient)
        plan.check()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            plan.energy(g, b, grad=gradient)
        t1.record()
        torch.cuda.synchronize(device)
        plan.check()
        ms = t0.elapsed_time(t1) / reps
        plan.close()
        del plan
        torch.cuda.empty_cache()
        return ms

    choice = {}
    timings = {}
    base = time_choice({})
    for lo, hi in bands:
        band = f"rank {lo}-{hi}"
        timings[band] = {1: base}
        best_span, best_ms = 1, base
        for sp in spans:
            if sp == 1:
                continue
            trial = dict(choice)
            trial.update({r: sp for r in range(lo, hi + 1)})
            ms = time_choice(trial)
            timings[band][sp] = ms
            if ms < best_ms:
                best_span, best_ms = sp, ms
        if best_span != 1:
            choice.update({r: best_span for r in range(lo, hi + 1)})
        base = best_ms
        timings[band] = {"tiles_per_task": best_span, "ms_per_candidate": timings[band]}
    return choice, timings


def contract_edge(n_vertices, edges, p, gamma, beta, edge, dtype="c128", device="cuda:0"):
    """<Z_j Z_k> of one edge through qt_build_lightcone / qt_order / qt_contract.
    Returns (value, width)."""
    net = qb.qt_build_lightcone(n_vertices, edges, p, gamma, beta, edge)
    try:
        order, width = qb.qt_order(net)
        nbytes = qb.qt_contract_workspace_size(net, order, DTYPES[dtype])
        ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        val = qb.qt_contract(net, order, DTYPES[dtype], _stream_handle(torch.device(device)), ws.data_ptr(), nbytes)
    finally:
        qb.qt_network_free(net)
    return val, width
