"""Single amplitudes <x| U(gamma, beta) |+>^n of the full QAOA circuit.

§Results: the paper's benchmark is the cost of one amplitude of the full
circuit.  ``AmplitudePlan`` plans one ket network per bitstring through
``qt_amplitude_plan_create`` (every qubit, diagonal ZZ phases on the qubits'
current indices, output indices fixed to the bits) and evaluates all of them
for B angle sets in one persistent launch; the values come back as a float64
tensor [n_strings, B, 2] (re, im).  PyTorch only provides the workspace and
the stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as qb
from .energy import DTYPES, MODES, _stream_handle


class AmplitudePlan:
    """Amplitudes of the bitstrings `bits` ([n_strings, n_vertices] of 0/1;
    qubit u is column u) for `batch` angle sets."""

    def __init__(self, n_vertices, edges, p, bits, batch=1, dtype="c128", mode="persistent", max_width=0,
                 slice=False, order_trials=0, order_seed=0, max_workspace=0, device="cuda:0"):
        self.n_vertices, self.p, self.batch = int(n_vertices), int(p), int(batch)
        self.bits = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8).reshape(-1, self.n_vertices))
        self.device = torch.device(device)
        opt = qb.qt_plan_options_default()
        opt.batch = self.batch
        opt.dtype = DTYPES[dtype]
        opt.mode = MODES[mode]
        opt.max_width = int(max_width)
        opt.slice = int(bool(slice))
        opt.order_trials = int(order_trials)
        opt.order_seed = int(order_seed)
        opt.max_workspace = int(max_workspace)
        self.plan = qb.qt_amplitude_plan_create(self.n_vertices, edges, self.p, self.bits, opt)
        self.n_strings = self.bits.shape[0]
        self.ws_bytes = qb.qt_plan_workspace_size(self.plan)
        self.stats = qb.qt_plan_stats(self.plan)
        self.widths = qb.qt_plan_edge_widths(self.plan, self.n_strings)
        self.slices = qb.qt_plan_edge_slices(self.plan, self.n_strings)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def amplitudes(self, gamma, beta, out=None):
        """Amplitudes [n_strings, B, 2] for float64 angle tensors [B, p] on the
        plan's device (asynchronous on the current stream)."""
        B, p = self.batch, self.p
        for t in (gamma, beta):
            if t.dtype != torch.float64 or t.device != self.device or tuple(t.shape) != (B, p):
                raise ValueError(f"angles must be float64 [{B}, {p}] on {self.device}")
        gamma, beta = gamma.contiguous(), beta.contiguous()
        amp = out if out is not None else torch.empty((self.n_strings, B, 2), dtype=torch.float64, device=self.device)
        qb.qt_plan_amplitudes(self.plan, gamma.data_ptr(), beta.data_ptr(), amp.data_ptr(), self.workspace.data_ptr(),
                              self.ws_bytes, _stream_handle(self.device))
        return amp

    def check(self):
        qb.qt_plan_check(self.plan, _stream_handle(self.device))

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
