"""GB300 (sm_103a) lightcone tensor-network QAOA MaxCut energies.

Method: arXiv:2106.15740, "Importance of Diagonal Gates in Tensor Network
Simulations" -- per-edge reverse-lightcone networks with diagonal gates kept
on shared indices, contracted by bucket elimination in greedy min-fill order
on hand-written CUDA kernels.

* ``binding``  -- ctypes binding of the C ABI (include/qtensor.h), same names.
* ``energy``   -- torch-facing helpers: device workspace, streams, plans.
* ``optimize`` -- multi-start angle optimisation driven by the adjoint gradient.
* ``sharding`` -- splitting a graph's edges between ranks.
"""
from . import binding  # noqa: F401
from .binding import QTError  # noqa: F401
