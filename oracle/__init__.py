"""CPU FP64 oracle for QAOA MaxCut lightcone energies (arXiv:2106.15740).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline arm of ``bench.py`` use it.  It shares no code with the CUDA path;
the only module both sides import is the seeded input generator
``workloads.py``, which holds none of the method's arithmetic.

Contents, each written from the paper's statement of the problem:

* ``statevector``  -- dense 2^n FP64 simulation of the QAOA ansatz, eq. (1)
  and eq. (2) of §QAOA algorithm, with the MaxCut cost of the same section.
* ``closed_form``  -- the published p=1 formula for <Z_j Z_k> on a general
  graph (Wang, Hadfield, Jiang, Rieffel, PRA 97, 022304 (2018)), restated in
  this library's convention.
* ``lightcone``    -- the per-edge reverse-lightcone tensor network with
  diagonal gates kept on shared indices (§Diagonal gate simplification), the
  greedy min-fill elimination order, a naive bucket elimination
  (§Tensor network contraction) and a literal Feynman-path sum of eq. (tn).
* ``default_net``  -- the same network without the diagonal simplification
  (4-index ZZ tensors, the "Default" representation of §Results).
* ``gradients``    -- central finite differences and parameter-shift
  gradients of the energy.

Convention used everywhere (one reading of the paper, see §QAOA algorithm
and Fig. 1): the ZZ gate of layer q on edge (j,k) is exp(-i gamma_q Z_j Z_k),
the mixer is RX(2 beta_q) = exp(-i beta_q X), layer q applies all ZZ gates
then all mixers, the initial state is |+>^n, and
E = sum_{(j,k) in E} (1 - <Z_j Z_k>) / 2.

Parity status: every function here is pinned by a test under ``tests/``
(``-m "not gpu"``) against something other than itself -- the paper's Fig. 1
circuit, the published p=1 closed form, scipy's matrix exponential, brute
force, and invariants.  The only unpinned property is the optimality of the
greedy order, which the paper does not define (parity unpinned: order quality).
"""
