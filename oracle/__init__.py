"""CPU FP64 oracle for the DNN-MG fine-level correction step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2008_11520_gb300``) never imports it, and this package
imports nothing from the product path: the two share no code.  Inputs are plain
NumPy arrays (the seeded generators that feed both sides hold none of the
method's arithmetic).

The oracle follows the paper (Margenberg, Hartmann, Lessig, Richter, "A neural
network multigrid solver for the Navier-Stokes equations", arXiv 2008.11520)
step by step, in float64, written for a reader checking it against the paper:

* ``mesh``      -- structured channel mesh, obstacle mask, node classes, patches
                   (Sec. 5.2 "A patch-based neural network", Sec. 6.1 Fig. geom).
* ``transfer``  -- prolongation P (interpolation) and restriction R = P^T
                   (Sec. 3.4, mesh transfer; the first and last stages of Algorithm 2's correction).
* ``fem``       -- Q1 Crank-Nicolson residual and right-hand side with local
                   projection stabilisation (Eq. nonlinearshort, Eq. 4cranknicholson3).
* ``features``  -- per-patch network inputs (Sec. 5.2 "Neural network inputs").
* ``gru``       -- GRU cell and fully connected output layer (Eq. gru, Sec. 6.2).
* ``head``      -- convolutional head of the K = 1 network and its fold into the
                   output layer (Sec. 6.2 parameter counts).
* ``average``   -- averaging of duplicate predictions on shared nodes (Sec. 5.2).
* ``step``      -- one DNN-MG correction step of Algorithm 2.

Parity status: every function above is pinned by tests under ``tests/`` that
check it against closed forms, invariants, hand-computed values and brute force
(see ``tests/test_oracle_pins.py``); the composed step has no closed form beyond
its parts and the zero-network reduction.
"""

from . import mesh, transfer, fem, features, gru, head, average, step  # noqa: F401
