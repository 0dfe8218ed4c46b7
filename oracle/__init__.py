"""CPU FP64 oracle for the SIMP + Optimality Criteria hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import, call or execute
anything in this package.  The CUDA library never links or calls it, and it
shares no code, table or constant generator with the CUDA library.

Each function is a plain, slow, checkable restatement of what the paper
(Kim & Kang, "PyTopo3D", arXiv 2504.05604) says the method computes:

* ``fem``     -- hex8 element stiffness, assembly, boundary conditions,
                 direct and Jacobi-PCG solves, compliance and sensitivities
                 (Section 2.2, Section 2.3).
* ``filters`` -- the linear-decay sensitivity and density filters (Section 2.4).
* ``oc``      -- the Optimality Criteria update with bisection on the volume
                 Lagrange multiplier and move limits (Section 2.3).
* ``topopt``  -- the optimisation loop (Section 2.5).
* ``cnn``     -- naive FP64 3D convolutions, forward and backward, for the
                 learned U-Net preconditioner.
* ``mg``      -- the learned multigrid preconditioner: hierarchy, coarse
                 moduli, transfer operators, V-cycle and its training loss.

Parity status of each function is stated in its docstring; all functions
here are pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants or brute force.
"""
from . import fem, filters, mg, oc, topopt  # noqa: F401
