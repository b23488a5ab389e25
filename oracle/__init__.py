"""CPU oracle for the assembly-free deflated FE hot path (arXiv 2203.15115).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path: it assembles the global stiffness K explicitly in FP64
(scipy CSR), solves K u = f directly or by plain Jacobi-PCG, and evaluates
compliance, element sensitivities, the level-set threshold and the
augmented-Lagrangian scalar updates from their plain definitions, each function
citing the passage of the paper it follows.

Readings of points where the paper is silent (the element, its quadrature, the
coarse space) are stated in each function's docstring.

Parity pins: every function here is pinned in ``tests/test_oracle_*.py`` by
closed forms, invariants, exact rational integration or brute force, except
where a docstring says "parity unpinned".
"""
from . import fe, sensitivity, deflation, levelset  # noqa: F401
