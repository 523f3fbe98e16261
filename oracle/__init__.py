"""CPU oracle for the skeletonized-FMM apply — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct FP64 (complex128 for Helmholtz) code written
from the paper's definitions:

* ``direct``   — the summation problem itself, u_i = sum_{j != i} G(x_i,x_j) q_j
                 (Section 1, Eq. (1)-(3)), in numpy and in plain C/OpenMP.
* ``kernels``  — the Laplace and Helmholtz Green's functions (Eq. (2), Eq. (5))
                 plus an exactly low-rank polynomial kernel used only as a pin.
* ``tree``     — adaptive quad/oct-tree, 2:1 balance, colleague / coarse / fine
                 neighbor lists (Section 3.1).
* ``skeleton`` — proxy surfaces and column-pivoted-QR interpolative
                 decompositions, level by level (Section 2.1, Algorithm 1).
* ``apply``    — Algorithm 2 step by step (upward pass, ifo / ifs / tfo
                 translations, level-1 sum, downward pass).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The library under
``paper_2310_16668_gb300`` never imports it, and this package never imports the
library: the two share only the seeded input generators in
``paper_2310_16668_gb300.workloads``, which hold none of the method's
arithmetic.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, brute force, an exactly low-rank kernel for which the
skeleton apply must reproduce the direct sum, symmetry and tolerance decay).
"""
