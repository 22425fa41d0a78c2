"""FP64 CPU oracle for complex constrained TV denoising and TV-regularised phase
retrieval (Gao & Cao, arXiv 2109.05496).

TEST INFRASTRUCTURE ONLY. It is the plain, slow reference the CUDA library is
checked against and shares no code with it. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and
``--impl reference``) may import it. The library must never route through it.

Modules:
    ops      D (Eq. (5)/(6)), its adjoint, TV (Eq. (3), (4), (7)-(10)),
             P_C (Eq. (26) + support) and P_S (Eq. (20), (33), (35), (37)).
    fgp      Algorithm 2 (FGP), Eq. (21) (GP), primal / dual / gap (Prop. 1, App. A).
    pr       Eq. (23), (24), (27) and Algorithm 1 (FISTA) / Eq. (14) (ISTA).
    exact    Small-problem solvers used to pin the above (brute force, closed forms).

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, brute force, finite differences); none is unpinned.
"""
from . import ops, fgp, pr  # noqa: F401
from .ops import Constraint  # noqa: F401
