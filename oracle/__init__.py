"""CPU oracle for the hierarchical-inverse EMT network solve.

TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only the test suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import or run
anything in this package. The GPU library never calls it and shares no code
with it; the only thing both sides read is the seeded raw element data from
``netgen`` (which holds none of the method's arithmetic).

Everything here is plain, slow, FP64 NumPy/SciPy written from the paper:
  companion.py  trapezoidal companion models, nodal assembly, injections (Sec. II, Eq. 1-2)
  dense.py      exact solve / explicit inverse by dense factorisation (Eq. 2)
  partition.py  recursive bisection tree and cut lists (Sec. III-B, Fig. 3)
  hinv.py       hierarchical inverse, exact (Woodbury) and approximate (Eq. 3-9, Algorithm 1)
  modify.py     inverse modification: explicit recomputation, Sherman-Morrison, Algorithm 2
  emt.py        time stepping with events (Eq. 1-2 per step)
"""
