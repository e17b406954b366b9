"""FP64 CPU oracle for the DTT-based PSTD method (Wise, Jaros, Cox & Treeby).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never imports the product package.

Modules:
  dtt         DCT/DST types I-IV as direct sums (Section 3.2, Eq. inverse_transforms)
  pstd        Table 2 / Tables A3, A6 staggered derivatives and the leapfrog (Section 4)
  modal       closed-form modal solution and discrete energy (derived from Section 4)
  reflection  weights for arbitrary reflection coefficients (Section 5)
"""
from . import dtt, modal, pstd, reflection  # noqa: F401
