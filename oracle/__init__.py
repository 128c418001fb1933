"""Plain FP64 CPU oracle of the Chebyshev stochastic-propagation hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg and reference arm may import this package.  The library under
paper_2510_17432_gb300/ never imports it and shares no code with it.

It computes, slowly and in FP64, exactly what the paper defines (arXiv 2510.17432):
  lattice.py    tight-binding lattices, Anderson disorder, vacancies, Gershgorin bounds
  philox.py     Philox4x32-10 (Salmon et al., SC'11), pinned to its known-answer vectors
  bessel.py     c_n(tau~) = 2(-i)^n J_n(tau~) (App. B) by Miller's recurrence; N(tau~) (Sec. II.A)
  propagate.py  Chebyshev states, moments, sequential / moment-based / state-based
                propagation (Sec. II.A, Eq. TE, Sec. III)
  spectra.py    Fourier DOS (Sec. III) and Jackson-kernel DOS
  cost.py       Tab. I operation counts, b_opt (Sec. II.B), Amdahl's law (Eq. amdahl)

Every function is pinned by tests/test_oracle_*.py against something other than
itself: published known-answer vectors, mpmath/scipy Bessel values, the paper's
R(tau~) figures, exact diagonalisation, closed-form clean-lattice moments and
invariants.
"""
from . import philox, lattice, bessel, propagate, spectra, cost  # noqa: F401
