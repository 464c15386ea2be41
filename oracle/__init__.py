"""Plain, slow CPU oracle for the spherical harmonic transform (test infrastructure only).

This package is the reference the GPU path is checked against.  It is NOT
part of the product: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never imports, links or calls anything here, and nothing
here imports the CUDA library.

Everything is float64 numpy, written for readability:

* ``oracle.legendre`` -- Gauss-Legendre nodes and weights (Section 2, eq.
  thetas) and the normalized associated Legendre functions of eq.
  association, evaluated with the classical three-term recurrence in x and
  explicit exponent tracking (Section 4 notes that underflow is countered by
  tracking exponents).
* ``oracle.sht`` -- the direct O(l^3) transform of Section 2: the sums over k
  of eq. alternate_expansion at the Gauss-Legendre nodes (the Legendre
  stage), their transpose (analysis), and the sums over m at the equispaced
  phis of eq. phis as a naive DFT.
* ``oracle.gauss_jacobi`` -- the paper's own per-order matrices of Section
  4: the zeros of P-bar^m_{m+2n} (resp. P-bar^m_{m+2n+1}) found by sign
  changes and bisection on the x recurrence, the weights of Lemma
  quadratures, and the direct transforms of eqs. transform and transform2.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
identities and library routines that do not share its arithmetic.
"""

from .legendre import gl_nodes_weights, legendre_table, legendre_value  # noqa: F401
from .sht import (  # noqa: F401
    triangle_offsets,
    legendre_synthesis,
    legendre_analysis,
    legendre_adjoint,
    phi_synthesis,
    phi_analysis,
    sht_synthesis,
    sht_analysis,
    phis,
    unit_matrix,
)
from .gauss_jacobi import gj_forward, gj_inverse, gj_matrix, gj_nodes_weights, gj_sigma_n  # noqa: F401
