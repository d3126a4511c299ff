"""Plain FP64 CPU oracle for the Carlson-integral distance path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path and never calls it.

* O1: adaptive quadrature of the defining integrals (2.3)-(2.5) in the scale
  factor, with the curvature map and distance modulus (Sec. 2.1.1, fn22), for
  z1 = 0, general limits z1 <= z2, and z2 -> infinity (age, horizon).
* O4: Leibniz-rule gradients of the same integrals (the approach fn23 names).
* O2: eqs. (3.7)-(3.9) / (B.1)-(B.3) assembled in complex FP64 from roots,
  for any limits z1 <= z2 (Sec. 3.1), and their z2 -> infinity limits.
* Comparators of the speed study (Sec. 3.2.2, Fig. 3): eqs. (B.4)-(B.7) in
  Legendre's form, and the hypergeometric flat radiationless distance.
* O3: roots of E^2 by companion-matrix eigenvalues (Sec. 3, fn12) with Newton
  polishing, and their derivatives by App. A, eqs. (A.1)-(A.4).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, identities, library cross-checks, brute force).
"""
from .core import (carlson, quad_distances, carlson_distances, simpson,
                   set_mutation, OUT_NAMES, quad_between, quad_limits,
                   carlson_between, carlson_limits, dmu_dz,
                   dout_dz, legendre_distances, legendre_assignment, hyp2f1_flat_distance)
from .roots import (poly_coeffs_x, roots_x, root_coef_jacobian,
                    root_param_jacobian, classify_roots, permutations)

__all__ = ["carlson", "quad_distances", "carlson_distances", "simpson",
           "quad_between", "quad_limits", "carlson_between", "carlson_limits", "dmu_dz",
           "dout_dz", "legendre_distances", "legendre_assignment", "hyp2f1_flat_distance",
           "set_mutation", "OUT_NAMES", "poly_coeffs_x", "roots_x",
           "root_coef_jacobian", "root_param_jacobian", "classify_roots",
           "permutations"]
