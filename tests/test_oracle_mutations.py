"""Each plausible mistake planted in the oracle (on the CPU) must make at
least one pin fail: dropped series term, wrong sign, transposed operands,
missing factor, missing closure term, simplified R_J sum, a forgotten lower
limit, a dropped term of the z2 -> infinity limit."""
import numpy as np
import pytest

import oracle

from test_oracle_carlson import (test_equal_arguments, test_rf_complete_and_agm,
                                 test_scipy_cross_check_real_and_conjugate_pair)
from test_oracle_distances import (test_carlson_cubic_vs_quadrature,
                                   test_carlson_vs_quadrature_random, test_milne,
                                   test_gradients_vs_finite_differences)

from test_oracle_limits import (test_carlson_between_vs_quadrature,
                                test_carlson_limits_vs_quadrature_and_differences)

PINS = [test_equal_arguments, test_rf_complete_and_agm,
        test_scipy_cross_check_real_and_conjugate_pair, test_carlson_vs_quadrature_random,
        test_carlson_cubic_vs_quadrature, test_milne, test_gradients_vs_finite_differences,
        test_carlson_between_vs_quadrature, test_carlson_limits_vs_quadrature_and_differences]


def _gradient_vs_closure_pin():
    """Omega_m gradient under closure against the explicit five-column form:
    d/dOm|closure = d/dOm - d/dOk."""
    p4 = np.array([[70.0, 0.3, 0.6, 5e-5]])
    p5 = np.column_stack([p4, 1 - p4[:, 1:4].sum(axis=1)])
    z = np.array([0.5, 2.0])
    _, J4 = oracle.quad_distances(p4, z, grad=True)
    _, J5 = oracle.quad_distances(p5, z, grad=True)
    assert np.allclose(J4[:, :, 1], J5[:, :, 1] - J5[:, :, 4], rtol=1e-12)


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5, 6, 7, 8])
def test_planted_mistake_is_caught(mutation):
    failures = 0
    oracle.set_mutation(mutation)
    try:
        for pin in PINS + [_gradient_vs_closure_pin]:
            try:
                pin()
            except AssertionError:
                failures += 1
    finally:
        oracle.set_mutation(0)
    assert failures >= 1


def test_unmutated_oracle_passes_battery():
    for pin in PINS + [_gradient_vs_closure_pin]:
        pin()
