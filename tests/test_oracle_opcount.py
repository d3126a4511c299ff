"""Pins of the operation counter (oracle/opcount.py): it restates O2's
per-pair evaluation with counted operations, so its values must be O2's to
within the truncation of a single-precision stopping rule, its duplication
sequences must stop where Carlson's rule (r = 2^-24) says, and the count of a
duplication must grow by the same amount per iteration."""
import math

import numpy as np

import oracle
from oracle import opcount, roots
from paper_2212_01937_gb300 import workloads


def test_values_are_o2s():
    b = workloads.general_batch(B=6, n=5, seed=3)
    rho, nr = roots.roots_x(b.params)
    perm = roots.permutations(rho, nr)
    ref = oracle.carlson_distances(b.params, b.z, b.offsets)
    for i in range(b.nnz):
        row = i // 5
        H0, Om, OL, Or = b.params[row]
        opcount.pair_ops(rho[row], perm[row, 1], perm[row, 2], perm[row, 0], H0, 1 - Om - OL - Or, b.z[i],
                         grad=False)
        c, t, x = opcount.LAST_VALUES
        s = Or ** -0.5
        got = np.array([c * s * 299792.458 / H0, t * s * 977.7922216807891 / H0, x * s * 299792.458 / H0])
        assert np.all(np.abs(got / ref[i, :3] - 1) < 2e-8), (i, got / ref[i, :3] - 1)


def _rf_steps(x, y, z):
    """Duplication steps of R_F under Carlson's rule at r = 2^-24: stop once
    4^-m Q < |A_m|, Q = (3r)^(-1/6) max |A_0 - x_j| (plain complex arithmetic)."""
    x, y, z = complex(x), complex(y), complex(z)
    A = (x + y + z) / 3
    Q = (3 * 2.0 ** -24) ** (-1 / 6) * max(abs(A - x), abs(A - y), abs(A - z))
    f, m = 1.0, 0
    while f * Q >= abs(A):
        sx, sy, sz = x ** 0.5, y ** 0.5, z ** 0.5
        lam = sx * sy + sx * sz + sy * sz
        A, x, y, z = (A + lam) / 4, (x + lam) / 4, (y + lam) / 4, (z + lam) / 4
        f /= 4
        m += 1
    return m


def test_stopping_rule_and_per_iteration_count():
    rng = np.random.default_rng(0)
    seen = {}
    for _ in range(30):
        x, y, z = rng.uniform(0.01, 10.0, 3) ** 3
        opcount.reset()
        opcount.rf(opcount.C(x), opcount.C(y), opcount.C(z))
        m = opcount.LAST_RF_ITERS
        assert m == _rf_steps(x, y, z)
        seen.setdefault(m, set()).add(sum(opcount.snapshot().values()))
    # one count per number of steps, growing by the same amount per step
    assert all(len(v) == 1 for v in seen.values()), seen
    ms = sorted(seen)
    assert len(ms) >= 3
    steps = {(min(seen[b]) - min(seen[a])) // (b - a) for a, b in zip(ms, ms[1:])}
    assert len(steps) == 1, steps
    # equal arguments: no step, the series only, and R_F(x, x, x) = x^-1/2
    v = opcount.rf(opcount.C(2.0), opcount.C(2.0), opcount.C(2.0))
    assert opcount.LAST_RF_ITERS == 0 and abs(v.re.v - 2.0 ** -0.5) < 1e-15


def test_adjoint_counts_the_gradient_rules():
    """The adjoint of one pair includes the R_D evaluations that (2.10)-(2.12)
    need (three for the shared triple, two per R_C): it cannot be cheaper
    than the forward R_J evaluations it replaces."""
    b = workloads.general_batch(B=2, n=2, seed=4)
    rho, nr = roots.roots_x(b.params)
    perm = roots.permutations(rho, nr)
    H0, Om, OL, Or = b.params[0]
    f, a = opcount.pair_ops(rho[0], perm[0, 1], perm[0, 2], perm[0, 0], H0, 1 - Om - OL - Or, 2.0)
    assert a["sqrt"] > 0 and a["mul"] > f["mul"] / 2
