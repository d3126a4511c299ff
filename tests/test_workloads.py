"""Host-side checks of the seeded input generators."""
import numpy as np

from paper_2212_01937_gb300 import workloads


def test_config_shapes_and_seeds():
    b = workloads.general_batch(B=8, n=5, seed=2)
    assert b.params.shape == (8, 4) and b.z.shape == (40,) and b.offsets[-1] == 40
    b2 = workloads.general_batch(B=8, n=5, seed=2)
    assert np.array_equal(b.params, b2.params) and np.array_equal(b.z, b2.z)
    assert np.all((b.params[:, 1] >= 0.05) & (b.params[:, 1] <= 0.6))
    assert np.all((b.params[:, 3] >= 1e-5) & (b.params[:, 3] <= 1e-4))
    r = workloads.ragged_batch(B=50, seed=3, nmax_exp=3.0)
    assert r.offsets[0] == 0 and r.offsets[-1] == r.nnz and np.all(np.diff(r.offsets) >= 1)
    assert r.m_obs.shape == r.z.shape
    c1 = workloads.flat_radiationless(n=100)
    assert c1.params.tolist() == [[70.0, 0.3, 0.7, 0.0]]


def test_stress_config_near_boundaries():
    s = workloads.precision_stress(B=4, n=3, seed=4)
    assert s.params.shape == (4, 5)
    assert np.all(np.abs(s.params[0::2, 4]) <= 1e-6 + 1e-15)
    for Om, OL, Or, Ok in s.params[1::2, 1:5]:
        assert workloads.has_big_bang(Om, OL, Or, Ok)
        assert not workloads.has_big_bang(Om, OL * (1 + 1e-5), Or, 1 - Om - OL * (1 + 1e-5) - Or)


def test_q_min_matches_grid():
    rng = np.random.default_rng(0)
    a = np.linspace(1e-6, 1.0, 200001)
    for _ in range(50):
        Om, OL, Or = rng.uniform(0, 1), rng.uniform(0, 3), 10 ** rng.uniform(-6, -3)
        Ok = 1 - Om - OL - Or
        grid = (Or + Om * a + Ok * a * a + OL * a ** 4).min()
        assert workloads.q_min(Om, OL, Or, Ok) <= grid + 1e-12
        assert workloads.q_min(Om, OL, Or, Ok) >= min(grid, Or) - 1e-9
