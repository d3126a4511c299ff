"""Host-side pieces of bench.py that run without a GPU: the oracle timings
used for the CPU baseline and the reference arm."""
import numpy as np

import bench
from paper_2212_01937_gb300 import workloads


def test_cpu_oracle_rates():
    b = workloads.general_batch(B=64, n=64, seed=2)
    r1, n1 = bench.cpu_oracle_rate(b, budget_s=0.2)
    r, n, procs = bench.cpu_oracle_rate_all(b, budget_s=0.2, procs=2)
    assert procs == 2 and 0 < n <= b.nnz and 0 < n1 <= b.nnz
    assert np.isfinite(r) and r > 0 and np.isfinite(r1) and r1 > 0


def test_cpu_model_and_carlson_rate():
    b = workloads.general_batch(B=64, n=64, seed=2)
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
    r, n = bench.cpu_carlson_rate(b, budget_s=0.2)
    assert np.isfinite(r) and r > 0 and 0 < n <= b.nnz
