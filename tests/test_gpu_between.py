"""Parity of the general-limits path (lcdm_distances_between, lcdm_limits,
through the C ABI) with the FP64 CPU oracle.

Tolerances as for the z1 = 0 path (test_gpu_parity.py), with the redshift
that sets the low-z terms of the gradient bound taken in the observer's frame,
z' = (z2 - z1)/(1 + z1): the path evaluates the shifted cosmology at z'.
  FP64: d_C, t, X, d_M, d_L <= 1e-12; mu <= 1e-11 mag.
  FP32: d_C, t, d_M, d_L <= 2e-6; X <= 1e-4; mu <= 1e-5 mag x condition number.
  Limits (FP64 always): chi(z1, inf), t(z1, inf) <= 1e-12; gradients <= 1e-9
  of the row's largest entry.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_01937_gb300 import workloads

from test_gpu_parity import COLS, TOL32, TOL64, _check, _t, jac_tol

pytestmark = pytest.mark.gpu

ALL = ("d_C", "t", "X", "d_M", "d_L", "mu")


def _batch_between():
    """24 rows of varying length (one empty, one of length 1), several tiles
    per row; z1 per row (a few exactly 0); z2 = z1 + dz with dz ~ U(0, 10),
    some dz = 0, some tiny, some z2 = 1100, and a few z2 < z1."""
    b = workloads.between_batch(B=24, n=1, seed=17)
    rng = np.random.default_rng(17)
    z1 = b.extra["z1"].copy()
    z1[[0, 5, 11]] = 0.0
    z1[2] = 6.0
    lens = rng.integers(1, 300, b.B)
    lens[3] = 0
    lens[7] = 1
    offs = np.zeros(b.B + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    rows = np.repeat(np.arange(b.B), lens)
    dz = rng.uniform(0.0, 10.0, offs[-1])
    dz[::97] = 0.0
    dz[5::53] = rng.uniform(1e-4, 1e-2, dz[5::53].size)
    z2 = z1[rows] + dz
    z2[9::61] = 1100.0
    bad = np.zeros(z2.size, dtype=bool)
    bad[13::89] = True
    return b.params, z1, z2, offs, rows, bad


def _zin(z2, z1, rows, bad, prec):
    """Upper limits in the path's dtype; the reversed intervals are made
    after rounding so that they stay reversed."""
    zin = z2.astype(np.float64 if prec == "fp64" else np.float32)
    zin[bad] = (z1[rows[bad]] - 0.5).astype(zin.dtype)
    zin[bad & (z1[rows] < 0.5)] = -1.0
    return zin


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_between_forward_vs_quadrature(lib, prec):
    params, z1, z2, offs, rows, bad = _batch_between()
    zin = _zin(z2, z1, rows, bad, prec)
    zq = zin.astype(np.float64)
    ref = oracle.quad_between(params, z1, zq, offs)
    res = lib.distances_between(_t(params), _t(z1), _t(zin), _t(offs), outputs=ALL, precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    # outside the domain: the planted reversed intervals, and in FP32 any z2 = z1
    # whose rounding to float32 fell below z1
    out_dom = zq < z1[rows]
    assert np.all(out_dom[bad])
    for n in ALL:
        assert torch.isnan(res[n][_t(out_dom)]).all(), n
    good = ~out_dom
    sub = {n: res[n][_t(good)] for n in ALL}
    # the mu condition number wants per-pair rows: keep the CSR of the good pairs
    offs_g = np.concatenate([[0], np.cumsum(np.bincount(rows[good], minlength=params.shape[0]))])
    _check(sub, ref[good], TOL64 if prec == "fp64" else TOL32, prec, (params, offs_g))


def test_between_dense_layout_and_z1_zero(lib):
    """Dense layout; rows with z1 = 0 agree with lcdm_distances."""
    b = workloads.between_batch(B=10, n=37, seed=19)
    z1 = b.extra["z1"].copy()
    z1[::2] = 0.0
    z2 = b.z.copy()
    rows = np.repeat(np.arange(b.B), 37)
    z2[np.isin(rows, np.arange(0, b.B, 2))] -= np.repeat(b.extra["z1"][::2], 37)
    ref = oracle.quad_between(b.params, z1, z2, b.offsets)
    res = lib.distances_between(_t(b.params), _t(z1), _t(z2), None, outputs=ALL, precision="fp64",
                                layout="dense")
    plain = lib.distances(_t(b.params), _t(z2), None, outputs=ALL, precision="fp64", layout="dense")
    torch.cuda.synchronize()
    _check(res, ref, TOL64, "fp64", (b.params, b.offsets))
    zero = _t(np.isin(rows, np.arange(0, b.B, 2)))
    for n in ("d_C", "t", "X", "d_M", "d_L"):
        a, c = res[n][zero].cpu().numpy(), plain[n][zero].cpu().numpy()
        nz = c != 0
        assert np.max(np.abs(a[nz] / c[nz] - 1)) < 1e-13, n


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_between_vjp_vs_leibniz_oracle(lib, prec):
    b = workloads.between_batch(B=7, n=45, seed=23)
    z1 = b.extra["z1"].copy()
    z1[0] = 0.0
    dt = np.float64 if prec == "fp64" else np.float32
    rng = np.random.default_rng(2)
    cot = {n: rng.normal(size=b.nnz).astype(dt) for n in ("d_C", "t", "X", "d_M", "mu")}
    zin = b.z.astype(dt)
    zq = zin.astype(np.float64)
    rows = np.repeat(np.arange(b.B), np.diff(b.offsets))
    zp = (zq - z1[rows]) / (1 + z1[rows])
    for ncol in (4, 5):
        params = b.params if ncol == 4 else np.column_stack([b.params, 1 - b.params[:, 1:4].sum(axis=1)])
        _, J = oracle.quad_between(params, z1, zq, b.offsets, grad=True)
        want = np.zeros((b.B, ncol))
        bound = np.zeros((b.B, ncol))
        for r in range(b.B):
            sl = slice(b.offsets[r], b.offsets[r + 1])
            for n, c in cot.items():
                tol = jac_tol(prec, zp, n)
                want[r] += (c[sl].astype(np.float64)[:, None] * J[sl, COLS[n], :]).sum(axis=0)
                bound[r] += (np.abs(c[sl]) * tol[sl] * np.abs(J[sl, COLS[n], :]).max(axis=1)).sum()
        res = lib.distances_between(_t(params), _t(z1), _t(zin), _t(b.offsets), outputs=(),
                                    cot={n: _t(v) for n, v in cot.items()}, precision=prec)
        torch.cuda.synchronize()
        assert int(res["status"].abs().sum()) == 0
        got = res["grad"].cpu().numpy()
        assert np.all(np.abs(got - want) <= bound + 1e-12 * np.abs(want)), (prec, ncol, np.abs(got - want) / bound)


def test_limits_vs_quadrature_and_gradients(lib):
    b = workloads.limits_batch(B=40, seed=29)
    z1 = b.extra["z1"].copy()
    z1[:4] = [0.0, 1e-3, 0.5, 1100.0]
    P = np.vstack([b.params, [[70.0, 0.3, 0.7, 0.0], [60.0, 0.05, 0.2, 0.0], [70.0, 0.3, 0.7, 5e-5]]])
    z1 = np.concatenate([z1, [0.0, 2.0, 30.0]])
    rng = np.random.default_rng(3)
    cc, ct = rng.normal(size=P.shape[0]), rng.normal(size=P.shape[0])
    for ncol in (4, 5):
        params = P if ncol == 4 else np.column_stack([P, 1 - P[:, 1:4].sum(axis=1)])
        ref, J = oracle.quad_limits(params, z1, grad=True)
        res = lib.limits(_t(params), _t(z1), cot_chi=_t(cc), cot_t=_t(ct), grad=True)
        torch.cuda.synchronize()
        assert int(res["status"].abs().sum()) == 0
        for k, n in enumerate(("chi_inf", "t_inf")):
            got = res[n].cpu().numpy()
            assert np.max(np.abs(got / ref[:, k] - 1)) < 1e-12, (ncol, n)
        want = cc[:, None] * J[:, 0, :] + ct[:, None] * J[:, 1, :]
        scale = np.abs(cc)[:, None] * np.abs(J[:, 0, :]) + np.abs(ct)[:, None] * np.abs(J[:, 1, :])
        got = res["grad"].cpu().numpy()
        rad = params[:, 3] > 0
        g, w, s = got[rad], want[rad], scale[rad].max(axis=1, keepdims=True)
        assert np.all(np.abs(g - w) <= 1e-9 * s), (ncol, np.max(np.abs(g - w) / s))
        # radiationless rows: no Omega_r0 direction (NaN there only)
        cub = ~rad
        cols = [c for c in range(ncol) if c != 3]
        assert np.all(np.isnan(got[cub][:, 3]))
        g, w = got[cub][:, cols], want[cub][:, cols]
        assert np.all(np.abs(g - w) <= 1e-9 * np.abs(w).max(axis=1, keepdims=True))


def test_limits_present_age_closed_form(lib):
    """t(0, inf) of flat radiationless cosmologies: (2/(3 H0 sqrt(OL))) asinh(sqrt(OL/Om))."""
    Om = np.array([0.1, 0.3, 0.5, 0.8])
    P = np.column_stack([np.full(4, 70.0), Om, 1 - Om, np.zeros(4)])
    res = lib.limits(_t(P), _t(np.zeros(4)))
    torch.cuda.synchronize()
    OL = 1 - Om
    age = 2 / (3 * np.sqrt(OL)) * 977.7922216807891 / 70.0 * np.arcsinh(np.sqrt(OL / Om))
    assert np.max(np.abs(res["t_inf"].cpu().numpy() / age - 1)) < 1e-12


def test_invalid_lower_limits(lib):
    P = np.tile([70.0, 0.3, 0.7, 5e-5], (3, 1))
    z1 = np.array([-0.5, np.nan, 1.0])
    res = lib.limits(_t(P), _t(z1))
    r2 = lib.distances_between(_t(P), _t(z1), _t(np.array([1.0, 2.0, 3.0], dtype=np.float32)), None,
                               outputs=("d_C",), layout="dense")
    torch.cuda.synchronize()
    assert res["status"].cpu().tolist() == [2, 2, 0]
    assert r2["status"].cpu().tolist() == [2, 2, 0]
    assert np.isnan(res["t_inf"][:2].cpu().numpy()).all() and np.isfinite(res["t_inf"][2].item())
    assert np.isnan(r2["d_C"][:2].cpu().numpy()).all() and np.isfinite(r2["d_C"][2].item())


def test_between_full_size_sampled(lib):
    """4096 rows x 1024 pairs (the general-limits bench workload), FP32 forward
    and fused adjoint in one launch configuration; 1024 sampled pairs against
    the Carlson oracle, and the gradient finite."""
    b = workloads.between_batch()
    z1 = b.extra["z1"]
    zin = b.z.astype(np.float32)
    rng = np.random.default_rng(31)
    cot = {"d_C": _t(rng.normal(size=b.nnz).astype(np.float32)), "mu": _t(rng.normal(size=b.nnz).astype(np.float32))}
    res = lib.distances_between(_t(b.params), _t(z1), _t(zin), _t(b.offsets), outputs=("d_C", "t", "X", "mu"),
                                cot=cot, precision="fp32")
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    assert torch.isfinite(res["grad"]).all()
    idx = np.sort(rng.choice(b.nnz, 1024, replace=False))
    rows = np.searchsorted(b.offsets, idx, side="right") - 1
    ref = oracle.carlson_between(b.params[rows], z1[rows], zin[idx].astype(np.float64), np.arange(idx.size + 1))
    sub = {n: res[n][_t(idx)] for n in ("d_C", "t", "X", "mu")}
    _check(sub, ref, TOL32, "fp32", (b.params[rows], np.arange(idx.size + 1)))


def test_limits_full_size_sampled(lib):
    b = workloads.limits_batch()
    res = lib.limits(_t(b.params), _t(b.extra["z1"]))
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    idx = np.random.default_rng(37).choice(b.B, 2048, replace=False)
    ref = oracle.carlson_limits(b.params[idx], b.extra["z1"][idx])
    got = np.column_stack([res["chi_inf"].cpu().numpy()[idx], res["t_inf"].cpu().numpy()[idx]])
    assert np.max(np.abs(got / ref - 1)) < 1e-12
