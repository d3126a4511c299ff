"""Degenerate and limiting root configurations on the GPU, against the FP64
oracle (quadrature and Leibniz-rule gradients, pinned to the closed forms of
Einstein-de Sitter and flat matter + radiation in the oracle's own tests).

* A triple root at rho = 0 (Omega_L0 = Omega_k0 = 0: E^2 = x^3 (Or x + Om);
  Einstein-de Sitter when Omega_r0 = 0).  Sec. 2.2 and fn10 ask for the
  limits of the reductions at repeated arguments; the roots are set exactly
  and (3.7)-(3.9) / (B.1)-(B.3) hold with the repeated roots.  Values only:
  the root derivatives (App. A) are singular there, so such a row's
  gradient is NaN in the density directions (the H0 entry needs no root
  derivative), and the other rows of the batch are unaffected.
* Omega_L0 -> 0: a double root at rho = 0 forms (a complex pair closing on
  the real axis).
* Omega_r0 -> 0 on the quartic path (fn13): values and gradients, including
  d X / d Omega_r0, continuous down to Omega_r0 = 1e-16, and equal to the
  cubic reduction's at Omega_r0 = 0.
"""
import numpy as np
import pytest
import torch

import oracle
from test_gpu_parity import COLS, DEV, TOL32, TOL64, _t, jac_tol

pytestmark = pytest.mark.gpu

Z = np.array([1e-4, 1e-3, 0.02, 0.1, 0.5, 1.0, 3.0, 10.0, 50.0, 300.0, 1100.0])


def _rows(P, z=Z):
    n = z.size
    return np.tile(z, len(P)), np.arange(len(P) + 1, dtype=np.int64) * n


def _vals_ok(res, ref, prec, names=("d_C", "t", "X", "d_M", "d_L")):
    tol = TOL64 if prec == "fp64" else TOL32
    for n in names:
        got = res[n].double().cpu().numpy()
        err = np.abs(got / ref[:, COLS[n]] - 1)
        assert err.max() <= tol[n], (prec, n, err.max(), np.argmax(err))
    fin = np.isfinite(ref[:, 5])
    e = np.abs(res["mu"].double().cpu().numpy()[fin] - ref[fin, 5])
    assert e.max() <= (1e-11 if prec == "fp64" else 1e-5), (prec, "mu", e.max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_triple_root_values(lib, prec):
    """Einstein-de Sitter and flat matter + radiation (closure and explicit
    Omega_k0 = 0) in one batch with an ordinary cosmology: values within the
    spec tolerances, status 0; gradient rows NaN in the density
    directions for the triple-root cosmologies, finite for the ordinary one."""
    for P in (np.array([[70.0, 1.0, 0.0, 0.0], [70.0, 0.9999, 0.0, 1e-4], [65.0, 0.99995, 0.0, 5e-5],
                        [70.0, 0.3, 0.7, 5e-5]]),
              np.array([[70.0, 1.0, 0.0, 0.0, 0.0], [70.0, 0.999, 0.0, 1e-3, 0.0], [68.0, 0.3, 0.7, 5e-5, -5e-5]])):
        z, off = _rows(P)
        zin = z if prec == "fp64" else z.astype(np.float32)
        ref = oracle.quad_distances(P, zin.astype(np.float64), off)
        outs = ("d_C", "t", "X", "d_M", "d_L", "mu")
        res = lib.distances(_t(P), _t(zin), _t(off), outputs=outs, precision=prec)
        g = lib.distances_vjp(_t(P), _t(zin), {"d_C": _t(np.ones_like(zin))}, _t(off), precision=prec)
        torch.cuda.synchronize()
        assert res["status"].cpu().tolist() == [0] * len(P)
        _vals_ok(res, ref, prec)
        grad = g["grad"].cpu().numpy()
        # the H0 entry (-value / H0 per pair) needs no root derivative
        assert np.all(np.isnan(grad[:-1, 1:])) and np.all(np.isfinite(grad[:-1, 0])), grad
        assert np.all(np.isfinite(grad[-1])), grad


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vanishing_lambda(lib, prec):
    """Omega_L0 from 1e-3 down to 0 (a double root at rho = 0 forms), with and
    without radiation: values and gradients against the oracle.  At
    Omega_L0 = 0 exactly the pair's imaginary part is ~1e-112 and its
    derivative ~1e111 (their products stay finite): FP64 carries them, FP32
    cannot (underflow and overflow), and its d / d Omega_L0 there is NaN."""
    P = np.array([[70.0, 0.3, ol, orad] for orad in (1e-4, 0.0) for ol in (1e-3, 1e-6, 1e-9, 1e-12, 0.0)])
    z, off = _rows(P)
    zin = z if prec == "fp64" else z.astype(np.float32)
    zq = zin.astype(np.float64)
    ref, J = oracle.quad_distances(P, zq, off, grad=True)
    res = lib.distances_jac(_t(P), _t(zin), _t(off), outputs=("d_C", "t", "X", "d_M", "d_L", "mu"), precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    _vals_ok(res, ref, prec)
    rows = np.repeat(np.arange(len(P)), np.diff(off))
    zero = P[rows, 2] == 0
    for n in (("d_C", "t", "X", "mu") if prec == "fp64" else ("d_C", "t", "mu")):
        got = res["jac"][n].double().cpu().numpy()
        want = J[:, COLS[n], :]
        if prec == "fp32":
            # the Omega_L0 entry where Omega_L0 = 0 exactly: NaN, the others as elsewhere
            assert np.all(np.isnan(got[zero, 2]))
            got[zero, 2] = want[zero, 2]
        for k in (3, 4):                                 # radiationless rows: no Omega_r0 column
            sel = np.where(P[rows, 3] > 0, 4, 3) == k
            err = np.abs(got[sel][:, :k] - want[sel][:, :k]).max(axis=1) / np.abs(want[sel][:, :k]).max(axis=1)
            assert np.all(err <= jac_tol(prec, zq[sel], n)), (prec, n, err.max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vanishing_radiation_continuity(lib, prec):
    """Omega_r0 from 1e-4 to 1e-16 on the quartic path (fn13's limit), for an
    ordinary and a nearly empty open cosmology: values and gradients against
    the oracle, d X / d Omega_r0 included in FP64; and the values at
    Omega_r0 = 1e-16 equal the cubic reduction's (Omega_r0 = 0)."""
    ors = [1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-14, 1e-16]
    P = np.array([[70.0, om, ol, o] for om, ol in ((0.3, 0.7), (0.2, 0.5)) for o in ors])
    z, off = _rows(P)
    zin = z if prec == "fp64" else z.astype(np.float32)
    zq = zin.astype(np.float64)
    ref, J = oracle.quad_distances(P, zq, off, grad=True)
    outs = ("d_C", "t", "X", "d_M", "d_L", "mu")
    res = lib.distances_jac(_t(P), _t(zin), _t(off), outputs=outs, precision=prec)
    P0 = P.copy()
    P0[:, 3] = 0.0
    cub = lib.distances(_t(P0), _t(zin), _t(off), outputs=outs, precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0 and int(cub["status"].abs().sum()) == 0
    _vals_ok(res, ref, prec)
    for n in (("d_C", "t", "X", "mu") if prec == "fp64" else ("d_C", "t", "mu")):
        got = res["jac"][n].double().cpu().numpy()
        want = J[:, COLS[n], :]
        err = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
        assert np.all(err <= jac_tol(prec, zq, n)), (prec, n, err.max())
    last = np.repeat(np.array(ors) == 1e-16, Z.size).reshape(-1)
    last = np.tile(last[:len(ors) * Z.size], 2)
    for n in ("d_C", "t", "X"):
        a = res[n].double().cpu().numpy()[last]
        b = cub[n].double().cpu().numpy()[last]
        assert np.all(np.abs(a / b - 1) <= (1e-12 if prec == "fp64" else 4e-6)), (prec, n)
