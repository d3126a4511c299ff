"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative unless stated):
  FP64 path: d_C, t, X, d_M, d_L <= 1e-12; mu <= 1e-11 mag.
  FP32 path: d_C, t, d_M, d_L <= 2e-6; X <= 1e-4 (eq. 3.9 keeps an O(rho_B^2)
  cancellation, O(100) when Omega_m0 and Omega_L0 are small); mu <= 1e-5 mag
  times the condition number |D S_k'(D) / S_k(D)| of the curvature map (large
  near the antipode of a closed universe, where d_M -> 0).
  Gradients, per pair, relative to the largest entry of the pair's row,
  against the Leibniz-rule oracle (itself pinned to central differences):
  FP64 <= 1e-9 + 1e-11/z; FP32 <= 3e-5 + 2e-6/z for d_C, d_M, d_L, mu,
  <= 1e-4 + 2e-6/z for t (its Omega_r0 entry: in eq. 3.8 with i = A the R_C
  and R_F terms' tangents carry d eps_A / d Omega_r0 ~ 1/Omega_m0 and cancel)
  and <= 1e-3 + 2e-6/z for X on these sets (X's FP32 gradient is not
  reliable for nearly empty open universes).  The 1/z terms: near z = 0
  every distance is z (1 + O(z)) and its parameter dependence sits in the
  O(z) part, while the Carlson arguments all tend to one value.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_01937_gb300 import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
COLS = {"d_C": 0, "t": 1, "X": 2, "d_M": 3, "d_L": 4, "mu": 5}
TOL64 = {"d_C": 1e-12, "t": 1e-12, "X": 1e-12, "d_M": 1e-12, "d_L": 1e-12}
TOL32 = {"d_C": 2e-6, "t": 2e-6, "X": 1e-4, "d_M": 2e-6, "d_L": 2e-6}


def _t(a, dtype=None):
    return torch.tensor(np.asarray(a), device=DEV, dtype=dtype)


def _batch_small():
    """Several tiles per row and a ragged tail: 24 rows of varying length."""
    b = workloads.general_batch(B=24, n=1, seed=11)
    rng = np.random.default_rng(11)
    lens = rng.integers(1, 300, b.B)
    lens[3] = 0
    lens[7] = 1
    offs = np.zeros(b.B + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    z = rng.uniform(0.0, 10.0, offs[-1])
    z[::97] = 0.0
    z[5::53] = rng.uniform(1e-4, 1e-2, z[5::53].size)
    z[9::61] = 1100.0
    return b.params, z, offs


def jac_tol(prec, z, name="d_C"):
    z = np.maximum(np.asarray(z, dtype=np.float64), 1e-12)
    if prec == "fp64":
        return 1e-9 + 1e-11 / z
    return {"t": 1e-4, "X": 1e-3}.get(name, 3e-5) + 2e-6 / z


def mu_cond(ref, params, offsets):
    """Condition number of mu through the curvature map, |D S_k'(D) / S_k(D)|
    with D = d_C and S_k(D) = d_M from the oracle and
    |S_k'(D)| = sqrt(|1 + Ok (d_M / D_H)^2|) (cosh or cos of sqrt|Ok| D / D_H)."""
    params = np.asarray(params, dtype=np.float64)
    rows = np.repeat(np.arange(params.shape[0]), np.diff(np.asarray(offsets)))
    H0 = params[rows, 0]
    Ok = params[rows, 4] if params.shape[1] >= 5 else 1.0 - params[rows, 1:4].sum(axis=1)
    dc, dm = ref[:, 0], ref[:, 3]
    sd = np.sqrt(np.abs(1.0 + Ok * (dm * H0 / 299792.458) ** 2))
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.abs(dc * sd / dm)
    return np.where(np.isfinite(c), np.maximum(c, 1.0), 1.0)


def _check(res, ref, tol, prec, cosmo, names=("d_C", "t", "X", "d_M", "d_L"), mu_lim=None):
    for n in names:
        if n not in res:
            continue
        got = res[n].double().cpu().numpy()
        want = ref[:, COLS[n]]
        nz = want != 0
        assert np.all(got[~nz] == 0), n
        err = np.abs(got[nz] / want[nz] - 1)
        assert err.max() <= tol[n], (prec, n, err.max(), np.argmax(err))
    if "mu" in res:
        got = res["mu"].double().cpu().numpy()
        want = ref[:, 5]
        fin = np.isfinite(want)
        # z = 0 gives -inf; d_M <= 0 (closed universes beyond the antipode) gives NaN
        assert np.all((got[~fin] == want[~fin]) | (np.isnan(got[~fin]) & np.isnan(want[~fin])))
        lim = (mu_lim if mu_lim is not None else (1e-11 if prec == "fp64" else 1e-5)) * mu_cond(ref, *cosmo)
        assert np.all(np.abs(got[fin] - want[fin]) <= lim[fin]), (prec, "mu", np.max(np.abs(got[fin] - want[fin])))


def test_roots_match_oracle(lib):
    P = np.vstack([workloads.general_batch(B=30, n=1, seed=4).params,
                   [[70, 0.3, 0.7, 0.0], [70, 0.3, 0.7, 1e-5], [60, 0.05, 0.2, 0.0], [70, 0.2, 0.06, 2.4e-5]]])
    r = lib.roots(_t(P))
    torch.cuda.synchronize()
    assert int(r["status"].abs().sum()) == 0
    got = r["roots"].cpu().numpy() + 1.0          # in x = 1+z, like the oracle
    rho, nroot = oracle.roots_x(P)
    J = oracle.root_param_jacobian(P, rho, nroot)
    dgot = r["droots"].cpu().numpy()
    kind = r["kind"].cpu().numpy()
    for b in range(P.shape[0]):
        m = nroot[b]
        slots = [0, 1, 2, 3] if m == 4 else [0, 2, 3]
        assert kind[b] in ((0, 1) if m == 4 else (2, 3))
        for s in slots:
            j = np.argmin(np.abs(rho[b, :m] - got[b, s]))
            assert abs(rho[b, j] - got[b, s]) <= 1e-13 * max(1.0, abs(rho[b, j])), (b, s)
            for k in range(3):
                if m == 3 and k == 2:
                    assert np.isnan(dgot[b, s, k].real)
                    continue
                want = J[b, j, k]
                assert abs(dgot[b, s, k] - want) <= 1e-8 * max(abs(want), 1.0), (b, s, k)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_forward_csr_vs_quadrature(lib, prec):
    params, z, offs = _batch_small()
    zin = z if prec == "fp64" else z.astype(np.float32)
    ref = oracle.quad_distances(params, zin.astype(np.float64), offs)
    res = lib.distances(_t(params), _t(zin), _t(offs), outputs=("d_C", "t", "X", "d_M", "d_L", "mu"),
                        precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    _check(res, ref, TOL64 if prec == "fp64" else TOL32, prec, (params, offs))


def test_config1_flat_radiationless(lib):
    b = workloads.flat_radiationless()
    ref = oracle.quad_distances(b.params, b.z, b.offsets)
    res = lib.distances(_t(b.params), _t(b.z), _t(b.offsets), outputs=("d_C", "mu"), precision="fp64")
    torch.cuda.synchronize()
    _check(res, ref, TOL64, "fp64", (b.params, b.offsets))


def test_layouts_agree(lib):
    b = workloads.general_batch(B=9, n=70, seed=8)
    p = _t(b.params)
    z = _t(b.z.astype(np.float32))
    dense = lib.distances(p, z, None, layout="dense", outputs=("d_C", "mu"))
    csr = lib.distances(p, z, _t(b.offsets), layout="csr", outputs=("d_C", "mu"))
    zs = z[:70]
    shared = lib.distances(p, zs, None, layout="shared", outputs=("d_C", "mu"))
    rep = lib.distances(p, zs.repeat(9), None, layout="dense", outputs=("d_C", "mu"))
    torch.cuda.synchronize()
    assert torch.equal(dense["d_C"], csr["d_C"]) and torch.equal(dense["mu"], csr["mu"])
    assert torch.equal(shared["d_C"], rep["d_C"])


def test_stress_near_flat_and_near_boundary(lib):
    s = workloads.precision_stress(B=8, n=40, seed=4)
    ref = oracle.quad_distances(s.params, s.z, s.offsets)
    r64 = lib.distances(_t(s.params), _t(s.z), _t(s.offsets), outputs=("d_C", "t", "X", "mu"), precision="fp64")
    z32 = s.z.astype(np.float32)
    ref32 = oracle.quad_distances(s.params, z32.astype(np.float64), s.offsets)
    r32 = lib.distances(_t(s.params), _t(z32), _t(s.offsets), outputs=("d_C", "t", "X", "mu"), precision="fp32")
    torch.cuda.synchronize()
    assert int(r64["status"].abs().sum()) == 0
    cosmo = (s.params, s.offsets)
    _check(r64, ref, TOL64, "fp64", cosmo, names=("d_C", "t", "X"))
    _check(r32, ref32, TOL32, "fp32", cosmo, names=("d_C", "t", "X"))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_jacobian_vs_leibniz_oracle(lib, prec):
    b = workloads.general_batch(B=6, n=33, seed=9)
    z = b.z.copy()
    z[:66:11] = [1e-4, 1e-3, 1e-2, 0.1, 30.0, 1100.0]
    zin = z if prec == "fp64" else z.astype(np.float32)
    zq = zin.astype(np.float64)
    _, J = oracle.quad_distances(b.params, zq, b.offsets, grad=True)
    res = lib.distances_jac(_t(b.params), _t(zin), _t(b.offsets), outputs=("d_C", "t", "X", "mu"), precision=prec)
    torch.cuda.synchronize()
    for n in ("d_C", "t", "X", "mu"):
        tol = jac_tol(prec, zq, n)
        got = res["jac"][n].double().cpu().numpy()
        want = J[:, COLS[n], :]
        scale = np.abs(want).max(axis=1)
        err = np.abs(got - want).max(axis=1) / scale
        bad = err > tol
        assert not bad.any(), (prec, n, err[bad], zq[bad])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vjp_matches_jacobian_and_oracle(lib, prec):
    b = workloads.general_batch(B=7, n=45, seed=10)
    dt = np.float64 if prec == "fp64" else np.float32
    rng = np.random.default_rng(1)
    cot = {n: rng.normal(size=b.nnz).astype(dt) for n in ("d_C", "t", "X", "mu")}
    zin = b.z.astype(dt)
    zq = zin.astype(np.float64)
    _, J = oracle.quad_distances(b.params, zq, b.offsets, grad=True)
    want = np.zeros((b.B, 4))
    bound = np.zeros((b.B, 4))
    for r in range(b.B):
        sl = slice(b.offsets[r], b.offsets[r + 1])
        for n, c in cot.items():
            tol = jac_tol(prec, zq, n)
            cj = c[sl].astype(np.float64)[:, None] * J[sl, COLS[n], :]
            want[r] += cj.sum(axis=0)
            bound[r] += (np.abs(c[sl]) * tol[sl] * np.abs(J[sl, COLS[n], :]).max(axis=1)).sum()
    res = lib.distances_vjp(_t(b.params), _t(zin), {n: _t(v) for n, v in cot.items()}, _t(b.offsets),
                            precision=prec)
    torch.cuda.synchronize()
    got = res["grad"].cpu().numpy()
    assert np.all(np.abs(got - want) <= bound + 1e-12 * np.abs(want)), (prec, np.abs(got - want) / bound)


def test_fp64_gradients_vs_central_differences(lib):
    """FP64 gradients against fourth-order central differences of the FP64
    forward pass on the GPU itself (<= 1e-6 relative), low and high z included.
    Steps per row: h = 2e-4 |theta|, and 1e-2 Omega_r0 in the Omega_r0
    direction, where the outputs vary on the scale of Omega_r0 itself
    (truncation about 4 (h/theta)^4 relative) and a smaller step leaves only
    rounding noise at low z.  The bound adds that noise, 1.5 x 8 ulp(f) / h
    (the coefficients' absolute sum is 18/12)."""
    b = workloads.general_batch(B=3, n=8, seed=12)
    z = b.z.copy()
    z[:4] = [1e-3, 0.05, 200.0, 1100.0]
    outs = ("d_C", "t", "X", "mu")
    res = lib.distances_jac(_t(b.params), _t(z), _t(b.offsets), outputs=outs, precision="fp64")
    torch.cuda.synchronize()

    def fwd(p):
        r = lib.distances(_t(p), _t(z), _t(b.offsets), outputs=outs, precision="fp64")
        torch.cuda.synchronize()
        return {n: r[n].cpu().numpy() for n in outs}

    rows = np.repeat(np.arange(b.B), np.diff(b.offsets))
    for k in range(4):
        hr = (1e-2 if k == 3 else 2e-4) * np.abs(b.params[:, k])
        h = hr[rows]
        f = {}
        for m in (-2, -1, 1, 2):
            pp = b.params.copy()
            pp[:, k] += m * hr
            f[m] = fwd(pp)
        for n in outs:
            fd = (-f[2][n] + 8 * f[1][n] - 8 * f[-1][n] + f[-2][n]) / (12 * h)
            got = res["jac"][n][:, k].cpu().numpy()
            scale = np.abs(res["jac"][n].cpu().numpy()).max(axis=1)
            fmax = np.max([np.abs(f[m][n]) for m in f], axis=0)
            noise = 1.5 * 8 * np.spacing(fmax) / h
            assert np.all(np.abs(got - fd) <= 1e-6 * scale + noise), (k, n, np.max(np.abs(got - fd) / scale))


def test_gauss_loglike_vs_oracle(lib):
    b = workloads.ragged_batch(B=20, seed=3, nmax_exp=2.5)
    for prec in ("fp64", "fp32"):
        dt = np.float64 if prec == "fp64" else np.float32
        zin, m = b.z.astype(dt), b.m_obs.astype(dt)
        ref, J = oracle.quad_distances(b.params, zin.astype(np.float64), b.offsets, grad=True)
        r = (m.astype(np.float64) - ref[:, 5] - b.M) / b.sigma
        ll = -0.5 * r ** 2 - np.log(b.sigma * np.sqrt(2 * np.pi))
        want = np.add.reduceat(ll, b.offsets[:-1]) if b.nnz else ll
        wg = (r / b.sigma)[:, None] * J[:, 5, :]
        wantg = np.add.reduceat(wg, b.offsets[:-1], axis=0)
        res = lib.gauss_loglike(_t(b.params), _t(zin), _t(m), _t(b.offsets), M=b.M, sigma=b.sigma, precision=prec)
        torch.cuda.synchronize()
        got, gg = res["loglike"].cpu().numpy(), res["grad"].cpu().numpy()
        if prec == "fp64":
            assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1)) <= 1e-10
        else:
            # mu is an FP32 number near 40 mag (ulp ~4e-6): allow |dl| <= sum |r|/sigma * 2e-5
            bound = np.add.reduceat(np.abs(r) / b.sigma, b.offsets[:-1]) * 2e-5 + 1e-6 * np.abs(want)
            assert np.all(np.abs(got - want) <= bound), prec
        sc = np.abs(wantg).max(axis=1, keepdims=True) + 1e-12
        assert np.max(np.abs(gg - wantg) / sc) <= (1e-8 if prec == "fp64" else 1e-4), prec


def test_status_codes_and_nan_outputs(lib):
    P = np.array([[70, 0.3, 0.7, 1e-5], [-70, 0.3, 0.7, 1e-5], [70, np.nan, 0.7, 1e-5], [70, 0.1, 2.5, 1e-5],
                  [70, 0.3, 0.7, -1e-5], [70, 0.0, 0.7, 0.0]])
    z = np.tile([0.5, 1.0], P.shape[0])
    res = lib.distances(_t(P), _t(z), None, layout="dense", outputs=("d_C", "mu"), precision="fp64")
    torch.cuda.synchronize()
    st = res["status"].cpu().numpy()
    assert st.tolist() == [0, 2, 2, 1, 2, 2]
    d = res["d_C"].cpu().numpy().reshape(-1, 2)
    assert np.all(np.isfinite(d[0])) and np.all(np.isnan(d[1:]))


def test_full_size_sampled_bench_configuration(lib):
    """general_batch at full size (4096 x 1024) in the benchmark's launch shape, a
    random sample checked pair by pair against the Carlson oracle."""
    b = workloads.general_batch()
    z32 = b.z.astype(np.float32)
    res = lib.distances(_t(b.params), _t(z32), _t(b.offsets), outputs=("d_C", "t", "X", "mu"), precision="fp32")
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(b.nnz, 3000, replace=False))
    rows = np.searchsorted(b.offsets, idx, side="right") - 1
    ref = oracle.quad_distances(b.params[rows], z32[idx].astype(np.float64), np.arange(idx.size + 1))
    sub = {n: res[n][torch.tensor(idx, device=DEV)] for n in ("d_C", "t", "X", "mu")}
    cosmo = (b.params[rows], np.arange(idx.size + 1))
    _check(sub, ref, TOL32, "fp32", cosmo, names=("d_C", "t", "X"))
    _check({"mu": sub["mu"]}, ref, TOL32, "fp32", cosmo, names=())


def test_full_size_sampled_gradients(lib):
    """Per-pair Jacobians of the benchmark batch at full size (4096 x 1024,
    one launch), 3000 random pairs against the Leibniz-rule oracle, for the
    outputs the benchmark step differentiates (d_C, t, mu): no pair above
    the bounds of jac_tol (3e-5 + 2e-6/z of the row's largest entry; t
    1e-4 + 2e-6/z).  X is computed by that step but
    not differentiated: its FP32 gradient is not within this bound for nearly
    empty open universes (eq. 3.9 with i = B cancels like rho_B^2)."""
    b = workloads.general_batch()
    z32 = b.z.astype(np.float32)
    res = lib.distances_jac(_t(b.params), _t(z32), _t(b.offsets), outputs=("d_C", "t", "X", "mu"), precision="fp32")
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(b.nnz, 3000, replace=False))
    rows = np.searchsorted(b.offsets, idx, side="right") - 1
    zq = z32[idx].astype(np.float64)
    _, J = oracle.quad_distances(b.params[rows], zq, np.arange(idx.size + 1), grad=True)
    it = torch.tensor(idx, device=DEV)
    for n in ("d_C", "t", "mu"):
        got = res["jac"][n][it].double().cpu().numpy()
        want = J[:, COLS[n], :]
        err = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
        bad = err > jac_tol("fp32", zq, n)
        assert not bad.any(), (n, int(bad.sum()), err.max())


def test_autotune_and_launch_count(lib):
    b = workloads.general_batch(B=64, n=256, seed=3)
    n0 = lib.launch_count()
    t = lib.autotune(_t(b.params), _t(b.z.astype(np.float32)), _t(b.offsets), outputs=("d_C", "mu"))
    assert t["block"] in (64, 128, 256) and t["blocks_per_sm"] >= 1 and t["ms"] > 0
    assert lib.launch_count() > n0


def test_ragged_loglike_step_in_cuda_graph(lib):
    """The per-row log-likelihood and gradient over a ragged CSR batch (row
    lengths logU(1, 10^3), empty rows included) captured in a CUDA graph:
    replays reproduce the eager call, and new parameters copied into the
    captured buffer are picked up by the replay."""
    b = workloads.ragged_batch(B=96, seed=3, nmax_exp=3.0)
    dev = torch.device(DEV)
    params = _t(b.params)
    z, m, off = _t(b.z.astype(np.float32)), _t(b.m_obs.astype(np.float32)), _t(b.offsets)
    call = lib.Call(params, z, off, precision="fp32")
    eager = lib.gauss_loglike(params, z, m, off, M=b.M, sigma=b.sigma, call=call)
    e_ll, e_g = eager["loglike"].clone(), eager["grad"].clone()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        lib.gauss_loglike(params, z, m, off, M=b.M, sigma=b.sigma, call=call)
    torch.cuda.current_stream(dev).wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        res = lib.gauss_loglike(params, z, m, off, M=b.M, sigma=b.sigma, call=call)
    n0 = lib.launch_count()
    g.replay()
    torch.cuda.synchronize()
    assert lib.launch_count() == n0
    assert torch.allclose(res["loglike"], e_ll, rtol=1e-12, atol=1e-9)
    assert torch.allclose(res["grad"], e_g, rtol=1e-10, atol=1e-9, equal_nan=True)
    # new parameters through the captured buffer
    p2 = b.params.copy()
    p2[:, 1] *= 1.05
    call.params.copy_(_t(p2))
    g.replay()
    want = lib.gauss_loglike(_t(p2), z, m, off, M=b.M, sigma=b.sigma, precision="fp32")
    torch.cuda.synchronize()
    assert torch.allclose(res["loglike"], want["loglike"], rtol=1e-12, atol=1e-9)


def _stress_sampled(lib, s, nsample, n_o1, seed=1):
    """Both precisions over the whole stress batch s in one launch each (the
    benchmark's launch shape), checked pair by pair on a random sample
    against the Carlson oracle (d_C and t; its X is eq. 3.9 as printed, which
    keeps a cancellation of about 1e-11 in FP64) and on a subset against the
    quadrature oracle (d_C, t and X; slow near the no-Big-Bang boundary, where
    it resolves the integrand's narrow peak).  Returns the worst errors."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(s.nnz, nsample, replace=False))
    rows = np.searchsorted(s.offsets, idx, side="right") - 1
    sub_off = np.arange(idx.size + 1)
    cosmo = (s.params[rows], sub_off)
    pick = np.sort(rng.choice(idx.size, n_o1, replace=False))
    worst = {}
    for prec in ("fp64", "fp32"):
        zin = s.z if prec == "fp64" else s.z.astype(np.float32)
        res = lib.distances(_t(s.params), _t(zin), _t(s.offsets), outputs=("d_C", "t", "X", "mu"), precision=prec)
        torch.cuda.synchronize()
        assert int(res["status"].abs().sum()) == 0
        it = torch.tensor(idx, device=DEV)
        sub = {n: res[n][it] for n in ("d_C", "t", "X", "mu")}
        del res
        zq = zin[idx].astype(np.float64)
        ref = oracle.carlson_distances(s.params[rows], zq, sub_off)
        tol = TOL64 if prec == "fp64" else TOL32
        _check(sub, ref, tol, prec, cosmo, names=("d_C", "t"))
        ref1 = oracle.quad_distances(s.params[rows][pick], zq[pick], np.arange(pick.size + 1))
        sub1 = {n: v[torch.tensor(pick, device=DEV)] for n, v in sub.items()}
        _check(sub1, ref1, tol, prec, (s.params[rows][pick], np.arange(pick.size + 1)), names=("d_C", "t", "X"))
        for n in ("d_C", "t"):
            worst[(prec, n)] = float(np.max(np.abs(sub[n].double().cpu().numpy() / ref[:, COLS[n]] - 1)))
        worst[(prec, "X")] = float(np.max(np.abs(sub1["X"].double().cpu().numpy() / ref1[:, 2] - 1)))
    return worst


def test_stress_sampled_vs_carlson_oracle(lib):
    """Precision stress (near-flat and within 1e-6 of the no-Big-Bang boundary,
    z from 1e-4 to 1100, explicit Omega_k0) on 64 x 2000 pairs, sampled
    against the Carlson oracle and the quadrature oracle at the north-star
    tolerances (FP64 1e-12; FP32 2e-6 in d_C and t)."""
    _stress_sampled(lib, workloads.precision_stress(B=64, n=2000, seed=4), 4000, 200)


def test_stress_full_size_sampled(lib):
    """The precision-stress configuration at full size (10^4 cosmologies x
    10^4 redshifts = 10^8 pairs, one launch per precision), 4000 sampled
    pairs against the Carlson oracle and 200 of them against the quadrature
    oracle."""
    _stress_sampled(lib, workloads.precision_stress(), 4000, 200, seed=2)


def test_lane_maps_agree_on_sorted_redshifts(lib):
    """Contiguous and interleaved lane maps give the same per-pair outputs and
    the same gradients (FP64 sums, order aside); the autotuner reports one."""
    b = workloads.general_batch(B=24, n=300, seed=14)
    z = np.sort(b.z.reshape(b.B, -1), axis=1).reshape(-1).astype(np.float32)
    g = np.random.default_rng(2).normal(size=z.size).astype(np.float32)
    p, zt, off = _t(b.params), _t(z), _t(b.offsets)
    cot = {n: _t(g) for n in ("d_C", "t", "X", "mu")}
    res = {m: lib.distances_vjp(p, zt, cot, off, outputs=("d_C", "t", "X", "mu"), precision="fp32", lane_map=m)
           for m in ("contiguous", "interleaved")}
    torch.cuda.synchronize()
    for n in ("d_C", "t", "X", "mu"):
        assert torch.equal(res["contiguous"][n], res["interleaved"][n]), n
    assert torch.allclose(res["contiguous"]["grad"], res["interleaved"]["grad"], rtol=1e-12, atol=1e-12)
    t = lib.autotune(p, zt, off, outputs=("d_C", "t", "X", "mu"), cot=cot)
    assert t["lane_map"] in ("contiguous", "interleaved")


def _cubic_three_real(a=0.5, b=0.8):
    """(Om, OL, Or = 0) with E^2 = Om (x - a)(x - b)(x + c): three real roots,
    two in (0, 1), so a Big Bang; c = ab / (a + b) removes the x^1 term and
    E^2(1) = 1 fixes Om (closure)."""
    c = a * b / (a + b)
    Om = 1.0 / ((1 - a) * (1 - b) * (1 + c))
    return [Om, Om * a * b * c, 0.0]


def _quartic_four_real(a=0.5, b=0.8, c=2.0):
    """(Om, OL, Or) with E^2 = Or (x - a)(x - b)(x + c)(x + d): four real roots,
    d from the vanishing x^1 term, Or from E^2(1) = 1 (closure)."""
    d = a * b * c / ((a + b) * c - a * b)
    lam = 1.0 / ((1 - a) * (1 - b) * (1 + c) * (1 + d))
    return [lam * ((c + d) - (a + b)), lam * a * b * c * d, lam]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_four_real_root_quartic_vs_oracle(lib, prec):
    """The quartic with four real roots (kind 1, both pair members real)."""
    P = np.array([[70.0] + _quartic_four_real(), [66.0] + _quartic_four_real(0.3, 0.7, 1.5)])
    rng = np.random.default_rng(6)
    n = 40
    z = rng.uniform(0.0, 20.0, P.shape[0] * n)
    z[::n] = [1e-3, 0.05]
    offs = np.arange(P.shape[0] + 1, dtype=np.int64) * n
    zin = z if prec == "fp64" else z.astype(np.float32)
    zq = zin.astype(np.float64)
    ref, J = oracle.quad_distances(P, zq, offs, grad=True)
    roots = lib.roots(_t(P))
    res = lib.distances_jac(_t(P), _t(zin), _t(offs), outputs=("d_C", "t", "X", "mu"), precision=prec)
    torch.cuda.synchronize()
    assert roots["kind"].cpu().tolist() == [1, 1]
    assert int(res["status"].abs().sum()) == 0
    _check(res, ref, TOL64 if prec == "fp64" else TOL32, prec, (P, offs), names=("d_C", "t", "X"))
    for name in ("d_C", "t", "X", "mu"):
        got = res["jac"][name].double().cpu().numpy()
        want = J[:, COLS[name], :]
        err = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
        assert np.all(err <= jac_tol(prec, zq, name)), (prec, name, err.max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cubic_jacobian_vs_leibniz_oracle(lib, prec):
    """Radiationless cosmologies (Omega_r0 = 0: the cubic reduction, eqs.
    B.1-B.3; one real root + a pair, and three real roots): Jacobians against
    the Leibniz-rule oracle, the Omega_r0 column NaN by construction."""
    P = np.array([[70.0, 0.3, 0.7, 0.0], [65.0, 0.5, 0.2, 0.0], [72.0] + _cubic_three_real(), [68.0, 1.4, 0.3, 0.0]])
    rng = np.random.default_rng(4)
    n = 30
    z = rng.uniform(0.0, 6.0, P.shape[0] * n)
    z[::n] = [1e-3, 0.02, 0.3, 3.0]
    offs = np.arange(P.shape[0] + 1, dtype=np.int64) * n
    zin = z if prec == "fp64" else z.astype(np.float32)
    zq = zin.astype(np.float64)
    _, J = oracle.quad_distances(P, zq, offs, grad=True)
    res = lib.distances_jac(_t(P), _t(zin), _t(offs), outputs=("d_C", "t", "X", "mu"), precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    cols = [0, 1, 2]                       # H0, Om, OL (Or has no cubic direction)
    for name in ("d_C", "t", "X", "mu"):
        got = res["jac"][name].double().cpu().numpy()
        assert np.all(np.isnan(got[:, 3])), name
        want = J[:, COLS[name], :][:, cols]
        err = np.abs(got[:, cols] - want).max(axis=1) / np.abs(want).max(axis=1)
        tol = jac_tol(prec, zq, name)
        assert np.all(err <= tol), (prec, name, err.max())


def test_autograd_function_matches_vjp(lib):
    """lcdm.Distances (torch.autograd.Function): backward of a weighted sum of
    the outputs equals the fused VJP entry point, and only params get a grad."""
    b = workloads.general_batch(B=5, n=64, seed=13)
    params = _t(b.params).requires_grad_(True)
    z = _t(b.z.astype(np.float32))
    off = _t(b.offsets)
    w = {n: torch.randn(b.nnz, device=DEV, generator=torch.Generator(device=DEV).manual_seed(i))
         for i, n in enumerate(("d_C", "mu"))}
    d_C, mu = lib.distances_autograd(params, z, off, outputs=("d_C", "mu"), precision="fp32")
    loss = (w["d_C"] * d_C).sum() + (w["mu"] * mu).sum()
    loss.backward()
    ref = lib.distances_vjp(params.detach(), z, w, off, outputs=("d_C", "mu"), precision="fp32")
    torch.cuda.synchronize()
    assert torch.allclose(params.grad, ref["grad"], rtol=1e-10, atol=1e-10)
    assert z.grad is None
