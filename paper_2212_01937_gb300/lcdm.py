"""Thin Python binding of liblcdm (include/lcdm.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of liblcdm.so.  PyTorch provides device memory and the stream.  There
is no fallback: if the library is missing, :func:`load` raises.

Layouts (see include/lcdm.h): ``"csr"`` (offsets [B+1] int64, z [nnz]),
``"dense"`` (z [B*n], n per row) and ``"shared"`` (z [n] shared by all rows).
Precision ``"fp32"`` (LCDM_FP32_MIXED: float32 I/O and per-pair arithmetic,
FP64 root preparation and reductions) or ``"fp64"``.
"""
import ctypes
import os

import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "liblcdm.so")
OUTS = ("d_C", "t", "X", "d_M", "d_L", "mu")
PRECISION = {"fp64": 0, "fp32": 1}
LAYOUT = {"csr": 0, "dense": 1, "shared": 2}

_lib = None


class Opts(ctypes.Structure):
    _fields_ = [("ncol", ctypes.c_int32), ("precision", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("lane_map", ctypes.c_int32),
                ("deterministic", ctypes.c_int32)]


LANE_MAP = {"tuned": 0, "contiguous": 1, "interleaved": 2}


_vp = ctypes.c_void_p
_VP6 = ctypes.c_void_p * 6


def load():
    """Load liblcdm.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblcdm.so not found at %s; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    i64, i32, sz, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t, ctypes.c_double
    op = ctypes.POINTER(Opts)
    lib.lcdm_workspace_size.argtypes = [i64, op, ctypes.POINTER(sz)]
    lib.lcdm_roots.argtypes = [_vp, i64, op, _vp, _vp, _vp, _vp, _vp, sz, _vp]
    lib.lcdm_distances.argtypes = [_vp, i64, _vp, _vp, i64, _VP6, _vp, op, _vp, sz, _vp]
    lib.lcdm_distances_jac.argtypes = [_vp, i64, _vp, _vp, i64, _VP6, _VP6, _vp, op, _vp, sz, _vp]
    lib.lcdm_distances_vjp.argtypes = [_vp, i64, _vp, _vp, i64, _VP6, _VP6, _vp, _vp, op, _vp, sz, _vp]
    lib.lcdm_gauss_loglike.argtypes = [_vp, i64, _vp, _vp, _vp, i64, dbl, dbl, _vp, _vp, _vp, _vp, op, _vp,
                                       sz, _vp]
    lib.lcdm_host_workspace_size.argtypes = [i64, i64, op, ctypes.POINTER(sz)]
    lib.lcdm_distances_vjp_host.argtypes = [_vp, i64, _vp, _vp, i64, _VP6, _VP6, _vp, _vp, op, _vp, sz, i32, _vp]
    lib.lcdm_autotune.argtypes = [_vp, i64, _vp, _vp, i64, _VP6, _VP6, _vp, _vp, op, _vp, sz, _vp,
                                  ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(i32)]
    lib.lcdm_between_workspace_size.argtypes = [i64, i64, op, ctypes.POINTER(sz)]
    lib.lcdm_distances_between.argtypes = [_vp, i64, _vp, _vp, _vp, i64, _VP6, _VP6, _vp, _vp, op, _vp, sz, _vp]
    lib.lcdm_limits.argtypes = [_vp, i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, op, _vp, sz, _vp]
    lib.lcdm_loglike_dz_workspace_size.argtypes = [i64, i64, op, ctypes.POINTER(sz)]
    lib.lcdm_gauss_loglike_dz.argtypes = [_vp, i64, _vp, _vp, _vp, i64, dbl, dbl, _vp, _vp, _vp, _vp, _vp, op,
                                          _vp, sz, _vp]
    lib.lcdm_distances_vjp_dz.argtypes = [_vp, i64, _vp, _vp, i64, _VP6, _VP6, _vp, _vp, _vp, op, _vp, sz, _vp]
    lib.lcdm_probe.argtypes = [i32, _vp, i32, i32, i32, _vp]
    lib.lcdm_probe.restype = ctypes.c_int
    lib.lcdm_probe_ops_per_thread.argtypes = [i32]
    lib.lcdm_probe_ops_per_thread.restype = i64
    lib.lcdm_status_string.argtypes = [ctypes.c_int]
    lib.lcdm_status_string.restype = ctypes.c_char_p
    lib.lcdm_launch_count.restype = i64
    for f in ("lcdm_workspace_size", "lcdm_roots", "lcdm_distances", "lcdm_distances_jac",
              "lcdm_distances_vjp", "lcdm_gauss_loglike", "lcdm_autotune", "lcdm_host_workspace_size",
              "lcdm_distances_vjp_host", "lcdm_between_workspace_size", "lcdm_distances_between",
              "lcdm_limits", "lcdm_loglike_dz_workspace_size", "lcdm_gauss_loglike_dz",
              "lcdm_distances_vjp_dz"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st):
    if st != 0:
        raise RuntimeError("liblcdm: " + load().lcdm_status_string(st).decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def launch_count():
    return int(load().lcdm_launch_count())


def probe_rate(what, device, iters=2048, reps=5):
    """Measured issue rate of one pipe (lcdm_probe): what = "ffma" (FP32
    fused multiply-adds/s), "mufu" (FP32 reciprocal square roots/s) or
    "dfma" (FP64 fused multiply-adds/s), over 8 resident 256-thread blocks
    per SM, best of ``reps`` timed launches after one warm-up."""
    kind = {"ffma": 0, "mufu": 1, "dfma": 2}[what]
    it = iters if kind != 2 else max(1, iters // 32)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, threads = 8 * sms, 256
    out = torch.empty(blocks * threads, dtype=torch.float64 if kind == 2 else torch.float32, device=device)
    lib = load()
    best = None
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(lib.lcdm_probe(kind, _ptr(out), blocks, threads, it, _stream(device)))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if r > 0 and (best is None or ms < best):
            best = ms
    return blocks * threads * lib.lcdm_probe_ops_per_thread(it) / (best / 1e3)


class Call:
    """Prepared arguments of one batch (validated and placed on the device)."""

    def __init__(self, params, z, offsets=None, layout=None, precision="fp32", block=0, blocks_per_sm=0,
                 workspace=None, lane_map="tuned", deterministic=False):
        lib = load()
        if not params.is_cuda:
            raise ValueError("params must be a CUDA tensor")
        self.device = params.device
        self.params = params.to(torch.float64).contiguous()
        self.B, ncol = self.params.shape
        if layout is None:
            layout = "csr" if offsets is not None else "dense"
        self.layout = layout
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.z = z.to(device=self.device, dtype=self.dtype).contiguous().reshape(-1)
        self.offsets = None
        if layout == "csr":
            if offsets is None:
                raise ValueError("csr layout needs offsets")
            self.offsets = offsets.to(device=self.device, dtype=torch.int64).contiguous()
            self.n = self.z.numel()
            self.npairs = self.n
        elif layout == "dense":
            if self.z.numel() % self.B:
                raise ValueError("dense layout needs len(z) divisible by B")
            self.n = self.z.numel() // self.B
            self.npairs = self.z.numel()
        else:
            self.n = self.z.numel()
            self.npairs = self.B * self.n
        self.opts = Opts(ncol, PRECISION[precision], LAYOUT[layout], block, blocks_per_sm, LANE_MAP[lane_map],
                         1 if deterministic else 0)
        nbytes = ctypes.c_size_t()
        _check(lib.lcdm_workspace_size(self.B, ctypes.byref(self.opts), ctypes.byref(nbytes)))
        if workspace is not None and workspace.numel() >= nbytes.value:
            self.ws = workspace
        else:
            self.ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self.ws_bytes = self.ws.numel()
        self.status = torch.empty(self.B, dtype=torch.int32, device=self.device)

    @property
    def ncol(self):
        return self.opts.ncol

    def out_buffers(self, outputs):
        out = {}
        for name in outputs:
            if name not in OUTS:
                raise ValueError("unknown output %r" % name)
            out[name] = torch.empty(self.npairs, dtype=self.dtype, device=self.device)
        return out, _VP6(*[(out[n].data_ptr() if n in out else None) for n in OUTS])

    def common(self):
        return (_ptr(self.params), self.B, _ptr(self.offsets), _ptr(self.z), self.n)

    def tail(self):
        return (ctypes.byref(self.opts), _ptr(self.ws), self.ws_bytes, _stream(self.device))


def roots(params, call=None):
    """Roots of E^2 in z with their derivatives (lcdm_roots).  A prepared
    ``call`` (dense layout, FP64, same params) skips the argument set-up."""
    c = call if call is not None else Call(params, torch.zeros(params.shape[0], device=params.device),
                                           layout="dense", precision="fp64")
    r = torch.empty(c.B, 4, 2, dtype=torch.float64, device=c.device)
    dr = torch.empty(c.B, 4, 2, c.ncol - 1, dtype=torch.float64, device=c.device)
    kind = torch.empty(c.B, dtype=torch.int32, device=c.device)
    _check(load().lcdm_roots(_ptr(c.params), c.B, ctypes.byref(c.opts), _ptr(r), _ptr(dr), _ptr(kind),
                             _ptr(c.status), _ptr(c.ws), c.ws_bytes, _stream(c.device)))
    return {"roots": torch.complex(r[..., 0], r[..., 1]), "droots": torch.complex(dr[..., 0, :], dr[..., 1, :]),
            "kind": kind, "status": c.status}


def distances(params, z, offsets=None, outputs=("d_C", "t", "X", "mu"), **kw):
    """Forward distances (lcdm_distances).  Returns {name: tensor, "status": ...}."""
    c = Call(params, z, offsets, **kw)
    out, vp = c.out_buffers(outputs)
    _check(load().lcdm_distances(*c.common(), vp, _ptr(c.status), *c.tail()))
    out["status"] = c.status
    return out


def distances_jac(params, z, offsets=None, outputs=("d_C", "t", "X", "mu"), jac_outputs=None, **kw):
    """Forward distances and per-pair Jacobians [npairs, ncol] (lcdm_distances_jac)."""
    c = Call(params, z, offsets, **kw)
    out, vp = c.out_buffers(outputs)
    jac_outputs = outputs if jac_outputs is None else jac_outputs
    jac = {n: torch.empty(c.npairs, c.ncol, dtype=c.dtype, device=c.device) for n in jac_outputs}
    jp = _VP6(*[(jac[n].data_ptr() if n in jac else None) for n in OUTS])
    _check(load().lcdm_distances_jac(*c.common(), vp, jp, _ptr(c.status), *c.tail()))
    out["jac"] = jac
    out["status"] = c.status
    return out


def distances_vjp(params, z, cot, offsets=None, outputs=(), call=None, grad_z=False, workspace=None, **kw):
    """Fused forward + adjoint (lcdm_distances_vjp): grad [B, ncol] of
    sum_o <cot[o], out_o>.  cot: {name: tensor [npairs]}.  A prepared
    ``call`` (same params, z, offsets) skips the argument set-up.  With
    grad_z, also "grad_z" [npairs] = sum_o cot_o d out_o / dz per pair
    (lcdm_distances_vjp_dz; ``workspace`` as for gauss_loglike)."""
    c = call if call is not None else Call(params, z, offsets, **kw)
    out, vp = c.out_buffers(outputs)
    cots = {n: v.to(device=c.device, dtype=c.dtype).contiguous() for n, v in cot.items() if v is not None}
    cp = _VP6(*[(cots[n].data_ptr() if n in cots else None) for n in OUTS])
    grad = torch.empty(c.B, c.ncol, dtype=torch.float64, device=c.device)
    if grad_z:
        gz = torch.empty(c.npairs, dtype=c.dtype, device=c.device)
        ws = workspace if workspace is not None else loglike_dz_workspace(c)
        _check(load().lcdm_distances_vjp_dz(*c.common(), cp, vp, _ptr(grad), _ptr(gz), _ptr(c.status),
                                            ctypes.byref(c.opts), _ptr(ws), ws.numel(), _stream(c.device)))
        out["grad_z"] = gz
    else:
        _check(load().lcdm_distances_vjp(*c.common(), cp, vp, _ptr(grad), _ptr(c.status), *c.tail()))
    out["grad"] = grad
    out["status"] = c.status
    return out


def _between_ws(c, n):
    nbytes = ctypes.c_size_t()
    _check(load().lcdm_between_workspace_size(c.B, n, ctypes.byref(c.opts), ctypes.byref(nbytes)))
    return torch.empty(max(nbytes.value, 1), dtype=torch.uint8, device=c.device)


def distances_between(params, z1, z2, offsets=None, outputs=("d_C", "t", "X", "mu"), cot=None, **kw):
    """Eqs. (2.3)-(2.5) from z1[b] (per row) to each pair's z2
    (lcdm_distances_between); with ``cot`` ({name: [npairs]}) also the fused
    adjoint, returned as "grad" [B, ncol].  d_L and mu are those of a source
    at z2 seen by a comoving observer at z1.  Layouts "csr" and "dense"."""
    c = Call(params, z2, offsets, **kw)
    if c.layout == "shared":
        raise ValueError("general limits need the csr or dense layout")
    z1d = torch.as_tensor(z1, dtype=torch.float64).to(c.device).reshape(-1).contiguous()
    if z1d.numel() != c.B:
        raise ValueError("z1 must hold one lower limit per row")
    ws = _between_ws(c, c.n)
    out, vp = c.out_buffers(outputs)
    cp, grad = _VP6(), None
    if cot is not None:
        cots = {n: v.to(device=c.device, dtype=c.dtype).contiguous() for n, v in cot.items() if v is not None}
        cp = _VP6(*[(cots[n].data_ptr() if n in cots else None) for n in OUTS])
        grad = torch.empty(c.B, c.ncol, dtype=torch.float64, device=c.device)
    _check(load().lcdm_distances_between(_ptr(c.params), c.B, _ptr(z1d), _ptr(c.offsets), _ptr(c.z), c.n, cp,
                                         vp, _ptr(grad), _ptr(c.status), ctypes.byref(c.opts), _ptr(ws),
                                         ws.numel(), _stream(c.device)))
    if grad is not None:
        out["grad"] = grad
    out["status"] = c.status
    return out


def limits(params, z1, cot_chi=None, cot_t=None, grad=False, **kw):
    """The upper limit at infinity per row (lcdm_limits): "chi_inf" [B] (Mpc,
    comoving distance to the particle horizon from z1) and "t_inf" [B] (Gyr,
    the age at z1), FP64; with grad, "grad" [B, ncol] of
    sum_b cot_chi[b] chi_inf[b] + cot_t[b] t_inf[b]."""
    kw.setdefault("precision", "fp64")
    c = Call(params, torch.zeros(params.shape[0], device=params.device), layout="dense", **kw)
    z1d = torch.as_tensor(z1, dtype=torch.float64).to(c.device).reshape(-1).contiguous()
    if z1d.numel() != c.B:
        raise ValueError("z1 must hold one lower limit per row")
    ws = _between_ws(c, 0)
    f64 = dict(dtype=torch.float64, device=c.device)
    chi = torch.empty(c.B, **f64)
    age = torch.empty(c.B, **f64)
    g = torch.empty(c.B, c.ncol, **f64) if grad else None
    cc = None if cot_chi is None else torch.as_tensor(cot_chi, **f64).reshape(-1).contiguous()
    ct = None if cot_t is None else torch.as_tensor(cot_t, **f64).reshape(-1).contiguous()
    _check(load().lcdm_limits(_ptr(c.params), c.B, _ptr(z1d), _ptr(chi), _ptr(age), _ptr(cc), _ptr(ct), _ptr(g),
                              _ptr(c.status), ctypes.byref(c.opts), _ptr(ws), ws.numel(), _stream(c.device)))
    res = {"chi_inf": chi, "t_inf": age, "status": c.status}
    if grad:
        res["grad"] = g
    return res


class HostVJP:
    """lcdm_distances_vjp_host: the fused forward + adjoint on host arrays,
    with chunked copies overlapping the kernels.  Inputs and the output arrays
    are CPU tensors (page-locked for overlap); the device workspace and the
    output buffers are allocated once here and reused by every call."""

    def __init__(self, B, n, outputs=("d_C", "t", "X", "mu"), ncol=4, precision="fp32", nchunks=4,
                 device="cuda", block=0, blocks_per_sm=0, lane_map="tuned"):
        lib = load()
        self.device = torch.device(device)
        self.opts = Opts(ncol, PRECISION[precision], LAYOUT["csr"], block, blocks_per_sm, LANE_MAP[lane_map])
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.B, self.n, self.nchunks = int(B), int(n), int(nchunks)
        nbytes = ctypes.c_size_t()
        _check(lib.lcdm_host_workspace_size(self.B, self.n, ctypes.byref(self.opts), ctypes.byref(nbytes)))
        self.ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self.outputs = tuple(outputs)
        self.out = {o: torch.empty(self.n, dtype=self.dtype, pin_memory=True) for o in self.outputs}
        self.grad = torch.empty(self.B, ncol, dtype=torch.float64, pin_memory=True)
        self.status = torch.empty(self.B, dtype=torch.int32, pin_memory=True)

    def __call__(self, params, z, cot, offsets):
        """params [B, ncol] float64, z [n], cot {name: [n]}, offsets [B+1] int64:
        CPU tensors.  Returns the (reused) host result tensors."""
        for t in (params, z, offsets, *cot.values()):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("host entry point: contiguous CPU tensors expected")
        cp = _VP6(*[(cot[o].data_ptr() if o in cot else None) for o in OUTS])
        op = _VP6(*[(self.out[o].data_ptr() if o in self.out else None) for o in OUTS])
        _check(load().lcdm_distances_vjp_host(_ptr(params), self.B, _ptr(offsets), _ptr(z), self.n, cp, op,
                                              _ptr(self.grad), _ptr(self.status), ctypes.byref(self.opts),
                                              _ptr(self.ws), self.ws.numel(), self.nchunks, _stream(self.device)))
        res = dict(self.out)
        res["grad"] = self.grad
        res["status"] = self.status
        return res


def gauss_loglike(params, z, m_obs, offsets=None, M=-19.3, sigma=0.1, grad=True, want_mu=False,
                  call=None, grad_z=False, workspace=None, **kw):
    """Gaussian log-likelihood of magnitudes per cosmology and its gradient
    (lcdm_gauss_loglike).  Returns {"loglike": [B], "grad": [B, ncol], ...};
    with grad_z, also "grad_z" [npairs], the derivative of each row's
    log-likelihood with respect to each pair's redshift
    (lcdm_gauss_loglike_dz; ``workspace``: a reusable uint8 device buffer of
    lcdm_loglike_dz_workspace_size bytes)."""
    c = call if call is not None else Call(params, z, offsets, **kw)
    m = m_obs.to(device=c.device, dtype=c.dtype).contiguous()
    ll = torch.empty(c.B, dtype=torch.float64, device=c.device)
    g = torch.empty(c.B, c.ncol, dtype=torch.float64, device=c.device) if grad else None
    mu = torch.empty(c.npairs, dtype=c.dtype, device=c.device) if want_mu else None
    if grad_z:
        gz = torch.empty(c.npairs, dtype=c.dtype, device=c.device)
        ws = workspace if workspace is not None else loglike_dz_workspace(c)
        _check(load().lcdm_gauss_loglike_dz(*c.common()[:4], _ptr(m), c.n, float(M), float(sigma), _ptr(ll), _ptr(g),
                                            _ptr(gz), _ptr(mu), _ptr(c.status), ctypes.byref(c.opts), _ptr(ws),
                                            ws.numel(), _stream(c.device)))
        res = {"loglike": ll, "status": c.status, "grad_z": gz}
        if grad:
            res["grad"] = g
        if want_mu:
            res["mu"] = mu
        return res
    _check(load().lcdm_gauss_loglike(*c.common()[:4], _ptr(m), c.n, float(M), float(sigma), _ptr(ll), _ptr(g),
                                     _ptr(mu), _ptr(c.status), *c.tail()))
    res = {"loglike": ll, "status": c.status}
    if grad:
        res["grad"] = g
    if want_mu:
        res["mu"] = mu
    return res


def loglike_dz_workspace(c):
    """Device workspace of lcdm_gauss_loglike_dz for a prepared Call."""
    nbytes = ctypes.c_size_t()
    _check(load().lcdm_loglike_dz_workspace_size(c.B, c.n, ctypes.byref(c.opts), ctypes.byref(nbytes)))
    return torch.empty(nbytes.value, dtype=torch.uint8, device=c.device)


def autotune(params, z, offsets=None, outputs=("d_C", "t", "X", "mu"), cot=None, **kw):
    """Pick the fastest launch shape for this workload class (lcdm_autotune)."""
    c = Call(params, z, offsets, **kw)
    out, vp = c.out_buffers(outputs)
    cp, grad = _VP6(), None
    if cot is not None:
        cots = {n: v.to(device=c.device, dtype=c.dtype).contiguous() for n, v in cot.items()}
        cp = _VP6(*[(cots[n].data_ptr() if n in cots else None) for n in OUTS])
        grad = torch.empty(c.B, c.ncol, dtype=torch.float64, device=c.device)
    bb, bbps, ms, bm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float(), ctypes.c_int32()
    _check(load().lcdm_autotune(*c.common(), cp, vp, _ptr(grad), _ptr(c.status), *c.tail(), ctypes.byref(bb),
                                ctypes.byref(bbps), ctypes.byref(ms), ctypes.byref(bm)))
    names = {v: k for k, v in LANE_MAP.items()}
    return {"block": bb.value, "blocks_per_sm": bbps.value, "ms": ms.value, "lane_map": names[bm.value]}


class Distances(torch.autograd.Function):
    """d_C, t, X, d_M, d_L, mu as differentiable functions of params and of
    the redshifts (csr and dense layouts).

    Forward runs lcdm_distances; backward runs the fused forward+adjoint
    kernel (lcdm_distances_vjp, or lcdm_distances_vjp_dz when the redshifts
    need a gradient) with the incoming gradients as cotangents."""

    @staticmethod
    def forward(ctx, params, z, offsets, outputs, layout, precision):
        res = distances(params, z, offsets, outputs=outputs, layout=layout, precision=precision)
        ctx.save_for_backward(params, z, offsets if offsets is not None else torch.empty(0))
        ctx.meta = (outputs, layout, precision, offsets is not None)
        return tuple(res[n] for n in outputs)

    @staticmethod
    def backward(ctx, *grads):
        params, z, offsets = ctx.saved_tensors
        outputs, layout, precision, has_off = ctx.meta
        cot = {n: g for n, g in zip(outputs, grads) if g is not None}
        want_z = ctx.needs_input_grad[1]
        if want_z and layout == "shared":
            raise ValueError("redshift gradients need the csr or dense layout")
        res = distances_vjp(params, z, cot, offsets if has_off else None, layout=layout, precision=precision,
                            grad_z=want_z)
        gz = res["grad_z"].reshape(z.shape).to(z.dtype) if want_z else None
        return res["grad"].to(params.dtype), gz, None, None, None, None


def distances_autograd(params, z, offsets=None, outputs=("d_C", "mu"), layout=None, precision="fp32"):
    """Differentiable wrapper: returns a tuple of output tensors."""
    return Distances.apply(params, z, offsets, tuple(outputs), layout, precision)
