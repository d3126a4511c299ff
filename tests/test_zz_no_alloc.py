"""lcdm_distances_static: the entry point for callers that cannot allocate
device memory (they pass inputs and outputs only; scratch is a fixed array in
the library).  Checked through the C ABI against lcdm_distances on the same
inputs, on two calls in a row.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_static_entry_matches_workspace_entry():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01937_gb300 import lcdm, workloads
    lib = lcdm.load()
    fn = lib.lcdm_distances_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                   ctypes.c_void_p * 6, ctypes.c_void_p, ctypes.POINTER(lcdm.Opts), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    dev = torch.device("cuda:0")
    for seed, prec in ((21, "fp32"), (22, "fp64")):
        b = workloads.general_batch(B=40, n=77, seed=seed)
        dt = torch.float32 if prec == "fp32" else torch.float64
        params = torch.tensor(b.params, device=dev)
        z = torch.tensor(b.z, dtype=dt, device=dev)
        offs = torch.tensor(b.offsets, device=dev)
        ref = lcdm.distances(params, z, offs, outputs=lcdm.OUTS, precision=prec)
        opts = lcdm.Opts(4, lcdm.PRECISION[prec], lcdm.LAYOUT["csr"], 0, 0)
        outs = {k: torch.full((b.nnz,), float("nan"), dtype=dt, device=dev) for k in lcdm.OUTS}
        vp = (ctypes.c_void_p * 6)(*[outs[k].data_ptr() for k in lcdm.OUTS])
        status = torch.full((b.B,), -1, dtype=torch.int32, device=dev)
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        for _ in range(2):
            st = fn(params.data_ptr(), b.B, offs.data_ptr(), z.data_ptr(), b.nnz, vp, status.data_ptr(),
                    ctypes.byref(opts), stream)
            assert st == 0, lib.lcdm_status_string(st)
            torch.cuda.synchronize()
            assert torch.equal(status, ref["status"])
            for k in lcdm.OUTS:
                a, r = outs[k].double().cpu().numpy(), ref[k].double().cpu().numpy()
                fin = np.isfinite(r)
                assert np.array_equal(np.isfinite(a), fin)
                assert np.allclose(a[fin], r[fin], rtol=1e-12, atol=0)
            for v in outs.values():
                v.fill_(float("nan"))
    # sizes beyond the stated maximum are rejected before anything is enqueued
    big = torch.tensor(np.tile(b.params[:1], (4097, 1)), device=dev)
    st = fn(big.data_ptr(), 4097, None, z.data_ptr(), 1, vp, status.data_ptr(),
            ctypes.byref(lcdm.Opts(4, 0, lcdm.LAYOUT["dense"], 0, 0)), stream)
    assert st == 1
