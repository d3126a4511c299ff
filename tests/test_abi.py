"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/lcdm.h declares; argument checks that run
before any CUDA call return the documented status codes."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lcdm.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:lcdm_status|const char\*|int64_t)\s+(lcdm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def cdll():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2212_01937_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("lcdm_workspace_size", "lcdm_roots", "lcdm_distances", "lcdm_distances_jac",
              "lcdm_distances_vjp", "lcdm_gauss_loglike", "lcdm_autotune", "lcdm_status_string",
              "lcdm_launch_count", "lcdm_between_workspace_size", "lcdm_distances_between", "lcdm_limits",
              "lcdm_loglike_dz_workspace_size", "lcdm_gauss_loglike_dz", "lcdm_distances_vjp_dz"):
        assert s in syms


def test_library_exports_every_declared_symbol(cdll):
    for s in declared_symbols():
        assert hasattr(cdll, s), s


def test_host_argument_checks(cdll):
    from paper_2212_01937_gb300.lcdm import Opts
    cdll.lcdm_status_string.restype = ctypes.c_char_p
    assert b"OK" in cdll.lcdm_status_string(0)
    good = Opts(4, 1, 0, 0, 0)
    n = ctypes.c_size_t()
    assert cdll.lcdm_workspace_size(ctypes.c_int64(4096), ctypes.byref(good), ctypes.byref(n)) == 0
    assert n.value >= 4096 * 38 * 16
    bad = Opts(3, 1, 0, 0, 0)
    assert cdll.lcdm_workspace_size(ctypes.c_int64(10), ctypes.byref(bad), ctypes.byref(n)) == 1
    # null params -> invalid before any CUDA call
    out = (ctypes.c_void_p * 6)()
    st = cdll.lcdm_distances(None, ctypes.c_int64(1), None, None, ctypes.c_int64(0), out, None,
                             ctypes.byref(good), None, ctypes.c_size_t(0), None)
    assert st == 1


def test_general_limits_argument_checks(cdll):
    from paper_2212_01937_gb300.lcdm import Opts
    n = ctypes.c_size_t()
    csr, shared = Opts(4, 1, 0, 0, 0), Opts(4, 1, 2, 0, 0)
    i64 = ctypes.c_int64
    assert cdll.lcdm_between_workspace_size(i64(16), i64(100), ctypes.byref(csr), ctypes.byref(n)) == 0
    small = n.value
    assert cdll.lcdm_between_workspace_size(i64(16), i64(200), ctypes.byref(csr), ctypes.byref(n)) == 0
    assert n.value > small
    # the shared layout has no per-row z1 shift; n = 0 (lcdm_limits) accepts any layout
    assert cdll.lcdm_between_workspace_size(i64(16), i64(100), ctypes.byref(shared), ctypes.byref(n)) == 1
    assert cdll.lcdm_between_workspace_size(i64(16), i64(0), ctypes.byref(shared), ctypes.byref(n)) == 0
    out = (ctypes.c_void_p * 6)()
    vp = ctypes.c_void_p
    # z1 missing -> invalid, before any CUDA call
    st = cdll.lcdm_distances_between(vp(8), i64(1), None, vp(8), vp(8), i64(4), None, out, None, vp(8),
                                     ctypes.byref(csr), None, ctypes.c_size_t(0), None)
    assert st == 1
    # gradient without cotangents -> invalid
    st = cdll.lcdm_distances_between(vp(8), i64(1), vp(8), vp(8), vp(8), i64(4), None, out, vp(8), vp(8),
                                     ctypes.byref(csr), None, ctypes.c_size_t(0), None)
    assert st == 1
    # limits: nothing requested -> invalid; missing workspace -> workspace error
    st = cdll.lcdm_limits(vp(8), i64(1), vp(8), None, None, None, None, None, vp(8), ctypes.byref(csr),
                          None, ctypes.c_size_t(0), None)
    assert st == 1
    st = cdll.lcdm_limits(vp(8), i64(1), vp(8), vp(8), None, None, None, None, vp(8), ctypes.byref(csr),
                          None, ctypes.c_size_t(0), None)
    assert st == 3


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2212_01937_gb300 import lcdm
    monkeypatch.setattr(lcdm, "_lib", None)
    monkeypatch.setattr(lcdm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        lcdm.load()


def test_seven_column_rows_refused_where_unsupported(cdll):
    """Seven-column rows (the further components) carry tangents in every
    direction, but the per-row shift of the general limits and the E(z) of
    the redshift-derivative kernel take four or five columns: those entry
    points return LCDM_ERR_UNSUPPORTED (4) before any CUDA call."""
    from paper_2212_01937_gb300.lcdm import Opts
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    o7 = Opts(7, 1, 0, 0, 0, 0)
    n = ctypes.c_size_t()
    assert cdll.lcdm_workspace_size(i64(4), ctypes.byref(o7), ctypes.byref(n)) == 0
    fake, ws = vp(0x1000), vp(0x100000)          # never dereferenced: the calls stop at the checks
    big = sz(1 << 40)
    six = lambda: (ctypes.c_void_p * 6)(*([0x1000] * 6))
    none6 = (ctypes.c_void_p * 6)()
    assert cdll.lcdm_distances_between(fake, i64(4), fake, fake, fake, i64(8), None, six(), None, fake,
                                       ctypes.byref(o7), ws, big, None) == 4
    assert cdll.lcdm_limits(fake, i64(4), fake, fake, fake, None, None, None, fake, ctypes.byref(o7), ws, big,
                            None) == 4
    assert cdll.lcdm_gauss_loglike_dz(fake, i64(4), fake, fake, fake, i64(8), ctypes.c_double(0.0),
                                      ctypes.c_double(0.1), fake, None, fake, None, fake, ctypes.byref(o7), ws,
                                      big, None) == 4
    assert cdll.lcdm_distances_vjp_dz(fake, i64(4), fake, fake, i64(8), six(), none6, None, fake, fake,
                                      ctypes.byref(o7), ws, big, None) == 4


def test_deterministic_workspace_and_refusals(cdll):
    """The deterministic reduction needs a larger workspace; the entry points
    that do not offer it refuse it before any CUDA call."""
    from paper_2212_01937_gb300.lcdm import Opts
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    n0, n1 = ctypes.c_size_t(), ctypes.c_size_t()
    assert cdll.lcdm_workspace_size(i64(64), ctypes.byref(Opts(4, 1, 0, 0, 0, 0, 0)), ctypes.byref(n0)) == 0
    od = Opts(4, 1, 0, 0, 0, 0, 1)
    assert cdll.lcdm_workspace_size(i64(64), ctypes.byref(od), ctypes.byref(n1)) == 0
    assert n1.value > n0.value
    assert cdll.lcdm_workspace_size(i64(64), ctypes.byref(Opts(4, 1, 0, 0, 0, 0, 2)), ctypes.byref(n1)) == 1
    fake, ws, big = vp(0x1000), vp(0x100000), sz(1 << 40)
    six = lambda: (ctypes.c_void_p * 6)(*([0x1000] * 6))
    none6 = (ctypes.c_void_p * 6)()
    assert cdll.lcdm_gauss_loglike_dz(fake, i64(4), fake, fake, fake, i64(8), ctypes.c_double(0.0),
                                      ctypes.c_double(0.1), fake, None, fake, None, fake, ctypes.byref(od), ws,
                                      big, None) == 4
    assert cdll.lcdm_distances_between(fake, i64(4), fake, fake, fake, i64(8), six(), six(), fake, fake,
                                       ctypes.byref(od), ws, big, None) == 4
    offs = (ctypes.c_int64 * 5)(0, 2, 4, 6, 8)
    assert cdll.lcdm_distances_vjp_host(fake, i64(4), offs, fake, i64(8), six(), none6, fake, fake,
                                        ctypes.byref(od), ws, big, ctypes.c_int32(2), None) == 4
