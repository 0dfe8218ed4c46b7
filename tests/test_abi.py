"""The C library builds for sm_103a, loads, and exports every declared symbol
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "to3d.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"TO3D_API[^;]*?\b(to3d_\w+)\s*\(", text, flags=re.S)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_05604_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_interface():
    syms = declared_symbols()
    for s in ("to3d_create", "to3d_step", "to3d_matvec", "to3d_matvec_lowp", "to3d_solve",
              "to3d_sensitivity", "to3d_filter_apply", "to3d_oc_update", "to3d_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_covers_every_declared_symbol(lib):
    from paper_2504_05604_gb300 import binding
    assert sorted(binding.exported_symbols()) == declared_symbols()


def test_default_params_without_gpu(lib):
    from paper_2504_05604_gb300 import binding
    p = binding.default_params()
    assert p.E0 == 1.0 and p.Emin == 1e-9 and p.nu == 0.3 and p.penal == 3.0
    assert p.cg_rtol == 1e-8 and p.move == 0.2 and p.bisect_tol == 1e-3
    assert lib.to3d_status_string  # callable symbol
    f = lib.to3d_status_string
    f.restype = ctypes.c_char_p
    assert f(4).startswith(b"no convergence")


def test_create_rejects_bad_sizes_without_touching_the_gpu(lib):
    from paper_2504_05604_gb300 import binding
    p = binding.default_params(nelx=0, nely=2, nelz=2)
    h = ctypes.c_void_p()
    fixed = (ctypes.c_uint8 * 27)()
    load = (ctypes.c_double * 27)()
    st = binding.load().to3d_create(ctypes.byref(p), fixed, load, None, None, ctypes.byref(h))
    assert st == 1 and not h.value
