"""Argument checks of the C interface that run before any CUDA call, so they
are exercised on the CPU: default parameters and rejected inputs."""
import ctypes as C
import os
import shutil

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_05604_gb300 import binding, build
    build.build()
    return binding.load()


def params(lib, **kw):
    from paper_2504_05604_gb300.binding import Params
    p = Params()
    assert lib.to3d_default_params(C.byref(p)) == 0
    p.nelx, p.nely, p.nelz = 4, 3, 2
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def create(lib, p, fixed=True, load=True, out=True):
    n = 3 * (p.nelx + 1) * (p.nely + 1) * (p.nelz + 1) if p.nelx > 0 else 3
    n = min(max(n, 3), 1 << 20)
    fx = np.zeros(n, np.uint8)
    f = np.zeros(n)
    h = C.c_void_p()
    return lib.to3d_create(C.byref(p), fx.ctypes.data if fixed else None,
                           f.ctypes.data if load else None, None, None,
                           C.byref(h) if out else None)


def test_default_params(lib):
    p = params(lib)
    assert (p.volfrac, p.penal, p.rmin, p.E0, p.Emin, p.nu) == (0.3, 3.0, 1.5, 1.0, 1e-9, 0.3)
    assert (p.move, p.bisect_tol, p.cg_rtol, p.inner_rtol) == (0.2, 1e-3, 1e-8, 0.3)
    assert (p.precision, p.precond, p.filter, p.oc_levels, p.warm_start) == (0, 0, 0, 3, 1)
    assert p.fcg_ref_iters == 0
    assert lib.to3d_default_params(None) == 1


@pytest.mark.parametrize("field,value", [
    ("nelx", 0), ("nely", -1), ("volfrac", 0.0), ("volfrac", 1.5), ("penal", 0.5),
    ("rmin", 0.0), ("E0", 0.0), ("Emin", 0.0), ("Emin", 2.0), ("nu", 0.5), ("nu", -1.0),
    ("move", 0.0), ("bisect_tol", 0.0), ("cg_rtol", 0.0), ("cg_maxit", 0), ("oc_levels", 0),
    ("oc_levels", 6), ("precision", 5), ("precision", -1), ("precond", 3), ("filter", 2),
    ("fcg_ref_iters", -1)])
def test_create_rejects_bad_parameters(lib, field, value):
    assert create(lib, params(lib, **{field: value})) == 1       # TO3D_EINVAL


def test_create_rejects_too_large_grid(lib):
    assert create(lib, params(lib, nelx=1024, nely=1024, nelz=1024)) == 1


def test_create_rejects_null_pointers(lib):
    p = params(lib)
    assert create(lib, p, fixed=False) == 1
    assert create(lib, p, load=False) == 1
    assert create(lib, p, out=False) == 1


def test_entry_points_reject_null_context(lib):
    assert lib.to3d_step(None, None) == 1
    assert lib.to3d_run(None, 1, None) == 1
    assert lib.to3d_cnn_init(None, 0) == 1
    assert lib.to3d_batch_step(None, None) == 1
    assert lib.to3d_launch_count(None) == 0
    lib.to3d_destroy(None)
    lib.to3d_batch_destroy(None)


def test_create_rejects_non_finite_load(lib):
    p = params(lib)
    n = 3 * (p.nelx + 1) * (p.nely + 1) * (p.nelz + 1)
    fx = np.zeros(n, np.uint8)
    for bad in (np.nan, np.inf):
        f = np.zeros(n)
        f[5] = bad
        h = C.c_void_p()
        assert lib.to3d_create(C.byref(p), fx.ctypes.data, f.ctypes.data, None, None,
                               C.byref(h)) == 1


def test_selftest_rejects_bad_limits(lib):
    st = C.c_int32()
    assert lib.to3d_selftest_wait_timeout(0, C.byref(st), None) == 1
    assert lib.to3d_selftest_wait_timeout(1 << 20, C.byref(st), None) == 1
    assert lib.to3d_selftest_wait_timeout(8, None, None) == 1


def test_noalloc_rejects_too_large_grid_before_any_cuda_call(lib):
    """The allocation-free entry point checks the grid against its fixed
    scratch before touching the GPU: non-null dummy pointers are never used."""
    d = np.zeros(4)
    comp = C.c_double()
    p = d.ctypes.data
    assert lib.to3d_sensitivity_noalloc(2049, 2048, 2, 3.0, 1.0, 1e-9, 0.3, p, p, p, p,
                                        C.byref(comp), None) == 1
    assert lib.to3d_sensitivity_noalloc(0, 4, 4, 3.0, 1.0, 1e-9, 0.3, p, p, p, p,
                                        C.byref(comp), None) == 1
    assert lib.to3d_sensitivity_noalloc(4, 4, 4, 3.0, 1.0, 1e-9, 0.5, p, p, p, p,
                                        C.byref(comp), None) == 1


def test_binding_refuses_arrays_of_the_wrong_length(lib):
    from paper_2504_05604_gb300 import binding
    ok, short = np.zeros(4 * 3 * 2), np.zeros(5)
    u = np.zeros(3 * 5 * 4 * 3)
    with pytest.raises(ValueError):
        binding.sensitivity_noalloc(4, 3, 2, short, u, ok, ok)
    with pytest.raises(ValueError):
        binding.sensitivity_noalloc(4, 3, 2, ok, short, ok, ok)
    with pytest.raises(ValueError):
        binding.sensitivity_noalloc(4, 3, 2, ok, u, ok, short)
