"""ctypes wrapper of the oracle's C part (csr_pcg.c): assembled-CSR FP64
Jacobi-PCG, element energies and sensitivities, the sensitivity filter and
the OC bisection, on OpenMP threads.  TEST INFRASTRUCTURE ONLY (see
``oracle/__init__``): used to time the oracle on all host cores; pinned
against the NumPy oracle in tests/test_oracle_csr.py."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build_c

_lib = None


class CSR(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.POINTER(C.c_int64)),
                ("col", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_c.build())
        D, U8 = C.POINTER(C.c_double), C.POINTER(C.c_uint8)
        L.csr_assemble.argtypes = [C.c_int, C.c_int, C.c_int, D, D, U8, C.POINTER(CSR)]
        L.csr_assemble.restype = C.c_int
        L.csr_free.argtypes = [C.POINTER(CSR)]
        L.csr_jacobi_pcg.argtypes = [C.POINTER(CSR), D, D, C.c_double, C.c_int64]
        L.csr_jacobi_pcg.restype = C.c_int64
        L.element_steps.argtypes = [C.c_int, C.c_int, C.c_int, D, D, D, C.c_double, C.c_double,
                                    C.c_double, D, D]
        L.element_steps.restype = C.c_double
        L.sensitivity_filter.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, D, D, D]
        L.oc_update.argtypes = [C.c_int64, D, D, U8, C.c_double, C.c_double, C.c_double, D]
        L.oc_update.restype = C.c_int
        L.omp_threads.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def threads() -> int:
    return int(lib().omp_threads())


class Operator:
    """The clamped operator K(E) as CSR (identity rows/columns on clamped dofs)."""

    def __init__(self, nelx, nely, nelz, E, KE, fixed):
        self.k = CSR()
        self.E = np.ascontiguousarray(E, np.float64)
        self.KE = np.ascontiguousarray(KE, np.float64)
        self.fixed = np.ascontiguousarray(np.asarray(fixed) != 0, np.uint8)
        st = lib().csr_assemble(nelx, nely, nelz, _d(self.E), _d(self.KE),
                                self.fixed.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(self.k))
        if st != 0:
            raise MemoryError("CSR assembly failed")
        self.n = self.k.n

    def matrix(self):
        import scipy.sparse as sp
        nnz = self.k.rowptr[self.n]
        rp = np.ctypeslib.as_array(self.k.rowptr, (self.n + 1,)).copy()
        col = np.ctypeslib.as_array(self.k.col, (nnz,)).copy()
        val = np.ctypeslib.as_array(self.k.val, (nnz,)).copy()
        return sp.csr_matrix((val, col, rp), shape=(self.n, self.n))

    def pcg(self, f, u=None, rtol=1e-8, maxit=10 ** 7):
        """Jacobi-PCG from u (zeros by default); returns (u, iterations)."""
        f = np.ascontiguousarray(f, np.float64)
        u = np.zeros(self.n) if u is None else np.ascontiguousarray(u, np.float64).copy()
        it = lib().csr_jacobi_pcg(C.byref(self.k), _d(f), _d(u), rtol, maxit)
        return u, int(it)

    def close(self):
        if self.k.rowptr:
            lib().csr_free(C.byref(self.k))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def element_steps(nelx, nely, nelz, KE, u, x, penal=3.0, E0=1.0, Emin=1e-9):
    nel = nelx * nely * nelz
    ce, dc = np.empty(nel), np.empty(nel)
    KE = np.ascontiguousarray(KE, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    c = lib().element_steps(nelx, nely, nelz, _d(KE), _d(u), _d(x), penal, E0, Emin, _d(ce), _d(dc))
    return c, ce, dc


def sensitivity_filter(nelx, nely, nelz, rmin, x, dc):
    out = np.empty(nelx * nely * nelz)
    lib().sensitivity_filter(nelx, nely, nelz, rmin, _d(np.ascontiguousarray(x, np.float64)),
                             _d(np.ascontiguousarray(dc, np.float64)), _d(out))
    return out


def oc_update(x, dcf, volfrac, passive=None, move=0.2, tol=1e-3):
    x = np.ascontiguousarray(x, np.float64)
    dcf = np.ascontiguousarray(dcf, np.float64)
    out = np.empty_like(x)
    pas = None if passive is None else np.ascontiguousarray(passive, np.uint8)
    h = lib().oc_update(x.size, _d(x), _d(dcf),
                        pas.ctypes.data_as(C.POINTER(C.c_uint8)) if pas is not None else None,
                        volfrac, move, tol, _d(out))
    return out, int(h)
