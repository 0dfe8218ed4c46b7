"""ctypes binding of the to3d C interface (include/to3d.h).

Argument marshalling only: every step of the path runs in the CUDA library.
Arrays may be NumPy arrays (host memory, ``on_device = 0``) or CUDA torch
tensors (device memory, ``on_device = 1``); the work goes on the stream the
context was created with (by default torch's current stream).

If the library is missing or cannot be loaded the import fails loudly: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libto3d.so")

F64, BF16_DC, BF16X2_DC, FP16_DC, FP16X2_DC = 0, 1, 2, 3, 4
JACOBI, CNN_FCG, LMG = 0, 1, 2
FILTER_SENS, FILTER_DENS = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
          4: "no convergence", 5: "numerical breakdown", 6: "device wait timed out",
          7: "invalid state"}


class Params(C.Structure):
    _fields_ = [("nelx", C.c_int32), ("nely", C.c_int32), ("nelz", C.c_int32),
                ("volfrac", C.c_double), ("penal", C.c_double), ("rmin", C.c_double),
                ("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double),
                ("move", C.c_double), ("bisect_tol", C.c_double), ("cg_rtol", C.c_double),
                ("inner_rtol", C.c_double),
                ("cg_maxit", C.c_int32), ("filter", C.c_int32), ("precision", C.c_int32),
                ("precond", C.c_int32), ("oc_levels", C.c_int32), ("warm_start", C.c_int32),
                ("fcg_ref_iters", C.c_int32), ("mg_sweeps", C.c_int32), ("fp64_tc", C.c_int32),
                ("mg_keep_dir", C.c_int32), ("mg_nu", C.c_int32), ("reserved", C.c_int32 * 1)]


class IterInfo(C.Structure):
    _fields_ = [("iter", C.c_int32), ("status", C.c_int32),
                ("compliance", C.c_double), ("volume", C.c_double), ("change", C.c_double),
                ("lam", C.c_double), ("relres", C.c_double),
                ("cg_iters", C.c_int32), ("outer_iters", C.c_int32), ("halvings", C.c_int32),
                ("pad", C.c_int32),
                ("ms_solve", C.c_double), ("ms_sens", C.c_double), ("ms_filter", C.c_double),
                ("ms_oc", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer", C.c_int32), ("status", C.c_int32),
                ("pad", C.c_int32), ("relres", C.c_double)]


class To3dError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"to3d status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


_lib = None
VP, I32, DP = C.c_void_p, C.c_int32, C.POINTER(C.c_double)

_SIGS = {
    "to3d_default_params": (I32, [C.POINTER(Params)]),
    "to3d_create": (I32, [C.POINTER(Params), VP, VP, VP, VP, C.POINTER(VP)]),
    "to3d_destroy": (None, [VP]),
    "to3d_last_error": (C.c_char_p, [VP]),
    "to3d_status_string": (C.c_char_p, [I32]),
    "to3d_launch_count": (C.c_int64, [VP]),
    "to3d_kernel_stats": (I32, [VP, I32, DP, C.POINTER(C.c_int64), I32]),
    "to3d_step": (I32, [VP, C.POINTER(IterInfo)]),
    "to3d_run": (I32, [VP, I32, C.POINTER(IterInfo)]),
    "to3d_get_density": (I32, [VP, VP, I32]),
    "to3d_set_density": (I32, [VP, VP, I32]),
    "to3d_get_displacement": (I32, [VP, VP, I32]),
    "to3d_set_displacement": (I32, [VP, VP, I32]),
    "to3d_get_iteration": (I32, [VP, C.POINTER(I32)]),
    "to3d_set_iteration": (I32, [VP, I32]),
    "to3d_selftest_wait_timeout": (I32, [I32, C.POINTER(I32), VP]),
    "to3d_matvec": (I32, [VP, VP, VP, VP, I32]),
    "to3d_matvec_lowp": (I32, [VP, VP, VP, VP, I32, I32]),
    "to3d_solve": (I32, [VP, VP, VP, VP, I32, C.POINTER(SolveInfo)]),
    "to3d_sensitivity": (I32, [VP, VP, VP, VP, VP, DP, I32]),
    "to3d_filter_apply": (I32, [VP, I32, VP, VP, VP, I32, I32]),
    "to3d_oc_update": (I32, [VP, VP, VP, VP, DP, DP, C.POINTER(I32), I32]),
    "to3d_sensitivity_noalloc": (I32, [I32, I32, I32, C.c_double, C.c_double, C.c_double,
                                       C.c_double, VP, VP, VP, VP, DP, VP]),
    "to3d_cnn_init": (I32, [VP, C.c_uint64]),
    "to3d_cnn_param_count": (I32, [VP, C.POINTER(C.c_int64)]),
    "to3d_cnn_get_params": (I32, [VP, VP, C.c_int64]),
    "to3d_cnn_set_params": (I32, [VP, VP, C.c_int64]),
    "to3d_cnn_apply": (I32, [VP, VP, VP, VP, I32]),
    "to3d_cnn_train": (I32, [VP, I32, I32, I32, C.c_double, C.c_uint64, I32, DP, DP]),
    "to3d_cnn_loss_grad": (I32, [VP, VP, VP, VP, I32, VP, C.c_int64, DP]),
    "to3d_mg_param_count": (I32, [VP, C.POINTER(C.c_int64)]),
    "to3d_mg_get_params": (I32, [VP, DP, C.c_int64]),
    "to3d_mg_set_params": (I32, [VP, DP, C.c_int64]),
    "to3d_mg_levels": (I32, [VP, C.POINTER(I32)]),
    "to3d_mg_apply": (I32, [VP, VP, VP, VP, I32]),
    "to3d_mg_train": (I32, [VP, I32, I32, C.c_double, C.c_uint64, I32, DP, DP]),
    "to3d_conv3d_forward": (I32, [I32, I32, I32, I32, I32, I32, VP, VP, VP, VP, I32, VP, VP]),
    "to3d_conv3d_backward": (I32, [I32, I32, I32, I32, I32, I32, VP, VP, VP, VP, VP, VP, VP, VP,
                                   VP]),
    "to3d_batch_create": (I32, [I32, C.POINTER(Params), C.POINTER(VP), C.POINTER(VP),
                                C.POINTER(VP), VP, C.POINTER(VP)]),
    "to3d_batch_step": (I32, [VP, C.POINTER(IterInfo)]),
    "to3d_batch_get_density": (I32, [VP, I32, VP, I32]),
    "to3d_batch_size": (I32, [VP]),
    "to3d_batch_set_mg_params": (I32, [VP, DP, C.c_int64]),
    "to3d_batch_destroy": (None, [VP]),
}


def exported_symbols():
    return list(_SIGS)


def load(path: str = LIB_PATH):
    """Load libto3d.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_params(**kw) -> Params:
    p = Params()
    load().to3d_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class _Arg:
    """Pointer + on_device flag for a NumPy array or a CUDA torch tensor."""

    def __init__(self, a, dtype):
        if _is_torch(a):
            import torch
            want = {np.float64: torch.float64, np.float32: torch.float32,
                    np.uint8: torch.uint8}[dtype]
            if not a.is_cuda or a.dtype != want or not a.is_contiguous():
                raise TypeError(f"expected a contiguous CUDA {want} tensor")
            self.obj, self.ptr, self.dev = a, a.data_ptr(), 1
        else:
            arr = np.ascontiguousarray(a, dtype=dtype)
            self.obj, self.ptr, self.dev = arr, arr.ctypes.data, 0


def _need(arg, n, name):
    """Refuse an array shorter or longer than the grid implies before its
    pointer reaches the library (which reads and writes exactly n entries)."""
    got = int(arg.obj.numel()) if _is_torch(arg.obj) else int(arg.obj.size)
    if got != n:
        raise ValueError(f"{name} has {got} entries, the grid needs {n}")
    return arg


def _same_kind(*args):
    devs = {a.dev for a in args if a is not None}
    if len(devs) > 1:
        raise TypeError("mix of host and device arrays in one call")
    return devs.pop() if devs else 0


class Context:
    """One problem on one GPU (wraps ``to3d_create`` / ``to3d_destroy``)."""

    def __init__(self, nelx, nely, nelz, fixed, load_vec, passive=None, stream=None, **params):
        lib = load()
        self.lib = lib
        self.params = default_params(nelx=nelx, nely=nely, nelz=nelz, **params)
        self.nelx, self.nely, self.nelz = nelx, nely, nelz
        self.nel = nelx * nely * nelz
        self.ndof = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
        fixed = np.ascontiguousarray(fixed, np.uint8)
        load_vec = np.ascontiguousarray(load_vec, np.float64)
        if fixed.size != self.ndof or load_vec.size != self.ndof:
            raise ValueError("fixed/load must have 3N entries")
        pas = None
        if passive is not None:
            pas = np.ascontiguousarray(passive, np.uint8)
            if pas.size != self.nel:
                raise ValueError("passive must have nel entries")
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        h = VP()
        st = lib.to3d_create(C.byref(self.params), fixed.ctypes.data, load_vec.ctypes.data,
                             pas.ctypes.data if pas is not None else None, VP(stream), C.byref(h))
        if st != 0:
            raise To3dError(st, "to3d_create failed")
        self.h = h

    @classmethod
    def from_problem(cls, prob, **params):
        kw = dict(volfrac=prob.volfrac, penal=prob.penal, rmin=prob.rmin, E0=prob.E0,
                  Emin=prob.Emin, nu=prob.nu, move=prob.move, bisect_tol=prob.bisect_tol)
        kw.update(params)
        return cls(prob.nelx, prob.nely, prob.nelz, prob.fixed, prob.load, prob.passive, **kw)

    def close(self):
        if getattr(self, "h", None):
            self.lib.to3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.to3d_last_error(self.h)
            raise To3dError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def launches(self) -> int:
        return int(self.lib.to3d_launch_count(self.h))

    def kernel_stats(self, which: int, reset: bool = False):
        """(summed ms, samples) of sampled launches of the tensor-core (0) or
        FP64 (1) matvec inside the solver."""
        ms, n = C.c_double(), C.c_int64()
        self._check(self.lib.to3d_kernel_stats(self.h, which, C.byref(ms), C.byref(n),
                                               int(reset)), "kernel_stats")
        return ms.value, n.value

    # ---- whole iterations
    def step(self) -> dict:
        info = IterInfo()
        self._check(self.lib.to3d_step(self.h, C.byref(info)), "to3d_step")
        return info.as_dict()

    def run(self, iters: int):
        hist = (IterInfo * max(iters, 1))()
        self._check(self.lib.to3d_run(self.h, iters, hist), "to3d_run")
        return [hist[i].as_dict() for i in range(iters)]

    def density(self, out=None):
        out = np.empty(self.nel) if out is None else out
        a = _need(_Arg(out, np.float64), self.nel, "x")
        self._check(self.lib.to3d_get_density(self.h, a.ptr, a.dev), "get_density")
        return out

    def set_density(self, x):
        a = _need(_Arg(x, np.float64), self.nel, "x")
        self._check(self.lib.to3d_set_density(self.h, a.ptr, a.dev), "set_density")

    def set_displacement(self, u):
        a = _need(_Arg(u, np.float64), self.ndof, "u")
        self._check(self.lib.to3d_set_displacement(self.h, a.ptr, a.dev), "set_displacement")

    @property
    def iteration(self) -> int:
        it = I32()
        self._check(self.lib.to3d_get_iteration(self.h, C.byref(it)), "get_iteration")
        return it.value

    def save_state(self, path):
        """Checkpoint: design, displacement and OC iteration to an .npz file."""
        np.savez(path, x=self.density(), u=self.displacement(), iteration=self.iteration)

    def load_state(self, path):
        """Resume from ``save_state``: the next OC iteration repeats the one
        the saved context would have run next."""
        with np.load(path) as d:
            self.set_density(np.ascontiguousarray(d["x"]))
            self.set_displacement(np.ascontiguousarray(d["u"]))
            self._check(self.lib.to3d_set_iteration(self.h, int(d["iteration"])), "set_iteration")

    def displacement(self, out=None):
        out = np.empty(self.ndof) if out is None else out
        a = _need(_Arg(out, np.float64), self.ndof, "u")
        self._check(self.lib.to3d_get_displacement(self.h, a.ptr, a.dev), "get_displacement")
        return out

    # ---- single steps
    def matvec(self, x, p, y=None):
        y = np.empty(self.ndof) if y is None else y
        ax, ap, ay = (_need(_Arg(x, np.float64), self.nel, "x"),
                      _need(_Arg(p, np.float64), self.ndof, "p"),
                      _need(_Arg(y, np.float64), self.ndof, "y"))
        dev = _same_kind(ax, ap, ay)
        self._check(self.lib.to3d_matvec(self.h, ax.ptr, ap.ptr, ay.ptr, dev), "matvec")
        return y

    def matvec_lowp(self, x, p32, prec=BF16_DC, y=None):
        y = np.empty(self.ndof, np.float32) if y is None else y
        ax, ap, ay = (_need(_Arg(x, np.float64), self.nel, "x"),
                      _need(_Arg(p32, np.float32), self.ndof, "p"),
                      _need(_Arg(y, np.float32), self.ndof, "y"))
        dev = _same_kind(ax, ap, ay)
        self._check(self.lib.to3d_matvec_lowp(self.h, ax.ptr, ap.ptr, ay.ptr, prec, dev),
                    "matvec_lowp")
        return y

    def solve(self, x, f=None, u=None):
        u = np.zeros(self.ndof) if u is None else u
        ax, au = _need(_Arg(x, np.float64), self.nel, "x"), _need(_Arg(u, np.float64), self.ndof, "u")
        af = _need(_Arg(f, np.float64), self.ndof, "f") if f is not None else None
        dev = _same_kind(ax, au, af)
        info = SolveInfo()
        st = self.lib.to3d_solve(self.h, ax.ptr, af.ptr if af else None, au.ptr, dev,
                                 C.byref(info))
        self._check(st, "solve")
        return u, {"iters": info.iters, "outer": info.outer, "status": info.status,
                   "relres": info.relres}

    def sensitivity(self, x, u, ce=None, dc=None):
        ce = np.empty(self.nel) if ce is None else ce
        dc = np.empty(self.nel) if dc is None else dc
        ax, au, ac, ad = (_need(_Arg(x, np.float64), self.nel, "x"),
                          _need(_Arg(u, np.float64), self.ndof, "u"),
                          _need(_Arg(ce, np.float64), self.nel, "ce"),
                          _need(_Arg(dc, np.float64), self.nel, "dc"))
        dev = _same_kind(ax, au, ac, ad)
        comp = C.c_double()
        self._check(self.lib.to3d_sensitivity(self.h, ax.ptr, au.ptr, ac.ptr, ad.ptr,
                                              C.byref(comp), dev), "sensitivity")
        return ce, dc, comp.value

    def filter(self, v, x=None, kind=FILTER_SENS, transpose=False, out=None):
        out = np.empty(self.nel) if out is None else out
        av, ao = _need(_Arg(v, np.float64), self.nel, "v"), _need(_Arg(out, np.float64), self.nel, "out")
        ax = _need(_Arg(x, np.float64), self.nel, "x") if x is not None else None
        dev = _same_kind(av, ao, ax)
        self._check(self.lib.to3d_filter_apply(self.h, kind, ax.ptr if ax else None, av.ptr,
                                               ao.ptr, int(transpose), dev), "filter")
        return out

    def oc_update(self, x, dcf, xnew=None):
        xnew = np.empty(self.nel) if xnew is None else xnew
        ax, ad, an = (_need(_Arg(x, np.float64), self.nel, "x"),
                      _need(_Arg(dcf, np.float64), self.nel, "dcf"),
                      _need(_Arg(xnew, np.float64), self.nel, "xnew"))
        dev = _same_kind(ax, ad, an)
        lam, vol, nh = C.c_double(), C.c_double(), I32()
        self._check(self.lib.to3d_oc_update(self.h, ax.ptr, ad.ptr, an.ptr, C.byref(lam),
                                            C.byref(vol), C.byref(nh), dev), "oc_update")
        return xnew, lam.value, vol.value, nh.value

    # ---- learned preconditioner (not in the paper; optional)
    def cnn_init(self, seed: int = 0):
        self._check(self.lib.to3d_cnn_init(self.h, seed), "cnn_init")

    def cnn_param_count(self) -> int:
        n = C.c_int64()
        self._check(self.lib.to3d_cnn_param_count(self.h, C.byref(n)), "cnn_param_count")
        return n.value

    def cnn_params(self) -> np.ndarray:
        p = np.empty(self.cnn_param_count(), np.float32)
        self._check(self.lib.to3d_cnn_get_params(self.h, p.ctypes.data, p.size), "cnn_params")
        return p

    def set_cnn_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.to3d_cnn_set_params(self.h, p.ctypes.data, p.size), "set_cnn_params")

    def cnn_apply(self, x, r, z=None):
        z = np.empty(self.ndof) if z is None else z
        ax, ar, az = (_need(_Arg(x, np.float64), self.nel, "x"),
                      _need(_Arg(r, np.float64), self.ndof, "r"),
                      _need(_Arg(z, np.float64), self.ndof, "z"))
        dev = _same_kind(ax, ar, az)
        self._check(self.lib.to3d_cnn_apply(self.h, ax.ptr, ar.ptr, az.ptr, dev), "cnn_apply")
        return z

    def cnn_loss_grad(self, x, r, e):
        g = np.empty(self.cnn_param_count(), np.float32)
        ax, ar, ae = (_need(_Arg(x, np.float64), self.nel, "x"),
                      _need(_Arg(r, np.float64), self.ndof, "r"),
                      _need(_Arg(e, np.float64), self.ndof, "e"))
        dev = _same_kind(ax, ar, ae)
        loss = C.c_double()
        self._check(self.lib.to3d_cnn_loss_grad(self.h, ax.ptr, ar.ptr, ae.ptr, dev,
                                                g.ctypes.data, g.size, C.byref(loss)),
                    "cnn_loss_grad")
        return loss.value, g

    def cnn_train(self, nsnap: int, per_design: int = 8, steps: int = 200, lr: float = 1e-3,
                  seed: int = 0, source: int = 0):
        """Take ``nsnap`` residual snapshots (source 0: Jacobi-PCG, 1: flexible
        CG with the current network) and run ``steps`` Adam steps; returns
        the mean energy loss of the first and last tenth of the steps."""
        a, b = C.c_double(), C.c_double()
        self._check(self.lib.to3d_cnn_train(self.h, nsnap, per_design, steps, lr, seed, source,
                                            C.byref(a), C.byref(b)), "cnn_train")
        return a.value, b.value

    # ---- learned multigrid preconditioner (not in the paper)
    def mg_params(self) -> np.ndarray:
        n = C.c_int64()
        self._check(self.lib.to3d_mg_param_count(self.h, C.byref(n)), "mg_param_count")
        th = np.empty(n.value)
        self._check(self.lib.to3d_mg_get_params(self.h, th.ctypes.data_as(DP), th.size),
                    "mg_params")
        return th

    def set_mg_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(self.lib.to3d_mg_set_params(self.h, th.ctypes.data_as(DP), th.size),
                    "set_mg_params")

    def mg_levels(self) -> int:
        n = I32()
        self._check(self.lib.to3d_mg_levels(self.h, C.byref(n)), "mg_levels")
        return n.value

    def mg_apply(self, x, r, z=None):
        z = np.empty(self.ndof) if z is None else z
        ax, ar, az = (_need(_Arg(x, np.float64), self.nel, "x"),
                      _need(_Arg(r, np.float64), self.ndof, "r"),
                      _need(_Arg(z, np.float64), self.ndof, "z"))
        dev = _same_kind(ax, ar, az)
        self._check(self.lib.to3d_mg_apply(self.h, ax.ptr, ar.ptr, az.ptr, dev), "mg_apply")
        return z

    def mg_train(self, nsnap: int = 8, steps: int = 40, lr: float = 0.05, seed: int = 0,
                 append: bool = False):
        """Take `nsnap` snapshots on the current design (added to earlier
        ones with `append`) and learn the multigrid parameters over all of
        them for `steps` Adam steps; returns the mean energy loss before and
        after."""
        a, b = C.c_double(), C.c_double()
        self._check(self.lib.to3d_mg_train(self.h, nsnap, steps, lr, seed, int(append),
                                           C.byref(a), C.byref(b)), "mg_train")
        return a.value, b.value


def selftest_wait_timeout(polls: int = 256, stream=None) -> int:
    """Status a bounded device-side wait reports when nothing completes it
    (``to3d_selftest_wait_timeout``): TO3D_ETIMEOUT."""
    st = I32()
    r = load().to3d_selftest_wait_timeout(polls, C.byref(st), _stream_ptr(stream))
    if r:
        raise To3dError(r, "to3d_selftest_wait_timeout")
    return st.value


def _stream_ptr(stream):
    if stream is None:
        import torch
        return VP(torch.cuda.current_stream().cuda_stream)
    return VP(stream)


def _dev_ptr(t, dtype_name):
    if t is None:
        return None
    if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
        raise TypeError("convolution hooks take contiguous CUDA tensors")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    return t.data_ptr()


def conv3d_forward(in1, W, out, in2=None, bias=None, relu=False, stream=None):
    """One 3x3x3 convolution (``to3d_conv3d_forward``): channels-last BF16
    in1 [Z,Y,X,C1] (+ in2 [Z,Y,X,C2]), W BF16 [27,Cout,C1+C2], FP32 bias and
    out [Z,Y,X,Cout]."""
    Z, Y, X, C1 = in1.shape
    C2 = in2.shape[3] if in2 is not None else 0
    st = load().to3d_conv3d_forward(Z, Y, X, C1, C2, out.shape[3], _dev_ptr(in1, "bfloat16"),
                                    _dev_ptr(in2, "bfloat16"), _dev_ptr(W, "bfloat16"),
                                    _dev_ptr(bias, "float32"), int(relu),
                                    _dev_ptr(out, "float32"), _stream_ptr(stream))
    if st:
        raise To3dError(st, "to3d_conv3d_forward")
    return out


def conv3d_backward(x1, W, gy, gw, gb=None, gx=None, x2=None, act=None, stream=None):
    """Backward of ``conv3d_forward`` (``to3d_conv3d_backward``): gw, gb
    accumulate, gx is overwritten."""
    Z, Y, X, C1 = x1.shape
    C2 = x2.shape[3] if x2 is not None else 0
    st = load().to3d_conv3d_backward(Z, Y, X, C1, C2, gy.shape[3], _dev_ptr(x1, "bfloat16"),
                                     _dev_ptr(x2, "bfloat16"), _dev_ptr(W, "bfloat16"),
                                     _dev_ptr(gy, "float32"), _dev_ptr(act, "bfloat16"),
                                     _dev_ptr(gx, "float32"), _dev_ptr(gw, "float32"),
                                     _dev_ptr(gb, "float32"), _stream_ptr(stream))
    if st:
        raise To3dError(st, "to3d_conv3d_backward")
    return gw, gb, gx



def sensitivity_noalloc(nelx, nely, nelz, x, u, ce, dc, penal=3.0, E0=1.0, Emin=1e-9, nu=0.3,
                        stream=None):
    """Energies, sensitivities and compliance into caller-owned CUDA tensors
    with no device allocation by the library (``to3d_sensitivity_noalloc``).
    x, u are inputs and ce, dc outputs: contiguous CUDA float64 tensors.
    Returns the compliance."""
    nel = int(nelx) * int(nely) * int(nelz)
    ndof = 3 * (int(nelx) + 1) * (int(nely) + 1) * (int(nelz) + 1)
    args = [_need(_Arg(t, np.float64), n, name)
            for t, n, name in ((x, nel, "x"), (u, ndof, "u"), (ce, nel, "ce"), (dc, nel, "dc"))]
    if any(a.dev != 1 for a in args):
        raise TypeError("sensitivity_noalloc takes CUDA tensors only")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    comp = C.c_double()
    st = load().to3d_sensitivity_noalloc(nelx, nely, nelz, penal, E0, Emin, nu, args[0].ptr,
                                         args[1].ptr, args[2].ptr, args[3].ptr, C.byref(comp),
                                         VP(stream))
    if st != 0:
        raise To3dError(st, "to3d_sensitivity_noalloc")
    return comp.value


class Batch:
    """Independent problems stepped together (``to3d_batch_*``)."""

    def __init__(self, probs, stream=None, **params):
        lib = load()
        self.lib = lib
        n = len(probs)
        self.params = (Params * n)()
        keep = []
        fixed = (VP * n)()
        loads = (VP * n)()
        pas = (VP * n)()
        for i, pr in enumerate(probs):
            kw = dict(volfrac=pr.volfrac, penal=pr.penal, rmin=pr.rmin, E0=pr.E0, Emin=pr.Emin,
                      nu=pr.nu, move=pr.move, bisect_tol=pr.bisect_tol, precision=BF16X2_DC)
            kw.update(params)
            self.params[i] = default_params(nelx=pr.nelx, nely=pr.nely, nelz=pr.nelz, **kw)
            f = np.ascontiguousarray(pr.fixed, np.uint8)
            l = np.ascontiguousarray(pr.load, np.float64)
            keep += [f, l]
            fixed[i], loads[i] = f.ctypes.data, l.ctypes.data
            if pr.passive is not None:
                pp = np.ascontiguousarray(pr.passive, np.uint8)
                keep.append(pp)
                pas[i] = pp.ctypes.data
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        h = VP()
        st = lib.to3d_batch_create(n, self.params, fixed, loads, pas, VP(stream), C.byref(h))
        if st != 0:
            raise To3dError(st, "to3d_batch_create failed")
        self.h, self.n = h, n
        self.nel = [pr.nel for pr in probs]

    def step(self):
        info = (IterInfo * self.n)()
        st = self.lib.to3d_batch_step(self.h, info)
        recs = [info[i].as_dict() for i in range(self.n)]
        if st != 0:
            raise To3dError(st, "to3d_batch_step")
        return recs

    def set_mg_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        st = self.lib.to3d_batch_set_mg_params(self.h, th.ctypes.data_as(DP), th.size)
        if st != 0:
            raise To3dError(st, "to3d_batch_set_mg_params")

    def density(self, i):
        out = np.empty(self.nel[i])
        st = self.lib.to3d_batch_get_density(self.h, i, out.ctypes.data, 0)
        if st != 0:
            raise To3dError(st, "to3d_batch_get_density")
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.to3d_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
