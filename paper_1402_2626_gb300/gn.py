"""Python binding of the C ABI in include/gn.h (argument marshalling only).

Every step of the computation runs in the CUDA kernels of ``libgn.so``; this
module only turns torch tensors into device pointers and streams.  It never
falls back to a CPU path: if the library is missing or no CUDA device is
present, calls raise.

Tensor layouts (float64, contiguous, on the CUDA device):
  x, dx : [n, 2, L]        complex vector, re limbs then im limbs
  f     : [N, 2, L]
  J     : [n, N, 2, L]     column-major Jacobian: J[v, i] is d f_i / d x_v
  Ab    : [n+1, m, 2, L]   column-major augmented matrix [A b]
  R     : [n+1, n+1, 2, L] column-major: R[j, k] is r_kj
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgn.so")

PREC = {"d": 1, "dd": 2, "qd": 4, 1: 1, 2: 2, 4: 4}
STATUS = {0: "GN_OK", 1: "GN_EINVAL", 2: "GN_ENOMEM", 3: "GN_ECUDA", 4: "GN_ESINGULAR",
          5: "GN_ENOCONV", 6: "GN_ENONFINITE", 7: "GN_ETIMEOUT"}
REPORT_MAX = 64

# exported symbols declared in include/gn.h
SYMBOLS = ("gn_system_create", "gn_system_destroy", "gn_system_set_arith", "gn_system_info",
           "gn_eval", "gn_lstsq", "gn_mgs", "gn_newton", "gn_batch_create", "gn_batch_destroy",
           "gn_batch_info", "gn_batch_newton", "gn_status_str", "gn_version", "gn_eval_noalloc",
           "gn_system_set_coef", "gn_adjoint", "gn_newton_mixed", "gn_set_wait_limit",
           "gn_batch_tuning")
# gn_arith: the faster per step (default), integer mantissas, or FP64
# error-free transformations
ARITH = {"auto": 0, "int": 1, "fp64": 2}
ADJ_REUSE = 1  # gn_adjoint flag: reuse the last factorisation


class GnError(RuntimeError):
    def __init__(self, status: int, what: str):
        name = STATUS.get(status, str(status))
        super().__init__(f"{what}: {name}")
        self.status = status


class Report(C.Structure):
    _fields_ = [("steps_done", C.c_int32), ("status", C.c_int32),
                ("res_norm", C.c_double * REPORT_MAX), ("dx_norm", C.c_double * REPORT_MAX)]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgn.so (built by ``paper_1402_2626_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1402_2626_gb300.build.build()")
        L = C.CDLL(path)
        vp, dp, i64p = C.c_void_p, C.c_double, C.POINTER(C.c_int64)
        L.gn_system_create.argtypes = [C.POINTER(vp), C.c_int32, C.c_int32, C.c_int64, i64p, i64p,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                                       C.POINTER(C.c_double), C.c_int32]
        L.gn_system_create.restype = C.c_int
        L.gn_system_destroy.argtypes = [vp]
        L.gn_system_destroy.restype = C.c_int
        L.gn_system_set_arith.argtypes = [vp, C.c_int]
        L.gn_system_set_arith.restype = C.c_int
        L.gn_system_info.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), i64p, i64p,
                                     C.POINTER(C.c_int32)]
        L.gn_system_info.restype = C.c_int
        L.gn_eval.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int64, vp]
        L.gn_eval.restype = C.c_int
        L.gn_eval_noalloc.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int64, vp]
        L.gn_eval_noalloc.restype = C.c_int
        L.gn_lstsq.argtypes = [vp, C.c_int, C.c_int32, C.c_int32, vp, C.c_int64, vp, vp, vp]
        L.gn_lstsq.restype = C.c_int
        L.gn_mgs.argtypes = [vp, C.c_int, C.c_int32, C.c_int32, vp, C.c_int64, vp, vp, vp]
        L.gn_mgs.restype = C.c_int
        L.gn_newton.argtypes = [vp, C.c_int, vp, C.c_int32, dp, C.POINTER(Report), vp]
        L.gn_newton.restype = C.c_int
        L.gn_system_set_coef.argtypes = [vp, vp, C.c_int32, vp]
        L.gn_system_set_coef.restype = C.c_int
        L.gn_adjoint.argtypes = [vp, C.c_int, vp, vp, vp, vp, C.c_int32, vp]
        L.gn_adjoint.restype = C.c_int
        L.gn_newton_mixed.argtypes = [vp, C.c_int, vp, C.c_int32, C.c_int32, dp, C.POINTER(Report), vp]
        L.gn_newton_mixed.restype = C.c_int
        L.gn_batch_create.argtypes = [C.POINTER(vp), C.c_int32, i64p, C.c_int64, i64p, i64p,
                                      C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                                      C.POINTER(C.c_double), C.c_int32]
        L.gn_batch_create.restype = C.c_int
        L.gn_batch_destroy.argtypes = [vp]
        L.gn_batch_destroy.restype = C.c_int
        L.gn_batch_info.argtypes = [vp, C.POINTER(C.c_int32), i64p, i64p, i64p, C.POINTER(C.c_int32)]
        L.gn_batch_info.restype = C.c_int
        L.gn_batch_newton.argtypes = [vp, C.c_int, vp, C.c_int32, vp, vp, vp]
        L.gn_batch_newton.restype = C.c_int
        L.gn_batch_tuning.argtypes = [vp, C.c_int] + [C.POINTER(C.c_int32)] * 5
        L.gn_batch_tuning.restype = C.c_int
        L.gn_set_wait_limit.argtypes = [C.c_int64, i64p]
        L.gn_set_wait_limit.restype = C.c_int
        L.gn_status_str.argtypes = [C.c_int]
        L.gn_status_str.restype = C.c_char_p
        L.gn_version.restype = C.c_int32
        _lib = L
        return L


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or t.dtype.is_complex or str(t.dtype) != "torch.float64" or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _check(st: int, what: str):
    if st != 0:
        raise GnError(st, what)


class System:
    """A polynomial system loaded into device memory (owns a gn_system)."""

    def __init__(self, system: inputs.System, coef_limbs: int = 4, arith: str = "auto"):
        L = load_library()
        self.N, self.n, self.T = system.N, system.n, system.T
        self._keep = [np.ascontiguousarray(system.poly_ptr, np.int64),
                      np.ascontiguousarray(system.mono_ptr, np.int64),
                      np.ascontiguousarray(system.var, np.int32),
                      np.ascontiguousarray(system.exp, np.uint8),
                      np.ascontiguousarray(system.coef[:, :, :coef_limbs], np.float64)]
        pp, mp, var, ex, cf = self._keep
        h = C.c_void_p()
        st = L.gn_system_create(C.byref(h), system.N, system.n, system.T,
                                pp.ctypes.data_as(C.POINTER(C.c_int64)),
                                mp.ctypes.data_as(C.POINTER(C.c_int64)),
                                var.ctypes.data_as(C.POINTER(C.c_int32)),
                                ex.ctypes.data_as(C.POINTER(C.c_uint8)),
                                cf.ctypes.data_as(C.POINTER(C.c_double)), coef_limbs)
        _check(st, "gn_system_create")
        self._h = h
        self._lib = L
        self.set_arith(arith)

    def set_arith(self, arith: str):
        """Arithmetic of evaluation and least squares: "auto", "int" or "fp64" (gn_arith)."""
        _check(self._lib.gn_system_set_arith(self._h, ARITH[arith]), "gn_system_set_arith")
        self.arith = arith

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gn_system_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        N, n, mx = C.c_int32(), C.c_int32(), C.c_int32()
        T, nnz = C.c_int64(), C.c_int64()
        _check(self._lib.gn_system_info(self._h, C.byref(N), C.byref(n), C.byref(T), C.byref(nnz),
                                        C.byref(mx)), "gn_system_info")
        return dict(N=N.value, n=n.value, T=T.value, nnz=nnz.value, max_support=mx.value)

    def eval(self, prec, x, f=None, J=None, stream=None):
        """f(x) into f [N,2,L] and J into J [n,N,2,L] (column-major), in place."""
        ldJ = self.N if J is None else J.shape[1]
        _check(self._lib.gn_eval(self._h, PREC[prec], _ptr(x), _ptr(f), _ptr(J), ldJ,
                                 _stream(stream)), "gn_eval")

    def eval_noalloc(self, prec, x, f=None, J=None, stream=None):
        """As eval(), through gn_eval_noalloc: no device allocation in the call."""
        ldJ = self.N if J is None else J.shape[1]
        _check(self._lib.gn_eval_noalloc(self._h, PREC[prec], _ptr(x), _ptr(f), _ptr(J), ldJ,
                                         _stream(stream)), "gn_eval_noalloc")

    def lstsq(self, prec, Ab, R, dx, stream=None):
        """MGS least squares on Ab [n+1, m, 2, L] in place; R and dx are outputs."""
        ncols, m = Ab.shape[0], Ab.shape[1]
        _check(self._lib.gn_lstsq(self._h, PREC[prec], m, ncols - 1, _ptr(Ab), m, _ptr(R), _ptr(dx),
                                  _stream(stream)), "gn_lstsq")

    def mgs(self, prec, Ab, R, status, stream=None):
        """MGS factorisation of Ab [n+1, m, 2, L] in place (no back substitution,
        no synchronisation); R is an output and status a 1-element int32 CUDA
        tensor that receives the device status."""
        ncols, m = Ab.shape[0], Ab.shape[1]
        if not status.is_cuda or str(status.dtype) != "torch.int32":
            raise ValueError("status must be an int32 CUDA tensor")
        _check(self._lib.gn_mgs(self._h, PREC[prec], m, ncols - 1, _ptr(Ab), m, _ptr(R),
                                C.c_void_p(status.data_ptr()), _stream(stream)), "gn_mgs")

    def set_coef(self, coef, stream=None):
        """Replace the coefficients from a CUDA tensor [T,2,Lc] (Lc = 1, 2 or 4)."""
        if coef.dim() != 3 or coef.shape[0] != self.T or coef.shape[1] != 2:
            raise ValueError("coef must have shape [T, 2, limbs]")
        _check(self._lib.gn_system_set_coef(self._h, _ptr(coef), coef.shape[2], _stream(stream)),
               "gn_system_set_coef")

    def adjoint(self, prec, x, g, grad, lam=None, reuse=False, stream=None):
        """Coefficient gradient at the root x [n,2,L] for the loss gradient
        g [n,2,L]: grad [T,2,L] (and lam [N,2,L] if given) are written;
        ``reuse`` takes the factorisation the last newton() or adjoint() left
        (GN_ADJ_REUSE) instead of factoring J at x; synchronizes the stream."""
        _check(self._lib.gn_adjoint(self._h, PREC[prec], _ptr(x), _ptr(g), _ptr(grad), _ptr(lam),
                                    ADJ_REUSE if reuse else 0, _stream(stream)), "gn_adjoint")

    def newton(self, prec, x, steps, tol=0.0, stream=None, raise_on_error=True):
        """``steps`` Gauss-Newton steps in place on x [n,2,L]; returns the report."""
        rep = Report()
        st = self._lib.gn_newton(self._h, PREC[prec], _ptr(x), steps, float(tol), C.byref(rep),
                                 _stream(stream))
        out = dict(status=st, steps_done=rep.steps_done,
                   res_norm=list(rep.res_norm[: rep.steps_done]),
                   dx_norm=list(rep.dx_norm[: rep.steps_done]))
        if raise_on_error and st != 0:
            raise GnError(st, "gn_newton")
        return out


    def newton_mixed(self, prec, x, d_steps, refine_steps, tol=0.0, stream=None,
                     raise_on_error=True):
        """Mixed-precision Gauss-Newton in place on x [n,2,L] (L = 2 or 4):
        ``d_steps`` double-precision steps, then ``refine_steps`` refinement
        steps with that factorisation and residuals at precision L."""
        rep = Report()
        st = self._lib.gn_newton_mixed(self._h, PREC[prec], _ptr(x), d_steps, refine_steps,
                                       float(tol), C.byref(rep), _stream(stream))
        out = dict(status=st, steps_done=rep.steps_done,
                   res_norm=list(rep.res_norm[: rep.steps_done]),
                   dx_norm=list(rep.dx_norm[: rep.steps_done]))
        if raise_on_error and st != 0:
            raise GnError(st, "gn_newton_mixed")
        return out


class Batch:
    """Independent square systems advanced together (owns a gn_batch)."""

    def __init__(self, batch: inputs.Batch, coef_limbs: int = 4):
        L = load_library()
        self.S, self.X = batch.S, int(batch.sys_var[-1])
        self._keep = [np.ascontiguousarray(np.diff(batch.sys_var), np.int64),
                      np.ascontiguousarray(batch.poly_ptr, np.int64),
                      np.ascontiguousarray(batch.mono_ptr, np.int64),
                      np.ascontiguousarray(batch.var, np.int32),
                      np.ascontiguousarray(batch.exp, np.uint8),
                      np.ascontiguousarray(batch.coef[:, :, :coef_limbs], np.float64)]
        ns, pp, mp, var, ex, cf = self._keep
        h = C.c_void_p()
        st = L.gn_batch_create(C.byref(h), batch.S, ns.ctypes.data_as(C.POINTER(C.c_int64)), batch.T,
                               pp.ctypes.data_as(C.POINTER(C.c_int64)),
                               mp.ctypes.data_as(C.POINTER(C.c_int64)),
                               var.ctypes.data_as(C.POINTER(C.c_int32)),
                               ex.ctypes.data_as(C.POINTER(C.c_uint8)),
                               cf.ctypes.data_as(C.POINTER(C.c_double)), coef_limbs)
        _check(st, "gn_batch_create")
        self._keep = None  # the library copied what it needs
        self._h = h
        self._lib = L

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        S, mx = C.c_int32(), C.c_int32()
        X, T, nnz = C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._lib.gn_batch_info(self._h, C.byref(S), C.byref(X), C.byref(T), C.byref(nnz),
                                       C.byref(mx)), "gn_batch_info")
        return dict(S=S.value, X=X.value, T=T.value, nnz=nnz.value, max_n=mx.value)

    def tuning(self, prec):
        """The launch choices of the first newton() call at ``prec`` (gn_batch_tuning)."""
        v = [C.c_int32() for _ in range(5)]
        _check(self._lib.gn_batch_tuning(self._h, PREC[prec], *[C.byref(q) for q in v]),
               "gn_batch_tuning")
        return dict(eval_block=v[0].value, eval_lanes=v[1].value, solve_threads=v[2].value,
                    solve_grid=v[3].value, largest_first=bool(v[4].value))

    def newton(self, prec, x, steps, status, norms=None, stream=None):
        """``steps`` Gauss-Newton steps on every system, in place on x [X,2,L];
        status [S] int32 (GN_OK on entry) and norms [steps,S,2] float64 are
        CUDA tensors the call writes; stream-ordered, no synchronisation."""
        if not status.is_cuda or str(status.dtype) != "torch.int32":
            raise ValueError("status must be an int32 CUDA tensor")
        _check(self._lib.gn_batch_newton(self._h, PREC[prec], _ptr(x), steps, _ptr(norms),
                                         C.c_void_p(status.data_ptr()), _stream(stream)),
               "gn_batch_newton")


def set_wait_limit(cycles: int) -> int:
    """Bound of one device-side wait of the MGS kernel in SM clock cycles on
    the current device (0 restores the default); returns the previous bound
    (gn_set_wait_limit)."""
    L = load_library()
    prev = C.c_int64()
    _check(L.gn_set_wait_limit(int(cycles), C.byref(prev)), "gn_set_wait_limit")
    return prev.value


_root_fn = None


def _root_function():
    global _root_fn
    if _root_fn is None:
        import torch

        class NewtonRoot(torch.autograd.Function):
            """x = root of the system with coefficients ``coef`` reached by
            ``steps`` Gauss-Newton steps from x0 (gn_newton); the backward pass
            is gn_adjoint at that root."""

            @staticmethod
            def forward(ctx, coef, system, prec, x0, steps):
                system.set_coef(coef)
                x = x0.detach().clone().contiguous()
                system.newton(prec, x, steps)
                ctx.save_for_backward(coef, x)
                ctx.system, ctx.prec = system, prec
                return x

            @staticmethod
            def backward(ctx, gx):
                coef, x = ctx.saved_tensors
                system, prec = ctx.system, ctx.prec
                system.set_coef(coef)  # the system may hold other coefficients by now
                # first order, a change of the root shows in its leading limb
                g = torch.zeros_like(x)
                g[..., 0] = gx[..., 0]
                grad = torch.empty((system.T, 2, PREC[prec]), dtype=torch.float64, device=x.device)
                system.adjoint(prec, x, g, grad)
                # a coefficient's value is the sum of its limbs: each limb gets dL/dc
                gc = grad[..., :1].expand(-1, -1, coef.shape[2]).contiguous()
                return gc, None, None, None, None

        _root_fn = NewtonRoot
    return _root_fn


def newton_root(system: System, prec, coef, x0, steps: int):
    """Differentiable root: ``steps`` Gauss-Newton steps from x0 [n,2,L] on
    ``system`` with its coefficients replaced by coef [T,2,Lc] (a CUDA
    tensor that may require grad).  Backward gives dL/dcoef by the adjoint
    (gn_adjoint); the loss gradient is taken from the leading limb of x, and
    every limb of a coefficient receives the coefficient's gradient."""
    return _root_function().apply(coef, system, prec, x0, steps)
