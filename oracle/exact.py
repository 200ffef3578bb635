"""Exact optimal values for tiny grids (test infrastructure only, see ``oracle/__init__``).

* ``ot_exact_mcf``     -- the full OT problem eq. (1) by our own successive-
                          shortest-path min-cost flow (``mcf.c``, plain C).
* ``ot_exact_lp``      -- eq. (1) as an LP, solved by SciPy's HiGHS (a library
                          primitive used as an independent check of the above).
* ``reduced_exact_lp`` -- the reduced model eq. (3) / (8) by HiGHS; by the
                          equivalence the paper cites (Auricchio et al., Thm 1)
                          its optimum equals that of eq. (1).
"""
import ctypes
import os
import subprocess
import numpy as np

from .reduced_model import build_A, build_b, build_c, full_cost_matrix, vec

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build_mcf(force=False):
    """Compile mcf.c into oracle/_build/libotmcf.so with the host gcc."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libotmcf.so")
    src = os.path.join(_HERE, "mcf.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_mcf())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.ot_mcf_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double,
                                     dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.ot_mcf_solve.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def transport_mcf(C, a, b, eps=1e-15, want_flow=False):
    """min <C, F> over F >= 0 with row sums a and column sums b (Σa = Σb)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    ns, nt = C.shape
    dp = ctypes.POINTER(ctypes.c_double)
    val = ctypes.c_double()
    its = ctypes.c_int()
    F = np.zeros((ns, nt)) if want_flow else None
    rc = _lib().ot_mcf_solve(ns, nt, C.ctypes.data_as(dp), a.ctypes.data_as(dp), b.ctypes.data_as(dp),
                             eps, F.ctypes.data_as(dp) if want_flow else None, ctypes.byref(val),
                             ctypes.byref(its))
    if rc != 0:
        raise RuntimeError("ot_mcf_solve failed with status %d" % rc)
    return (val.value, F) if want_flow else val.value


def ot_exact_mcf(mu1, mu2, xs=None, ys=None, want_plan=False):
    """Exact optimum of eq. (1) by min-cost flow; the plan is indexed by vec positions."""
    m, n = np.shape(mu1)
    C = full_cost_matrix(m, n, xs, ys)
    return transport_mcf(C, vec(mu1), vec(mu2), want_flow=want_plan)


def ot_exact_lp(mu1, mu2, xs=None, ys=None):
    """Exact optimum of eq. (1) by HiGHS."""
    import scipy.sparse as sp
    from scipy.optimize import linprog
    m, n = np.shape(mu1)
    M = m * n
    C = full_cost_matrix(m, n, xs, ys)
    # pi flattened row-major over (source s, target t): row sums over t, column sums over s
    rows = sp.kron(sp.identity(M), np.ones((1, M)))
    cols = sp.kron(np.ones((1, M)), sp.identity(M))
    Aeq = sp.vstack([rows, cols]).tocsr()
    beq = np.concatenate([vec(mu1), vec(mu2)])
    res = linprog(C.reshape(-1), A_eq=Aeq, b_eq=beq, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    return float(res.fun)


def reduced_exact_lp(mu1, mu2, xs=None, ys=None, want_x=False):
    """Exact optimum of the reduced model (eq. 8 form) by HiGHS."""
    from scipy.optimize import linprog
    m, n = np.shape(mu1)
    A = build_A(m, n)
    b = build_b(mu1, mu2)
    c = build_c(m, n, xs, ys)
    res = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    return (float(res.fun), res.x) if want_x else float(res.fun)
