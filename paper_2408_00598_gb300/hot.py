"""Python binding of libhot (include/hot.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts numpy
arrays / torch tensors into pointers and C structs.  It raises ``HotError``
when the library is missing or a call fails -- there is no fallback.

The functions keep the C names (``hot_create``, ``hot_solve``,
``hot_recover_plan``, ``hot_submit``, ``hot_poll``, ...); ``Context`` wraps
them for convenience.  Histograms are row-major (m, n) float64 arrays (numpy
on the host, or torch CUDA tensors on the context's device).

Example::

    from paper_2408_00598_gb300 import hot
    with hot.Context(precision="fp32") as ctx:        # or "fp64"
        r = ctx.solve(mu, nu, tol=1e-6)                 # mu, nu: (m, n), each summing to 1
        src, dst, mass, l1 = ctx.recover_plan(r)        # entries src = i*n + j -> dst = k*n + l
        ctx.release(r)
    # r["ot_value"], r["dual_value"], r["rel_kkt"], r["iters"], ...
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhot.so")

HOT_OK = 0
HOT_PENDING = 1
HOT_NOT_CONVERGED = 2
HOT_EINVAL = -1
HOT_ENOMEM = -2
HOT_NUMERIC = -3
HOT_TIMEOUT = -4
HOT_ECUDA = -5
HOT_ENOTFOUND = -6
HOT_ECANCELLED = -7
HOT_EBUSY = -8

HOT_FP32_BULK = 0
HOT_FP64 = 1
HOT_SPACE_HOST = 0
HOT_SPACE_DEVICE = 1
HOT_METHOD_HALPERN = 0
HOT_METHOD_GADMM = 1
HOT_STOP_RELATIVE = 0
HOT_STOP_ABSOLUTE = 1


class HotError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


_STATUS = {v: k for k, v in dict(HOT_OK=0, HOT_PENDING=1, HOT_NOT_CONVERGED=2, HOT_EINVAL=-1, HOT_ENOMEM=-2,
                                  HOT_NUMERIC=-3, HOT_TIMEOUT=-4, HOT_ECUDA=-5, HOT_ENOTFOUND=-6,
                                  HOT_ECANCELLED=-7, HOT_EBUSY=-8).items()}


class hot_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("check_every", ctypes.c_int), ("sigma0", ctypes.c_double),
                ("restart_sufficient", ctypes.c_double), ("restart_necessary", ctypes.c_double),
                ("restart_long", ctypes.c_double), ("mem_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("autotune_cache", ctypes.c_char_p),
                ("keep_batch_solutions", ctypes.c_int), ("method", ctypes.c_int), ("relaxation", ctypes.c_double),
                ("stop_rule", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class hot_result(ctypes.Structure):
    _fields_ = [("ot_value", ctypes.c_double), ("dual_value", ctypes.c_double), ("rel_kkt", ctypes.c_double),
                ("rel_dual", ctypes.c_double), ("rel_comp", ctypes.c_double), ("rel_primal", ctypes.c_double),
                ("sigma", ctypes.c_double), ("cost_scale", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("iters", ctypes.c_longlong), ("restarts", ctypes.c_int),
                ("status", ctypes.c_int), ("solution_id", ctypes.c_ulonglong), ("max_abs_dual", ctypes.c_float),
                ("m", ctypes.c_int), ("n", ctypes.c_int), ("kernel_launches", ctypes.c_longlong),
                ("blocks", ctypes.c_longlong), ("abs_kkt", ctypes.c_double)]

    def to_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class hot_kernel_times(ctypes.Structure):
    _fields_ = [("sweep_ms", ctypes.c_double), ("sweep_launches", ctypes.c_longlong),
                ("sweep_check_ms", ctypes.c_double), ("sweep_check_launches", ctypes.c_longlong),
                ("solve_ms", ctypes.c_double), ("solve_launches", ctypes.c_longlong),
                ("block_end_ms", ctypes.c_double), ("block_end_launches", ctypes.c_longlong),
                ("sweep_bytes", ctypes.c_double)]

    def to_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class hot_request(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("nu", ctypes.c_void_p), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_longlong), ("keep_solution", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


class hot_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("cancelled", ctypes.c_longlong), ("rejected", ctypes.c_longlong), ("queued", ctypes.c_int),
                ("running", ctypes.c_int), ("device_bytes_in_use", ctypes.c_size_t), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_queue_ms", ctypes.c_double), ("blocks_run", ctypes.c_longlong)]

    def to_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_LIB = None


def load_library(path=None):
    """Load libhot.so (built in-tree by ``paper_2408_00598_gb300.build``)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise HotError(HOT_ECUDA, "libhot.so not found at %s; build it with "
                                  "`python -m paper_2408_00598_gb300.build`" % p)
    lib = ctypes.CDLL(p)
    P = ctypes.POINTER
    vp, i, d, ll, ull, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                             ctypes.c_ulonglong, ctypes.c_size_t)
    sig = {
        "hot_config_default": (None, [P(hot_config)]),
        "hot_create": (i, [P(vp), P(hot_config)]),
        "hot_destroy": (None, [vp]),
        "hot_status_string": (ctypes.c_char_p, [i]),
        "hot_last_error": (ctypes.c_char_p, [vp]),
        "hot_solve": (i, [vp, vp, vp, i, i, i, d, ll, P(hot_result)]),
        "hot_solve_batch": (i, [vp, i, P(vp), P(vp), P(i), P(i), i, d, ll, P(hot_result)]),
        "hot_solve_coords": (i, [vp, vp, vp, i, i, i, vp, vp, d, ll, P(hot_result)]),
        "hot_solve_profiled": (i, [vp, vp, vp, i, i, i, d, ll, P(hot_result), P(hot_kernel_times)]),
        "hot_sweep_timing": (i, [vp, i, P(d), P(ll), P(d)]),
        "hot_get_flows": (i, [vp, ull, vp, i]),
        "hot_recover_plan": (i, [vp, ull, vp, vp, vp, i, sz, P(sz), P(d)]),
        "hot_release": (i, [vp, ull]),
        "hot_submit": (i, [vp, P(hot_request), P(ull)]),
        "hot_poll": (i, [vp, ull, P(hot_result)]),
        "hot_wait": (i, [vp, ull, d, P(hot_result)]),
        "hot_cancel": (i, [vp, ull]),
        "hot_forget": (i, [vp, ull]),
        "hot_serve_stats_get": (i, [vp, P(hot_serve_stats)]),
        "hot_barycentric_map": (i, [vp, vp, vp, sz, vp, i, i, vp, vp, i, vp]),
        "hot_autotune": (i, [vp, i, P(i), P(d)]),
        "hot_autotune_cache_lookup": (i, [ctypes.c_char_p, ctypes.c_char_p, i, i, P(i), P(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def _err(lib, ctx, rc):
    msg = lib.hot_last_error(ctx)
    return HotError(rc, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, space, keep-alive) for a numpy array or torch tensor of float64."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.dtype.__repr__() != "torch.float64":
            raise HotError(HOT_EINVAL, "tensors must be float64")
        t = a.contiguous()
        return t.data_ptr(), (HOT_SPACE_DEVICE if t.is_cuda else HOT_SPACE_HOST), t
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr.ctypes.data, HOT_SPACE_HOST, arr


def _grid(mu, nu):
    """(m, n) of a histogram pair; both must be 2-D arrays of the same shape."""
    if len(mu.shape) != 2 or tuple(nu.shape) != tuple(mu.shape):
        raise HotError(HOT_EINVAL, "mu and nu must be 2-D arrays of the same shape, got %s and %s"
                       % (tuple(mu.shape), tuple(nu.shape)))
    return int(mu.shape[0]), int(mu.shape[1])


# ----------------------------------------------------------- C-named calls --

def hot_config_default():
    cfg = hot_config()
    load_library().hot_config_default(ctypes.byref(cfg))
    return cfg



def hot_barycentric_map(src, dst, mass, y, nsrc, out=None, weight=None, stream=None):
    """Barycentric projection of a plan (device tensors): out[s] = sum pi y[t] / sum pi,
    weight[s] = sum pi.  src/dst int32, mass float64 (nnz each), y float64 (ndst, D)."""
    import torch
    lib = load_library()
    if not (src.is_cuda and dst.is_cuda and mass.is_cuda and y.is_cuda):
        raise HotError(HOT_EINVAL, "hot_barycentric_map takes device tensors")
    if src.dtype != torch.int32 or dst.dtype != torch.int32 or mass.dtype != torch.float64 or y.dtype != torch.float64:
        raise HotError(HOT_EINVAL, "src/dst must be int32 and mass/y float64")
    y2 = y.reshape(y.shape[0], -1).contiguous()
    D = y2.shape[1]
    if out is None:
        out = torch.empty((nsrc, D), dtype=torch.float64, device=y.device)
    if weight is None:
        weight = torch.empty(nsrc, dtype=torch.float64, device=y.device)
    s, t, m = src.contiguous(), dst.contiguous(), mass.contiguous()
    rc = lib.hot_barycentric_map(s.data_ptr(), t.data_ptr(), m.data_ptr(), s.numel(), y2.data_ptr(), y2.shape[0], D,
                                 out.data_ptr(), weight.data_ptr(), nsrc,
                                 ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream))
    if rc != HOT_OK:
        raise _err(lib, None, rc)
    return out, weight


def hot_autotune_cache_lookup(path, device, precision, S):
    """(TR, microseconds per iteration) of an autotune cache entry, or None."""
    lib = load_library()
    tr = ctypes.c_int()
    us = ctypes.c_double()
    rc = lib.hot_autotune_cache_lookup(path.encode(), device.encode(), precision, S, ctypes.byref(tr), ctypes.byref(us))
    if rc == HOT_ENOTFOUND:
        return None
    if rc != HOT_OK:
        raise _err(lib, None, rc)
    return tr.value, us.value

def hot_create(cfg=None):
    lib = load_library()
    c = cfg if cfg is not None else hot_config_default()
    h = ctypes.c_void_p()
    rc = lib.hot_create(ctypes.byref(h), ctypes.byref(c))
    if rc != HOT_OK:
        raise _err(lib, None, rc)
    return h


def hot_destroy(ctx):
    load_library().hot_destroy(ctx)


def hot_status_string(status):
    return load_library().hot_status_string(status).decode()


def hot_solve(ctx, mu, nu, tol=1e-6, max_iter=100000):
    lib = load_library()
    pm, sm, km = _ptr(mu)
    pn, sn, kn = _ptr(nu)
    if sm != sn:
        raise HotError(HOT_EINVAL, "mu and nu must live in the same space")
    m, n = _grid(mu, nu)
    res = hot_result()
    rc = lib.hot_solve(ctx, pm, pn, m, n, sm, float(tol), int(max_iter), ctypes.byref(res))
    if rc not in (HOT_OK, HOT_NOT_CONVERGED):
        raise _err(lib, ctx, rc)
    return res.to_dict()


def hot_solve_coords(ctx, mu, nu, xs, ys, tol=1e-6, max_iter=100000):
    """hot_solve with bin coordinates xs (rows, m values) and ys (columns, n values)."""
    lib = load_library()
    pm, sm, km = _ptr(mu)
    pn, sn, kn = _ptr(nu)
    if sm != sn:
        raise HotError(HOT_EINVAL, "mu and nu must live in the same space")
    m, n = _grid(mu, nu)
    ax = np.ascontiguousarray(xs, dtype=np.float64)
    ay = np.ascontiguousarray(ys, dtype=np.float64)
    if ax.shape != (m,) or ay.shape != (n,):
        raise HotError(HOT_EINVAL, "xs must have m entries and ys n entries")
    res = hot_result()
    rc = lib.hot_solve_coords(ctx, pm, pn, m, n, sm, ax.ctypes.data, ay.ctypes.data, float(tol), int(max_iter),
                              ctypes.byref(res))
    if rc not in (HOT_OK, HOT_NOT_CONVERGED):
        raise _err(lib, ctx, rc)
    return res.to_dict()


def hot_solve_profiled(ctx, mu, nu, tol=1e-6, max_iter=100000):
    """hot_solve with per-kernel-family CUDA-event timings: (result, times)."""
    lib = load_library()
    pm, sm, km = _ptr(mu)
    pn, sn, kn = _ptr(nu)
    m, n = _grid(mu, nu)
    res = hot_result()
    kt = hot_kernel_times()
    rc = lib.hot_solve_profiled(ctx, pm, pn, m, n, sm, float(tol), int(max_iter), ctypes.byref(res),
                                ctypes.byref(kt))
    if rc not in (HOT_OK, HOT_NOT_CONVERGED):
        raise _err(lib, ctx, rc)
    return res.to_dict(), kt.to_dict()


def hot_sweep_timing(ctx, enable):
    """Switch the live in-graph sweep timing on (1), off (0) or leave it (-1);
    returns the counters since the last call: {"ms", "launches", "bytes"}."""
    lib = load_library()
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    b = ctypes.c_double()
    rc = lib.hot_sweep_timing(ctx, int(enable), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b))
    if rc != HOT_OK:
        raise _err(lib, ctx, rc)
    return {"ms": ms.value, "launches": n.value, "bytes": b.value}


def hot_solve_batch(ctx, mus, nus, tol=1e-6, max_iter=100000):
    lib = load_library()
    keep = []
    pm = (ctypes.c_void_p * len(mus))()
    pn = (ctypes.c_void_p * len(mus))()
    ms = (ctypes.c_int * len(mus))()
    ns = (ctypes.c_int * len(mus))()
    space = None
    for q, (a, b) in enumerate(zip(mus, nus)):
        p1, s1, k1 = _ptr(a)
        p2, s2, k2 = _ptr(b)
        keep += [k1, k2]
        if space is None:
            space = s1
        if s1 != space or s2 != space:
            raise HotError(HOT_EINVAL, "all histograms must live in the same space")
        pm[q], pn[q] = p1, p2
        ms[q], ns[q] = _grid(a, b)
    out = (hot_result * len(mus))()
    rc = lib.hot_solve_batch(ctx, len(mus), pm, pn, ms, ns, space or 0, float(tol), int(max_iter), out)
    if rc != HOT_OK:
        raise _err(lib, ctx, rc)
    return [r.to_dict() for r in out]


def hot_get_flows(ctx, solution_id, m, n, out=None):
    """x-bar in the paper's vec order (eq. 4-6); numpy by default, or into a
    float64 torch CUDA tensor ``out``."""
    lib = load_library()
    V = m * m * n + m * n * n
    if out is None:
        x = np.empty(V)
        rc = lib.hot_get_flows(ctx, solution_id, x.ctypes.data, HOT_SPACE_HOST)
    else:
        x = out
        rc = lib.hot_get_flows(ctx, solution_id, out.data_ptr(), HOT_SPACE_DEVICE)
    if rc != HOT_OK:
        raise _err(lib, ctx, rc)
    return x


def hot_recover_plan(ctx, solution_id, out=None):
    """Algorithm 1 on the device.

    * ``out=None``: returns (src, dst, mass, marg_l1) as numpy arrays;
    * ``out=()``: only counts, returns (nnz, marg_l1);
    * ``out=(src, dst, mass)``: int32 / int32 / float64 arrays (torch CUDA
      tensors, pinned or plain host tensors, or numpy arrays) with room for the
      plan; returns (nnz, marg_l1).
    """
    lib = load_library()
    nnz = ctypes.c_size_t()
    l1 = (ctypes.c_double * 2)()
    if out is None or len(out) == 0:
        rc = lib.hot_recover_plan(ctx, solution_id, None, None, None, HOT_SPACE_HOST, 0, ctypes.byref(nnz), l1)
        if rc != HOT_OK:
            raise _err(lib, ctx, rc)
        if out is not None:
            return nnz.value, (l1[0], l1[1])
        n = nnz.value
        src = np.empty(max(n, 1), dtype=np.int32)
        dst = np.empty(max(n, 1), dtype=np.int32)
        mass = np.empty(max(n, 1), dtype=np.float64)
        rc = lib.hot_recover_plan(ctx, solution_id, src.ctypes.data, dst.ctypes.data, mass.ctypes.data,
                                  HOT_SPACE_HOST, max(n, 1), ctypes.byref(nnz), l1)
        if rc != HOT_OK:
            raise _err(lib, ctx, rc)
        return src[:n], dst[:n], mass[:n], (l1[0], l1[1])
    s, d, m = out

    def addr(a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr(), (HOT_SPACE_DEVICE if a.is_cuda else HOT_SPACE_HOST), a.numel()
        return a.ctypes.data, HOT_SPACE_HOST, a.size
    (ps, sp, ns), (pd, _, nd), (pm, _, nm) = addr(s), addr(d), addr(m)
    rc = lib.hot_recover_plan(ctx, solution_id, ps, pd, pm, sp, min(ns, nd, nm), ctypes.byref(nnz), l1)
    if rc != HOT_OK:
        raise _err(lib, ctx, rc)
    return nnz.value, (l1[0], l1[1])


def hot_release(ctx, solution_id):
    lib = load_library()
    rc = lib.hot_release(ctx, solution_id)
    if rc != HOT_OK:
        raise _err(lib, ctx, rc)


def hot_submit(ctx, mu, nu, tol=1e-6, max_iter=100000, keep_solution=False):
    lib = load_library()
    a = np.ascontiguousarray(mu, dtype=np.float64)
    b = np.ascontiguousarray(nu, dtype=np.float64)
    _grid(a, b)
    req = hot_request(a.ctypes.data, b.ctypes.data, a.shape[0], a.shape[1], float(tol), int(max_iter),
                      1 if keep_solution else 0)
    t = ctypes.c_ulonglong()
    rc = lib.hot_submit(ctx, ctypes.byref(req), ctypes.byref(t))
    if rc != HOT_OK:
        raise _err(lib, ctx, rc)
    return t.value


def hot_poll(ctx, ticket):
    """(status, result dict or None); status HOT_PENDING while not finished."""
    lib = load_library()
    r = hot_result()
    rc = lib.hot_poll(ctx, ticket, ctypes.byref(r))
    if rc == HOT_PENDING:
        return rc, None
    if rc == HOT_ENOTFOUND:
        raise _err(lib, ctx, rc)
    return rc, r.to_dict()


def hot_wait(ctx, ticket, timeout_ms=-1.0):
    lib = load_library()
    r = hot_result()
    rc = lib.hot_wait(ctx, ticket, float(timeout_ms), ctypes.byref(r))
    if rc in (HOT_TIMEOUT, HOT_PENDING):
        return rc, None
    if rc == HOT_ENOTFOUND:
        raise _err(lib, ctx, rc)
    return rc, r.to_dict()


def hot_cancel(ctx, ticket):
    return load_library().hot_cancel(ctx, ticket)


def hot_forget(ctx, ticket):
    return load_library().hot_forget(ctx, ticket)


def hot_serve_stats_get(ctx):
    lib = load_library()
    s = hot_serve_stats()
    rc = lib.hot_serve_stats_get(ctx, ctypes.byref(s))
    if rc != HOT_OK:
        raise _err(lib, ctx, rc)
    return s.to_dict()


class Context:
    """Owns one hot_ctx.  ``precision``: "fp32" (FP32 bulk) or "fp64";
    ``method``: "hot" (Algorithm 2) or "gadmm" (generalized ADMM, ``relaxation``
    rho); ``stop``: "relative" (eq. kkt_res) or "absolute" (Table VI)."""

    def __init__(self, device=0, precision="fp32", stream=None, method="hot", stop="relative", **kw):
        cfg = hot_config_default()
        cfg.device = device
        cfg.precision = HOT_FP64 if precision == "fp64" else HOT_FP32_BULK
        if method not in ("hot", "gadmm") or stop not in ("relative", "absolute"):
            raise ValueError("method must be 'hot' or 'gadmm', stop 'relative' or 'absolute'")
        cfg.method = HOT_METHOD_GADMM if method == "gadmm" else HOT_METHOD_HALPERN
        cfg.stop_rule = HOT_STOP_ABSOLUTE if stop == "absolute" else HOT_STOP_RELATIVE
        if stream is not None:
            cfg.stream = ctypes.c_void_p(stream)
        for k, v in kw.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.ctx = hot_create(cfg)

    def close(self):
        if self.ctx:
            hot_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, S):
        """Time the candidate tile heights for S x S and keep the fastest: (TR, us per iteration)."""
        lib = load_library()
        tr = ctypes.c_int()
        us = ctypes.c_double()
        rc = lib.hot_autotune(self.ctx, S, ctypes.byref(tr), ctypes.byref(us))
        if rc != HOT_OK:
            raise _err(lib, self.ctx, rc)
        return tr.value, us.value

    def solve(self, mu, nu, tol=1e-6, max_iter=100000, xs=None, ys=None):
        if xs is not None or ys is not None:
            return hot_solve_coords(self.ctx, mu, nu, xs, ys, tol, max_iter)
        return hot_solve(self.ctx, mu, nu, tol, max_iter)

    def solve_profiled(self, mu, nu, tol=1e-6, max_iter=100000):
        return hot_solve_profiled(self.ctx, mu, nu, tol, max_iter)

    def solve_batch(self, mus, nus, tol=1e-6, max_iter=100000):
        return hot_solve_batch(self.ctx, mus, nus, tol, max_iter)

    def sweep_timing(self, enable=-1):
        return hot_sweep_timing(self.ctx, enable)

    def flows(self, res, out=None):
        return hot_get_flows(self.ctx, res["solution_id"], res["m"], res["n"], out)

    def recover_plan(self, res, device_out=None):
        return hot_recover_plan(self.ctx, res["solution_id"], device_out)

    def recover_plan_host(self, res, src, dst, mass):
        return hot_recover_plan(self.ctx, res["solution_id"], (src, dst, mass))

    def release(self, res):
        hot_release(self.ctx, res["solution_id"])

    def submit(self, mu, nu, tol=1e-6, max_iter=100000, keep_solution=False):
        return hot_submit(self.ctx, mu, nu, tol, max_iter, keep_solution)

    def poll(self, ticket):
        return hot_poll(self.ctx, ticket)

    def wait(self, ticket, timeout_ms=-1.0):
        return hot_wait(self.ctx, ticket, timeout_ms)

    def cancel(self, ticket):
        return hot_cancel(self.ctx, ticket)

    def forget(self, ticket):
        return hot_forget(self.ctx, ticket)

    def serve_stats(self):
        return hot_serve_stats_get(self.ctx)
