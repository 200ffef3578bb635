"""hot_recover_plan_static: Algorithm 1 without any device allocation.

Callers that cannot let a library allocate device memory at call time (a
fixed, pre-accounted device footprint, or a latency-critical loop that must
not synchronise on an allocation) use this entry point; its scratch is a
static device array inside the library.  The tests call it through the C ABI
twice in a row, on the same flows, and check each result against the plan of
the allocating entry point hot_recover_plan and, entry by entry, against the
oracle's literal loops of Algorithm 1 on the same flows.  They run alone or
after the other tests (the static array keeps the previous call's contents,
which the entry point must not depend on).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bind(lib):
    f = lib.hot_recover_plan_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    return f


def _dense(src, dst, mass, M):
    P = np.zeros((M, M))
    np.add.at(P, (np.asarray(src, dtype=np.int64), np.asarray(dst, dtype=np.int64)), mass)
    return P


# shapes pairs have bins of zero mass: empty sources and sinks at many nodes
@pytest.mark.parametrize("kind,precision", [("gauss", "fp64"), ("shapes", "fp64"), ("shapes", "fp32")])
def test_static_recovery_matches_allocating_recovery_and_oracle_twice(kind, precision):
    import torch
    from oracle import recover as orec
    from paper_2408_00598_gb300 import hot
    from paper_2408_00598_gb300 import synthetic as syn

    lib = hot.load_library()
    fn = _bind(lib)
    S = 48
    mu1, mu2 = syn.make_pair(kind, S, 2)
    with hot.Context(precision=precision) as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-8)
        src, dst, mass, l1 = ctx.recover_plan(r)
        x = torch.empty(2 * S ** 3, dtype=torch.float64, device="cuda")
        ctx.flows(r, out=x)
        ctx.release(r)
    d_mu = torch.from_numpy(mu1).cuda()
    d_nu = torch.from_numpy(mu2).cuda()
    cap = S * S * (2 * S - 1)
    o_src = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    o_dst = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    o_mass = torch.full((cap,), -1.0, dtype=torch.float64, device="cuda")
    # the oracle's literal Algorithm 1 on the same (clipped) flows
    ent = orec.recover_from_x(x.cpu().numpy(), S, S)
    Po = _dense([i * S + j for i, j, k, l, p in ent], [k * S + l for i, j, k, l, p in ent],
                [p for i, j, k, l, p in ent], S * S)
    Pg = _dense(src, dst, mass, S * S)
    torch.cuda.synchronize()
    for call in range(2):
        nnz = ctypes.c_size_t()
        l1s = (ctypes.c_double * 2)()
        rc = fn(x.data_ptr(), S, S, d_mu.data_ptr(), d_nu.data_ptr(), o_src.data_ptr(), o_dst.data_ptr(),
                o_mass.data_ptr(), cap, ctypes.byref(nnz), l1s, None)
        assert rc == hot.HOT_OK, lib.hot_last_error(None)
        n = nnz.value
        hs, hd, hm = o_src[:n].cpu().numpy(), o_dst[:n].cpu().numpy(), o_mass[:n].cpu().numpy()
        assert hm.min() > 0
        Ps = _dense(hs, hd, hm, S * S)
        # against the oracle entry by entry (FP64 prefix sums against the
        # sequential subtraction of the loops: rounding of the running sums)
        assert np.abs(Ps - Po).max() <= 1e-12
        if precision == "fp64":
            # the library's own FP64 recovery: the same algorithm, the same entries
            assert n == len(mass)
            np.testing.assert_array_equal(hs, src)
            np.testing.assert_array_equal(hd, dst)
            np.testing.assert_allclose(hm, mass, rtol=0, atol=1e-12)
            assert abs(l1s[0] - l1[0]) <= 1e-12 and abs(l1s[1] - l1[1]) <= 1e-12
        else:
            # the library recovers an FP32 solution from its FP32 flows with
            # double-float prefix sums; this entry point takes the FP64 export
            assert np.abs(Ps - Pg).max() <= 1e-12
            assert abs(l1s[0] - l1[0]) <= 1e-10 and abs(l1s[1] - l1[1]) <= 1e-10
        # clobber the outputs so the second call has to rewrite them
        o_src.fill_(-1)
        o_dst.fill_(-1)
        o_mass.fill_(-1.0)
        torch.cuda.synchronize()


def test_static_recovery_rejects_grids_beyond_its_scratch():
    from paper_2408_00598_gb300 import hot
    lib = hot.load_library()
    fn = _bind(lib)
    nnz = ctypes.c_size_t()
    # 260 > 256: refused before anything touches the (unused) pointer
    rc = fn(ctypes.c_void_p(16), 260, 260, None, None, None, None, None, 0, ctypes.byref(nnz), None, None)
    assert rc == hot.HOT_EINVAL
    assert b"256" in lib.hot_last_error(None)
