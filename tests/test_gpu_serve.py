"""Serving through hot_submit / hot_poll: continuous batching, results that do
not depend on the mix, cancellation and admission by device memory."""
import time

import numpy as np
import pytest

from paper_2408_00598_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2408_00598_gb300 import hot
    hot.load_library()
    return hot


MIX = [("white", 16, 1), ("gauss", 32, 2), ("shapes", 64, 3), ("cauchy", 48, 4), ("translate", 32, 5),
       ("white", 128, 6), ("gauss", 96, 7), ("shapes", 16, 8)]


def test_results_are_the_same_alone_and_in_the_mix(lib):
    pairs = [syn.make_pair(k, S, s) for k, S, s in MIX]
    with lib.Context(precision="fp32") as solo:
        alone = []
        for a, b in pairs:
            r = solo.solve(a, b, tol=1e-6)
            solo.release(r)
            alone.append(r)
    with lib.Context(precision="fp32") as srv:
        # staggered arrivals: half now, half while the first half runs
        tickets = [srv.submit(a, b, tol=1e-6) for a, b in pairs[:4]]
        time.sleep(0.002)
        tickets += [srv.submit(a, b, tol=1e-6) for a, b in pairs[4:]]
        got = []
        for t in tickets:
            st, res = srv.wait(t, timeout_ms=300000)
            assert st == lib.HOT_OK, st
            got.append(res)
        stats = srv.serve_stats()
    for a, g in zip(alone, got):
        assert g["ot_value"] == a["ot_value"]
        assert g["iters"] == a["iters"]
        assert g["rel_kkt"] == a["rel_kkt"]
    assert stats["completed"] == len(pairs)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_poll_pending_then_done(lib):
    a, b = syn.make_pair("gauss", 64, 11)
    with lib.Context(precision="fp32") as srv:
        t = srv.submit(a, b, tol=1e-7)
        st, _ = srv.poll(t)
        assert st in (lib.HOT_PENDING, lib.HOT_OK)
        deadline = time.time() + 120
        while st == lib.HOT_PENDING and time.time() < deadline:
            time.sleep(0.001)
            st, res = srv.poll(t)
        assert st == lib.HOT_OK
        assert res["rel_kkt"] <= 1e-7
        assert srv.forget(t) == lib.HOT_OK
        with pytest.raises(lib.HotError):
            srv.poll(t)


def test_cancel_queued_and_running(lib):
    a, b = syn.make_pair("white", 128, 3)
    with lib.Context(precision="fp32", max_batch=1) as srv:
        t1 = srv.submit(a, b, tol=0.0, max_iter=10 ** 9)    # never converges
        t2 = srv.submit(a, b, tol=1e-6)                      # waits for the only slot
        assert srv.cancel(t2) == lib.HOT_OK
        st2, _ = srv.poll(t2)                                # a queued request leaves at once
        assert st2 == lib.HOT_ECANCELLED
        time.sleep(0.05)
        assert srv.cancel(t1) == lib.HOT_OK
        st1, r1 = srv.wait(t1, timeout_ms=60000)
        st2, r2 = srv.wait(t2, timeout_ms=60000)
        assert st1 == lib.HOT_ECANCELLED and st2 == lib.HOT_ECANCELLED
        assert srv.serve_stats()["cancelled"] == 2


def test_admission_is_bounded_by_device_memory(lib):
    a, b = syn.make_pair("white", 128, 3)
    # 128^3 * 2 * 4 B * 5 buffers ~ 84 MB per instance: a 10 MB budget can never hold it
    with lib.Context(precision="fp32", mem_budget=10 * 1024 * 1024) as srv:
        t = srv.submit(a, b, tol=1e-6)
        st, _ = srv.wait(t, timeout_ms=60000)
        assert st == lib.HOT_ENOMEM
        assert srv.serve_stats()["rejected"] == 1


def test_invalid_request(lib):
    a, b = syn.make_pair("white", 16, 3)
    with lib.Context(precision="fp32") as srv:
        with pytest.raises(lib.HotError):
            srv.submit(a * 2, b)
        with pytest.raises(lib.HotError):
            srv.submit(a, b, max_iter=0)
