"""Host-side checks of the C ABI that need no GPU: the library builds, exports
every function include/hot.h declares, and the ctypes structs of the binding
have the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hot.h")


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                names |= set(re.findall(r"HOT_API[^;(]*?\b(hot_\w+)\s*\(", f.read()))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2408_00598_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["hot_create", "hot_solve", "hot_recover_plan", "hot_submit", "hot_poll", "hot_destroy"]:
        assert must in names
    assert len(names) >= 16


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name)


def test_library_loads_and_calls_host_only_entry_points(libpath):
    from paper_2408_00598_gb300 import hot
    lib = hot.load_library()
    assert hot.hot_status_string(hot.HOT_NOT_CONVERGED) == "HOT_NOT_CONVERGED"
    cfg = hot.hot_config_default()
    assert cfg.check_every == 10 and cfg.precision == hot.HOT_FP32_BULK
    assert abs(cfg.restart_sufficient - 0.2) < 1e-15
    # invalid configuration is rejected before any device work
    bad = hot.hot_config_default()
    bad.check_every = 3
    h = ctypes.c_void_p()
    assert lib.hot_create(ctypes.byref(h), ctypes.byref(bad)) == hot.HOT_EINVAL
    assert lib.hot_create(None, ctypes.byref(cfg)) == hot.HOT_EINVAL
    assert lib.hot_sweep_timing(None, 1, None, None, None) == hot.HOT_EINVAL


C_PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "hot.h"
#define P(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f));
int main(void) {
  printf("hot_config %zu\nhot_result %zu\nhot_request %zu\nhot_serve_stats %zu\nhot_kernel_times %zu\n",
         sizeof(hot_config), sizeof(hot_result), sizeof(hot_request), sizeof(hot_serve_stats),
         sizeof(hot_kernel_times));
  P(hot_config, sigma0) P(hot_config, mem_budget) P(hot_config, autotune_cache) P(hot_config, keep_batch_solutions)
  P(hot_result, iters) P(hot_result, solution_id) P(hot_result, max_abs_dual) P(hot_result, n) P(hot_result, blocks)
  P(hot_request, tol) P(hot_request, keep_solution)
  P(hot_serve_stats, device_bytes_in_use) P(hot_serve_stats, blocks_run)
  return 0;
}
"""


def test_ctypes_layout_matches_c_header():
    from paper_2408_00598_gb300 import hot
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        with open(src, "w") as f:
            f.write(C_PROBE)
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    kv = dict(line.split() for line in out if line.strip())
    structs = {"hot_config": hot.hot_config, "hot_result": hot.hot_result, "hot_request": hot.hot_request,
               "hot_serve_stats": hot.hot_serve_stats, "hot_kernel_times": hot.hot_kernel_times}
    for name, cls in structs.items():
        assert int(kv[name]) == ctypes.sizeof(cls), name
    for key, val in kv.items():
        if "." in key:
            s, fld = key.split(".")
            assert getattr(structs[s], fld).offset == int(val), key
