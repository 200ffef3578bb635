"""Write tests/golden/oracle_values.json: FP64 oracle results for the GPU parity cases.

Calls only ``oracle/`` (and the seeded input generators).  Each record holds
the inputs' SHA-256 so a test can tell whether the generator reproduced the
same histograms on its machine (else it reruns the oracle live, where that is
cheap, or skips).

    python tests/golden/make_oracle_values.py [--jobs N] [--only REGEX]

``--only`` recomputes the matching cases and keeps every other stored record.
The large cases (256 x 256, the 64 x 64 absolute-KKT runs) take from about
15 minutes to over an hour each on one core.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import re
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import hot, exact  # noqa: E402
from paper_2408_00598_gb300 import synthetic as syn  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")

# (name, kind, S, seed, tol, max_iter, with_exact[, stop])
CASES = [("c1_white16", "white", 16, 1, 1e-8, 100000, True)]
for kind in syn.KINDS:
    CASES.append(("c2_%s64" % kind, kind, 64, 2, 1e-6, 100000, False))
    CASES.append(("c2_%s32" % kind, kind, 32, 3, 1e-6, 100000, False))
    CASES.append(("s16_%s" % kind, kind, 16, 4, 1e-6, 100000, True))
# 256 x 256 white-noise pair of the throughput benchmark (seed 1000), at the
# paper's stopping rule (440 iterations; the 3.8e4 iterations to relative KKT
# 1e-8 would take the oracle over a day)
CASES.append(("c3_white256", "white", 256, 1000, 1e-6, 100000, False))
# one 128 x 128 pair per class at the paper's stopping rule
for kind in syn.KINDS:
    CASES.append(("c3_%s128" % kind, kind, 128, 5, 1e-6, 100000, False))
# absolute KKT 1e-6 (Table VI) on 64 x 64 pairs: 1e4-1e5 iterations
CASES.append(("f3_shapes64_abs", "shapes", 64, 6, 1e-6, 400000, False, "absolute"))
CASES.append(("f3_gauss64_abs", "gauss", 64, 6, 1e-6, 400000, False, "absolute"))


def digest(mu1, mu2):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(mu1).tobytes())
    h.update(np.ascontiguousarray(mu2).tobytes())
    return h.hexdigest()


def run_case(case):
    name, kind, S, seed, tol, max_iter, with_exact = case[:7]
    stop = case[7] if len(case) > 7 else "relative"
    mu1, mu2 = syn.make_pair(kind, S, seed)
    t = time.time()
    r = hot.hot_solve(mu1, mu2, tol=tol, max_iter=max_iter, params=hot.HotParams(stop=stop))
    rec = dict(name=name, kind=kind, S=S, seed=seed, tol=tol, max_iter=max_iter, sha256=digest(mu1, mu2),
               ot_value=float(r.ot_value), dual_value=float(r.dual_value), rel_kkt=float(r.rel_kkt),
               abs_kkt=float(r.abs_kkt), iters=int(r.iters), restarts=int(r.restarts),
               converged=bool(r.converged), sigma=float(r.sigma), seconds=time.time() - t)
    if stop != "relative":
        rec["stop"] = stop
    if with_exact:
        rec["exact"] = float(exact.ot_exact_mcf(mu1, mu2))
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--only", default=None, help="regex: recompute only the matching cases, keep the others")
    args = ap.parse_args()
    cases = [c for c in CASES if args.only is None or re.search(args.only, c[0])]
    old = {}
    if args.only is not None and os.path.exists(OUT):
        with open(OUT) as f:
            old = json.load(f)["cases"]
    # largest first, so the long runs start at once
    cases.sort(key=lambda c: -c[2] ** 3 * (10 if c[4] < 1e-7 or len(c) > 7 else 1))
    about = ("FP64 oracle (oracle/hot.py, Algorithm 2 with the stated restart reading) on seeded "
             "synthetic pairs; written by tests/golden/make_oracle_values.py. 'exact' is the "
             "min-cost-flow optimum of eq. (1) (oracle/mcf.c).")
    # the file is rewritten as each case finishes, so a long run keeps what it has
    with mp.get_context("spawn").Pool(min(args.jobs, max(1, len(cases)))) as pool:
        for r in pool.imap_unordered(run_case, cases, chunksize=1):
            old[r["name"]] = r
            with open(OUT, "w") as f:
                json.dump({"about": about, "cases": old}, f, indent=1, sort_keys=True)
            print("wrote", r["name"], "%.0f s" % r["seconds"], flush=True)


if __name__ == "__main__":
    main()
