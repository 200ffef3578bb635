"""Write tests/golden/oracle_values.json: FP64 oracle results for the GPU parity cases.

Calls only ``oracle/`` (and the seeded input generators).  Each record holds
the inputs' SHA-256 so a test can tell whether the generator reproduced the
same histograms on its machine (else it reruns the oracle live).

    python tests/golden/make_oracle_values.py [--jobs N]
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import hot, exact  # noqa: E402
from paper_2408_00598_gb300 import synthetic as syn  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")

# (name, kind, S, seed, tol, max_iter, with_exact)
CASES = [("c1_white16", "white", 16, 1, 1e-8, 100000, True)]
for kind in syn.KINDS:
    CASES.append(("c2_%s64" % kind, kind, 64, 2, 1e-6, 100000, False))
    CASES.append(("c2_%s32" % kind, kind, 32, 3, 1e-6, 100000, False))
    CASES.append(("s16_%s" % kind, kind, 16, 4, 1e-6, 100000, True))


def digest(mu1, mu2):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(mu1).tobytes())
    h.update(np.ascontiguousarray(mu2).tobytes())
    return h.hexdigest()


def run_case(case):
    name, kind, S, seed, tol, max_iter, with_exact = case
    mu1, mu2 = syn.make_pair(kind, S, seed)
    t = time.time()
    r = hot.hot_solve(mu1, mu2, tol=tol, max_iter=max_iter)
    rec = dict(name=name, kind=kind, S=S, seed=seed, tol=tol, max_iter=max_iter, sha256=digest(mu1, mu2),
               ot_value=float(r.ot_value), dual_value=float(r.dual_value), rel_kkt=float(r.rel_kkt),
               iters=int(r.iters), restarts=int(r.restarts), converged=bool(r.converged), sigma=float(r.sigma),
               seconds=time.time() - t)
    if with_exact:
        rec["exact"] = float(exact.ot_exact_mcf(mu1, mu2))
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        recs = pool.map(run_case, CASES)
    data = {"about": "FP64 oracle (oracle/hot.py, Algorithm 2 with the stated restart reading) on seeded "
                     "synthetic pairs; written by tests/golden/make_oracle_values.py. 'exact' is the "
                     "min-cost-flow optimum of eq. (1) (oracle/mcf.c).",
            "cases": {r["name"]: r for r in recs}}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
