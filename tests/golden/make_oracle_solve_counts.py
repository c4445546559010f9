"""Write the oracle's MINRES iteration counts on the named workloads (oracle_solve_counts.json).

The GPU tests hold each precision form's iteration count to the FP64 oracle's count at the same
alpha and tolerance.  At the workloads' full sizes the oracle's solve takes minutes, so its
counts are computed once by this script and stored; it calls nothing but ``oracle`` and
``workloads``.

Usage (from the repository root):
    python tests/golden/make_oracle_solve_counts.py [--workloads a,b] [--alphas 1e-8,1e-6,1e-3]
        [--out tests/golden/oracle_solve_counts.json]
    python tests/golden/make_oracle_solve_counts.py --batched --alphas 1e-8,1e-2,1e-6

Each entry records the workload, alpha, tol, the iteration count, the recurrence estimates
|eta_j|/eta_0 and the true relative residual ||Yf - YAu|| / ||Yf|| of the returned iterate
(stopping rule of Sec. 5.2 read as: the estimate, then the true residual, both <= tol).
Existing entries for other (workload, alpha) pairs are kept.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from workloads import batched_systems, heat_bdf_problem, rhs_smoothed_field, workload  # noqa: E402


def _heat3d_m63():
    # the 3-D backward-Euler heat family at m = 63 (65 M unknowns), same right-hand-side recipe
    p = heat_bdf_problem(3, 63, 256)
    return p, (lambda: rhs_smoothed_field(p.N, 3, p.m, 3))


EXTRA = {"heat3d_bdf_N256_m63": _heat3d_m63}


def batched_sample(out, alphas, tol):
    """The oracle's counts for the small systems of the 96-system batched workload (M <= 3969
    and at most 600,000 unknowns), every right-hand side (seeded U[-1, 1], seed 4 + 1000 s + r),
    at each alpha."""
    doc = {"source": "FP64 oracle (oracle.solve) on the small systems of batched_systems(96, 4, "
                     "seed=4); written by tests/golden/make_oracle_solve_counts.py --batched",
           "tol": tol, "cases": []}
    for s, (p, rhs) in enumerate(batched_systems(96, 4, seed=4)):
        if p.M > 3969 or p.n > 600_000:
            continue
        for r, rf in enumerate(rhs):
            f = rf()
            for alpha in alphas:
                res = O.solve(p, f, alpha=alpha, tol=tol, maxit=100)
                entry = dict(system=s, rhs=r, name=p.name, N=p.N, M=p.M, alpha=alpha,
                             iters=int(res["iters"]), status=res["status"])
                print(json.dumps(entry), flush=True)
                doc["cases"].append(entry)
    with open(out, "w") as fh:
        json.dump(doc, fh, indent=0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="frac1d_N64_m63_g0.5,frac2d_N1024_m255_g0.7")
    ap.add_argument("--alphas", default="1e-8,1e-6,1e-3")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "oracle_solve_counts.json"))
    ap.add_argument("--batched", action="store_true",
                    help="write oracle_counts_batched_sample.json instead")
    args = ap.parse_args()
    if args.batched:
        batched_sample(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                    "oracle_counts_batched_sample.json"),
                       [float(a) for a in args.alphas.split(",")], args.tol)
        return
    doc = {"source": "FP64 oracle (oracle.solve: textbook preconditioned MINRES, structured "
                     "P_alpha^{-1} of Sec. 5.1) on the named seeded workloads; written by "
                     "tests/golden/make_oracle_solve_counts.py",
           "cases": []}
    if os.path.exists(args.out):
        with open(args.out) as fh:
            doc = json.load(fh)
    for name in args.workloads.split(","):
        prob, rf = EXTRA[name]() if name in EXTRA else workload(name)
        f = rf()
        for alpha in (float(a) for a in args.alphas.split(",")):
            t0 = time.time()
            r = O.solve(prob, f, alpha=alpha, tol=args.tol, maxit=100)
            entry = dict(workload=name, N=prob.N, M=prob.M, alpha=alpha, tol=args.tol,
                         iters=int(r["iters"]), status=r["status"],
                         relres_true=float(r["relres_true"]),
                         eta_history=[float(h) for h in r["eta_history"]],
                         cpu_seconds=round(time.time() - t0, 1))
            print(json.dumps(entry), flush=True)
            doc["cases"] = [c for c in doc["cases"]
                            if not (c["workload"] == name and c["alpha"] == alpha
                                    and c["tol"] == args.tol)]
            doc["cases"].append(entry)
            with open(args.out, "w") as fh:
                json.dump(doc, fh, indent=1)
        del f


if __name__ == "__main__":
    main()
