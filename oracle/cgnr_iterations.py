"""Iteration count of the oracle's CGNR solve at the couplings of the large workloads
(test and measurement infrastructure: calls only the oracle and the seeded input generators).

    python oracle/cgnr_iterations.py [--dims 32 32 32 64] [--eps 0.6] [--kappa 0.126] [--csw 1.7]
                                     [--seed 4001] [--cv-seed 4002] [--tol 1e-10]

Solves D x = b for the first distillation source of the workload (timeslice 0, colour vector 0,
spin 0; Sec. 3.1 sources) with the oracle's conjugate gradients on the normal equations until the
FP64 true residual is below tol, and writes the iteration count, the final true residual and the
time per iteration to oracle/cgnr_iterations.json (one entry per lattice and coupling set).  The
CPU baseline of bench.py scales its live per-iteration timing of the oracle by this count.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cgnr_iterations.json")


def key(dims, eps, kappa, csw, seed):
    return "%dx%dx%dx%d eps=%g kappa=%g csw=%g seed=%d" % (tuple(dims) + (eps, kappa, csw, seed))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[32, 32, 32, 64])
    ap.add_argument("--eps", type=float, default=0.6)
    ap.add_argument("--kappa", type=float, default=0.126)
    ap.add_argument("--csw", type=float, default=1.7)
    ap.add_argument("--seed", type=int, default=4001)
    ap.add_argument("--cv-seed", type=int, default=4002)
    ap.add_argument("--tol", type=float, default=1e-10)
    a = ap.parse_args()

    from lqcd_inputs import colour_vectors, gauge_field
    from oracle.dirac import WilsonClover
    from oracle.distill import sources
    from oracle.solve import cgnr

    dims = tuple(a.dims)
    t0 = time.time()
    U = gauge_field(dims, a.eps, a.seed)
    op = WilsonClover(U, a.kappa, a.csw)
    V0 = colour_vectors(dims, 1, a.cv_seed, timeslices=[0])
    b = sources(V0[0], 0, dims)[:1]
    t1 = time.time()
    x, info = cgnr(op, b, tol=a.tol)
    t2 = time.time()
    it = int(info["iters"][0])
    entry = {"dims": list(dims), "eps": a.eps, "kappa": a.kappa, "c_sw": a.csw, "seed": a.seed,
             "cv_seed": a.cv_seed, "source": "t=0, colour vector 0, spin 0", "tol": a.tol, "iters": it,
             "true_resid": float(info["true_resid"][0]), "setup_s": t1 - t0, "solve_s": t2 - t1,
             "s_per_iter": (t2 - t1) / max(it, 1)}
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data[key(dims, a.eps, a.kappa, a.csw, a.seed)] = entry
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print(json.dumps(entry))


if __name__ == "__main__":
    main()
