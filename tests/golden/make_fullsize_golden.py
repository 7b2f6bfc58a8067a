"""Write the oracle's values for the full-size parity tests (calls only oracle/ and the seeded
input generators; nothing here comes from the CUDA path).

    python tests/golden/make_fullsize_golden.py [--part tau|eigs|all]

Workload: the 16^3 x 32 mixed-precision configuration (U = exp(i 0.5 H), seed 2001; kappa 0.125,
c_sw 1.6; antiperiodic in time; eight time domains of extent 4), 32 seeded orthonormal colour
vectors per timeslice (seed 2002).  Written to tests/golden/fullsize_16x16x16x32.json:

* tau_full: perambulator columns (Sec. 3.1) of the full operator for source timeslice 0 and the
  sampled source vectors J (every spin): tau[i][alpha][j][beta] at t' = t = 0 for j in J,
  from the oracle's CGNR solve to true residual 1e-12;
* tau_dom: the same columns for the domain operator of Sec. 2.1 with one multi-site source per
  (j, beta) covering the source timeslices 0, 4, ..., 28 (one per domain, Sec. 4), projected on
  each source timeslice;
* eig_lambda: the 32 lowest eigenvalues of the covariant 3D Laplacian on timeslice 0 of the same
  gauge field (dense Hermitian eigensolve), for the GPU eigensolver test.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 32)
EPS, KAPPA, CSW = 0.5, 0.125, 1.6
GAUGE_SEED, CV_SEED = 2001, 2002
N_EV = 32
EXTENTS = [4] * 8
J_SAMPLE = [0, 17]
TOL = 1e-12
OUT = os.path.join(HERE, "fullsize_16x16x16x32.json")


def cplx_list(a):
    a = np.asarray(a, dtype=np.complex128).ravel()
    return [[float(v.real), float(v.imag)] for v in a]


def tau_part(out):
    from lqcd_inputs import colour_vectors, gauge_field
    from oracle.dirac import WilsonClover
    from oracle.distill import project, sources
    from oracle.solve import cgnr

    U = gauge_field(DIMS, EPS, GAUGE_SEED)
    op = WilsonClover(U, KAPPA, CSW)
    T = DIMS[3]
    t_dom = list(range(0, T, 4))
    V = colour_vectors(DIMS, N_EV, CV_SEED, timeslices=t_dom)  # slot k = timeslice 4 k
    # full operator, source timeslice 0
    b_all = sources(V[0], 0, DIMS)
    cols = [j * 4 + beta for j in J_SAMPLE for beta in range(4)]
    t0 = time.time()
    X, info = cgnr(op, b_all[cols], tol=TOL)
    assert np.all(info["true_resid"] <= TOL)
    tau_f = project(V[0], X, 0)  # [i, alpha, col]
    out["tau_full"] = {"t": 0, "j": J_SAMPLE, "shape": [N_EV, 4, len(J_SAMPLE), 4],
                       "values": cplx_list(tau_f.reshape(N_EV, 4, len(J_SAMPLE), 4)),
                       "cgnr_iters": [int(v) for v in info["iters"]], "seconds": time.time() - t0}
    # domain operator, multi-site sources: one source timeslice per domain
    opd = op.restricted(EXTENTS)
    b = np.zeros_like(b_all[cols])
    for k, t in enumerate(t_dom):
        b += sources(V[k], t, DIMS)[cols]
    t0 = time.time()
    Xd, info = cgnr(opd, b, tol=TOL)
    assert np.all(info["true_resid"] <= TOL)
    tau_d = np.array([project(V[k], Xd, t) for k, t in enumerate(t_dom)])  # [k, i, alpha, col]
    out["tau_dom"] = {"t": t_dom, "j": J_SAMPLE, "extents": EXTENTS,
                      "shape": [len(t_dom), N_EV, 4, len(J_SAMPLE), 4],
                      "values": cplx_list(tau_d.reshape(len(t_dom), N_EV, 4, len(J_SAMPLE), 4)),
                      "cgnr_iters": [int(v) for v in info["iters"]], "seconds": time.time() - t0}


def eig_part(out):
    from lqcd_inputs import gauge_field
    from oracle.distill import laplacian_dense

    U = gauge_field(DIMS, EPS, GAUGE_SEED)
    t0 = time.time()
    M = laplacian_dense(U, 0)
    lam = np.linalg.eigvalsh(M)[:N_EV]
    out["eig_lambda"] = {"t": 0, "n_ev": N_EV, "values": [float(v) for v in lam], "seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--part", default="all", choices=["tau", "eigs", "all"])
    a = ap.parse_args()
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    out["workload"] = {"dims": list(DIMS), "eps": EPS, "kappa": KAPPA, "c_sw": CSW, "gauge_seed": GAUGE_SEED,
                       "cv_seed": CV_SEED, "n_ev": N_EV, "bc": "antiperiodic", "tol": TOL,
                       "generator": "tests/golden/make_fullsize_golden.py (oracle only)"}
    if a.part in ("eigs", "all"):
        eig_part(out)
    if a.part in ("tau", "all"):
        tau_part(out)
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
