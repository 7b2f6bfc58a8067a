"""Shared synthetic cases for the GPU parity tests (inputs from lqcd_inputs only)."""
import numpy as np

from lqcd_inputs import gauge_field

# 4^3 x 8, eps 0.3, kappa 0.12, c_sw 1.5, N_ev 4, two time domains of 4 (the plain FP64 workload)
SMALL = dict(dims=(4, 4, 4, 8), eps=0.3, kappa=0.12, c_sw=1.5, n_ev=4, extents=[4, 4])
# rough field at the mixed-precision workload's couplings
ROUGH = dict(dims=(4, 4, 4, 8), eps=0.5, kappa=0.125, c_sw=1.6, n_ev=4, extents=[4, 4])


def gauge(case, seed):
    return gauge_field(case["dims"], case["eps"], seed)


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def per_domain_resid(b, r, extents):
    """||r||/||b|| per (rhs, domain) for spinor arrays [nrhs, t, z, y, x, 4, 3]."""
    out = []
    for k in range(b.shape[0]):
        t0 = 0
        row = []
        for e in extents:
            nb = np.linalg.norm(b[k, t0:t0 + e])
            row.append(np.linalg.norm(r[k, t0:t0 + e]) / nb if nb > 0 else 0.0)
            t0 += e
        out.append(row)
    return np.array(out)
