"""Distillation, quark loops and disconnected correlators (oracle; test infrastructure).

Definitions followed (paper section / equation):

* Laplacian eigenvectors (Sec. 3.1, 3.2): v_i(t) are eigenvectors of the gauge-covariant 3D
  Laplacian on timeslice t; here
      (-Lap psi)(x) = sum_{k=x,y,z} [ 2 psi(x) - U_k(x) psi(x+k) - U_k(x-k)^dag psi(x-k) ]
  (spatially periodic), lowest n_ev eigenpairs from a dense Hermitian eigensolve, each
  vector's largest-modulus component (first on ties) made real and positive.
* Sources (Sec. 3.1): b_{t,j,beta}(x) = delta_{x0,t} e_beta (x) v_j(t)(xvec).
* Perambulators: tau(t',t)^{ij}_{alpha beta} = sum_{xvec,a} v_i(t')^*(xvec,a)
  X_{t,j,beta}(t',xvec,alpha,a) with X = D^{-1} b (full) or D_Lambda^{-1} b (domain operator of
  Sec. 2.1; the solution of a source in domain k lives in domain k only).
  Stored as tau[t_src][i][alpha][j][beta] (sink eigvec, sink spin, source eigvec, source spin).
* Quark loops (Sec. 2 loop definition with the distillation elementals of Sec. 3.2):
      L_Gamma(t) = sum_i w_i sum_{alpha beta} Gamma_{alpha beta} tau^{ii}_{beta alpha}(t,t),
  w_i = 1 for standard distillation, |g_k(lambda_i)|^2 for the Gaussian profiles
  g_k(lambda) = exp(-lambda^2 / (2 (0.8 omega_k)^2)).  No fermion-loop sign (it cancels in the
  product of two loops).  The loop with the conjugate insertion uses Gamma-tilde.
* Correlators with the ensemble average <.> taken as the mean over configurations:
      C(x0,y0)    = <L_G(x0) Lt_G(y0)> - <L_G(x0)><Lt_G(y0)>                     (Eq. Cdisc)
      C_LL(x0,y0) = same with the domain loops of the domains holding x0 and y0 (the completely
                    factorised term of Eq. correlator_factorised)
      dC          = C - C_LL                                       (Eq. subtracted_correlator)
  valid only where dom(x0) != dom(y0) (non-overlapping regions, Sec. 3.1); the average over
  source positions y0 (Sec. 3.1) is taken over all y0 for C and over the valid y0 for dC.
  The four VEV-subtracted pieces of Eqs. corr1-corr4 use dL = L - L_Lambda (Sec. 4).
* Quark-line connected part of Eq. Cfull with distilled quark lines V tau V^dag:
      C^(c)_G(x0,y0) = - Tr[ G tau(x0,y0) Gt tau(y0,x0) ]   (trace over eigenvector and spin),
  the Wick contraction of the same bilinears whose disconnected part is <L_G Lt_G> (the minus
  sign is the fermion loop), read from all-sink perambulators of every source timeslice.
* Noise-reduced estimator (Sec. 4): C^NR_Delta(x0,y0) = C^(c)(x0,y0) + dC_Delta(x0,y0), with the
  block size Delta chosen per separation x0 - y0; where no Delta is assigned the standard
  disconnected part C^(d) is used.

Pinned by (tests/test_oracle_distill.py): free-field eigenvalues, eigen-residuals and
orthonormality; the free-field closed form of tau^{ii}(t,t); the complete-basis identity
L_Gamma(t) = sum_xvec Tr[Gamma D^{-1}(x,x)] against dense LU; gauge invariance of the loops;
the reality properties implied by gamma_5-hermiticity; correlators against numpy's covariance.
"""
import numpy as np

from .gamma import clifford_table, gamma_tilde
from .dirac import domain_of_t
from .solve import cgnr

GAUSSIAN_PROFILE_WIDTHS = (0.05, 0.129, 0.208, 0.287)  # omega_k of Sec. 3.2


# ----------------------------------------------------------------------------- Laplacian
def laplacian3d(U, t, phi):
    """(-Lap phi) on timeslice t; phi[..., z, y, x, 3]."""
    out = 6.0 * phi
    for k in range(3):
        ax = {0: -2, 1: -3, 2: -4}[k]
        Uk = U[t, :, :, :, k]
        fwd = np.einsum("zyxab,...zyxb->...zyxa", Uk, np.roll(phi, -1, axis=ax))
        bwd = np.roll(np.einsum("zyxba,...zyxb->...zyxa", np.conj(Uk), phi), 1, axis=ax)
        out -= fwd + bwd
    return out


def laplacian_dense(U, t):
    Lt, Lz, Ly, Lx = U.shape[:4]
    n = 3 * Lx * Ly * Lz
    E = np.eye(n, dtype=np.complex128).reshape(n, Lz, Ly, Lx, 3)
    return laplacian3d(U, t, E).reshape(n, n).T


def fix_phase(v):
    """Make the largest-modulus component (first on ties) of each row real positive."""
    flat = v.reshape(v.shape[0], -1)
    k = np.argmax(np.abs(flat), axis=1)
    ph = flat[np.arange(flat.shape[0]), k]
    return (flat * (np.abs(ph) / ph)[:, None]).reshape(v.shape)


def laplace_eigs(U, n_ev, timeslices=None):
    """Lowest n_ev eigenpairs of -Lap per timeslice: (lam[t][i], V[t, i, z, y, x, 3])."""
    Lt, Lz, Ly, Lx = U.shape[:4]
    ts = range(Lt) if timeslices is None else timeslices
    lams, vecs = [], []
    for t in ts:
        M = laplacian_dense(U, t)
        w, Q = np.linalg.eigh(M)
        lams.append(w[:n_ev])
        vecs.append(fix_phase(Q[:, :n_ev].T.copy()).reshape(n_ev, Lz, Ly, Lx, 3))
    return np.array(lams), np.array(vecs)


# ----------------------------------------------------------------------------- sources / tau
def sources(V_t, t, dims):
    """b[j*4 + beta] = delta_{x0,t} e_beta (x) v_j(t) for one source timeslice; V_t[j,z,y,x,3]."""
    Lx, Ly, Lz, Lt = dims
    n_ev = V_t.shape[0]
    b = np.zeros((n_ev, 4, Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    for beta in range(4):
        b[:, beta, t, :, :, :, beta, :] = V_t
    return b.reshape(n_ev * 4, Lt, Lz, Ly, Lx, 4, 3)


def project(V_tp, X, tp):
    """tau[i, alpha, r] = sum_{xvec,a} v_i(t')^* X_r(t', xvec, alpha, a)."""
    return np.einsum("izyxa,rzyxsa->isr", np.conj(V_tp), X[:, tp])


def perambulators(op, V, t_src, solver=None, sinks="diag", tol=1e-13):
    """tau for each source timeslice: diag -> [n_t, i, alpha, j, beta] at t' = t;
    all -> [n_t, t', i, alpha, j, beta].  ``op`` is D or a domain operator D_Lambda.
    V[t] holds the eigenvectors of timeslice t for every t (full array)."""
    dims = op.dims
    n_ev = V.shape[1]
    out = []
    for t in t_src:
        b = sources(V[t], t, dims)
        if solver is None:
            X, info = cgnr(op, b, tol=tol)
            assert np.all(info["true_resid"] <= tol), info["true_resid"].max()
        else:
            X = solver(b)
        if sinks == "diag":
            tau = project(V[t], X, t)  # [i, alpha, (j beta)]
            out.append(tau.reshape(n_ev, 4, n_ev, 4))
        else:
            out.append(np.array([project(V[tp], X, tp).reshape(n_ev, 4, n_ev, 4)
                                 for tp in range(dims[3])]))
    return np.array(out)


# ----------------------------------------------------------------------------- loops
def profile_weights(lam, omega):
    """|g_k(lambda)|^2 with g_k(lambda) = exp(-lambda^2 / (2 (0.8 omega)^2)) (Sec. 3.2)."""
    g = np.exp(-(lam ** 2) / (2.0 * (0.8 * omega) ** 2))
    return np.abs(g) ** 2


def loops(tau, gamma_ids, weights=None):
    """(L, Lt)[g, n_t]: Gamma and Gamma-tilde loops from diagonal perambulators tau[n_t,i,a,j,b]."""
    table = clifford_table()
    n_t, n_ev = tau.shape[0], tau.shape[1]
    w = np.ones((n_t, n_ev)) if weights is None else np.asarray(weights, dtype=np.float64)
    L = np.zeros((len(gamma_ids), n_t), dtype=np.complex128)
    Lt = np.zeros_like(L)
    for gi, g in enumerate(gamma_ids):
        G = table[g]
        Gt = gamma_tilde(G)
        for k in range(n_t):
            for i in range(n_ev):
                T_ii = tau[k, i, :, i, :]  # [sink spin beta, source spin alpha]
                L[gi, k] += w[k, i] * np.trace(G @ T_ii)
                Lt[gi, k] += w[k, i] * np.trace(Gt @ T_ii)
    return L, Lt


def point_loops(Dinv_diag, gamma_ids):
    """sum_xvec Tr[Gamma D^{-1}(x,x)] per timeslice from the site-diagonal 12x12 blocks
    Dinv_diag[t, z, y, x, 12, 12] (index spin*3 + colour) of the exact inverse (Sec. 2)."""
    table = clifford_table()
    blocks = Dinv_diag.reshape(Dinv_diag.shape[:4] + (4, 3, 4, 3))
    # spin matrix summed over colour and space: M_t[s, q] = sum_{xvec, a} Dinv(x,x)_{s a, q a}
    Mt = np.einsum("tzyxsaqa->tsq", blocks)
    out = np.zeros((len(gamma_ids), Dinv_diag.shape[0]), dtype=np.complex128)
    for gi, g in enumerate(gamma_ids):
        out[gi] = np.einsum("sq,tqs->t", table[g], Mt)
    return out


# ----------------------------------------------------------------------------- correlators
def disc_correlators(L, Lt, Ld, Ltd, extents, vev=True, t_start=0):
    """Full, completely factorised and subtracted disconnected correlators.

    L, Lt, Ld, Ltd: [n_cfg, n_gamma, T] full and domain loops (Gamma and Gamma-tilde); the
    domains are the tiling `extents` starting at t_start.
    Returns dict with C, C_dd, dC [n_gamma, T, T] (index [g, x0, y0]), valid [T, T],
    C_avg, dC_avg [n_gamma, T] (index Delta t = x0 - y0 mod T), n_valid [T], and the four
    pieces of Eqs. corr1-corr4 as terms [4, n_gamma, T, T]."""
    n_cfg, n_g, T = L.shape

    def conn(A, B):
        c = np.einsum("cgx,cgy->gxy", A, B) / n_cfg
        if vev:
            c = c - np.einsum("gx,gy->gxy", A.mean(0), B.mean(0))
        return c

    C = conn(L, Lt)
    C_dd = conn(Ld, Ltd)
    dC = C - C_dd
    dom = domain_of_t(extents, T, t_start)
    valid = (dom[:, None] != dom[None, :]).astype(np.int32)
    C_avg = np.zeros((n_g, T), dtype=np.complex128)
    dC_avg = np.zeros((n_g, T), dtype=np.complex128)
    n_valid = np.zeros(T, dtype=np.int32)
    for dt in range(T):
        for y0 in range(T):
            x0 = (y0 + dt) % T
            C_avg[:, dt] += C[:, x0, y0] / T
            if valid[x0, y0]:
                dC_avg[:, dt] += dC[:, x0, y0]
                n_valid[dt] += 1
        if n_valid[dt]:
            dC_avg[:, dt] /= n_valid[dt]
    dL, dLt = L - Ld, Lt - Ltd
    terms = np.array([conn(Ld, Ltd), conn(Ld, dLt), conn(dL, Ltd), conn(dL, dLt)])
    return dict(C=C, C_dd=C_dd, dC=dC, valid=valid, C_avg=C_avg, dC_avg=dC_avg,
                n_valid=n_valid, terms=terms)


def window_average(C, dC, valid, t_lo, t_hi):
    """Averages over source positions restricted to a bulk window (Sec. 3: source and sink both
    in t_lo <= x0, y0 <= t_hi, away from the open time boundaries; Sec. 4 quotes 24a..71a):
        C_avg[g, dt]  = mean over y0 in [t_lo, t_hi - dt] of C[g, y0 + dt, y0]        (no wrap),
        dC_avg[g, dt] = the same over the pairs with valid[y0 + dt, y0] (distinct domains),
    with n_pairs[dt] = t_hi - t_lo + 1 - dt and n_valid[dt] the number of valid pairs (0 where no
    pair exists, the averages then 0), dt = 0 .. T-1."""
    n_g, T = C.shape[0], C.shape[1]
    if not 0 <= t_lo <= t_hi < T:
        raise ValueError("window outside [0, T)")
    C_avg = np.zeros((n_g, T), dtype=np.complex128)
    dC_avg = np.zeros((n_g, T), dtype=np.complex128)
    n_pairs = np.zeros(T, dtype=np.int32)
    n_valid = np.zeros(T, dtype=np.int32)
    for dt in range(T):
        for y0 in range(t_lo, t_hi + 1):
            x0 = y0 + dt
            if x0 > t_hi:
                break
            C_avg[:, dt] += C[:, x0, y0]
            n_pairs[dt] += 1
            if valid[x0, y0]:
                dC_avg[:, dt] += dC[:, x0, y0]
                n_valid[dt] += 1
        if n_pairs[dt]:
            C_avg[:, dt] /= n_pairs[dt]
        if n_valid[dt]:
            dC_avg[:, dt] /= n_valid[dt]
    return dict(C_avg=C_avg, dC_avg=dC_avg, n_pairs=n_pairs, n_valid=n_valid)


def conn_correlator(tau_all, t_src, gamma_ids):
    """C[g, x0, k] = C^(c)(x0, y0 = t_src[k]) and its y0 average C_avg[g, dt] = mean over k of
    C[g, (t_src[k] + dt) mod T, k].  tau_all[k, t', i, a, j, b] = tau(t', t_src[k]) (all sinks);
    t_src must contain every timeslice, so tau(y0, x0) is read directly from the perambulator of
    source x0 (no gamma_5-hermiticity is used here)."""
    n_t, T, n_ev = tau_all.shape[0], tau_all.shape[1], tau_all.shape[2]
    pos = {int(t): k for k, t in enumerate(t_src)}
    if sorted(pos) != list(range(T)):
        raise ValueError("conn_correlator needs the perambulators of every source timeslice")
    table = clifford_table()
    one = np.eye(n_ev)
    C = np.zeros((len(gamma_ids), T, n_t), dtype=np.complex128)
    for gi, g in enumerate(gamma_ids):
        Gx = np.kron(one, table[g])  # acts on the (eigvec, spin) index at x0
        Gy = np.kron(one, gamma_tilde(table[g]))  # at y0
        for k, y0 in enumerate(t_src):
            for x0 in range(T):
                A = tau_all[k, x0].reshape(4 * n_ev, 4 * n_ev)  # tau(x0, y0)
                B = tau_all[pos[x0], int(y0)].reshape(4 * n_ev, 4 * n_ev)  # tau(y0, x0)
                C[gi, x0, k] = -np.trace(Gx @ A @ Gy @ B)
    C_avg = np.zeros((len(gamma_ids), T), dtype=np.complex128)
    for dt in range(T):
        for k, y0 in enumerate(t_src):
            C_avg[:, dt] += C[:, (int(y0) + dt) % T, k] / n_t
    return C, C_avg


def point_conn_correlator(Dinv, dims, gamma_ids):
    """C^(c)(x0, y0) = - sum_{xvec, yvec} Tr[G D^{-1}(x,y) Gt D^{-1}(y,x)] from the dense inverse
    (rows and columns ordered (site, spin, colour), sites x fastest): the point-source form that
    distillation with a complete basis reproduces."""
    Lx, Ly, Lz, Lt = dims
    L3 = Lx * Ly * Lz
    table = clifford_table()
    Db = Dinv.reshape(Lt, L3, 4, 3, Lt, L3, 4, 3)
    out = np.zeros((len(gamma_ids), Lt, Lt), dtype=np.complex128)
    for gi, g in enumerate(gamma_ids):
        G, Gt = table[g], gamma_tilde(table[g])
        # trace over spin and colour of G S(x,y) Gt S(y,x), summed over xvec and yvec
        out[gi] = -np.einsum("da,xpaqyrbs,bc,yrcsxpdq->xy", G, Db, Gt, Db, optimize=True)
    return out


def nr_estimator(C_conn_avg, C_disc_avg, dC_avg_by_delta, delta_of_dt):
    """C^NR[g, dt] = C_conn_avg[g, dt] + dC_avg_by_delta[delta_of_dt[dt], g, dt], or
    + C_disc_avg[g, dt] where delta_of_dt[dt] < 0 (no block size assigned)."""
    out = np.array(C_conn_avg, dtype=np.complex128)
    for dt, d in enumerate(delta_of_dt):
        out[:, dt] += dC_avg_by_delta[d][:, dt] if d >= 0 else C_disc_avg[:, dt]
    return out


def effective_mass(C_of_dt):
    """a m_eff(dt) = ln[C(dt) / C(dt + 1)] (Sec. 3.2)."""
    C = np.asarray(C_of_dt)
    return np.log(C[..., :-1] / C[..., 1:])
