"""Clover-improved Wilson operator and its domain restriction (oracle; test infrastructure).

Follows Sec. 2.1 (block form of D, Dirichlet restriction D_Lambda) and Sec. 3 (Wilson-clover
action).  The paper fixes neither normalisation nor signs; this oracle takes the hopping form

    D = A - kappa H,
    (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
    A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu}(x),
    Fhat_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / 8,   Q = sum of the four plaquette leaves at x,

fermion boundary condition in time as a phase on the t-links leaving t = T-1 (antiperiodic: -1,
periodic: +1, open: 0), periodic in space; the clover term uses the original links.

Domain restriction (Sec. 2.1): the time axis is tiled by consecutive domains starting at
t = t_start (0 unless a shifted tiling places the regions around chosen x0, y0, Fig. 1; the last
domain then wraps around the time boundary).  D_Lambda keeps every term of D whose two sites lie
in the same domain, i.e. it is D with the t-hops between t and t+1 (mod T) removed wherever
dom(t) != dom(t+1); the clover term is kept.
For a single domain covering all of T nothing is removed.  The block-diagonal operator over all
domains is what the simultaneous multi-site-source solves of Sec. 4 invert.

Pinned by (tests/test_oracle_dirac.py): the free-field momentum-space closed form, U(1)
background fields (twisted momenta and the abelian clover closed form), gamma_5-hermiticity
against the independently coded adjoint, gauge covariance, and the dense block structure of
D_Lambda.
"""
import numpy as np

from .gamma import gammas, sigma, PLANES

BC_PERIODIC = 0
BC_ANTIPERIODIC = 1
BC_OPEN = 2

# numpy axis (counted from the end of a spinor array [..., t, z, y, x, spin, colour]) per mu
_SPINOR_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}
# numpy axis of a link-like array [t, z, y, x, ...(2 trailing matrix dims)] per mu
_LINK_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


# ----------------------------------------------------------------------------- geometry tables
def site_index(dims, x, y, z, t):
    """Flat lexicographic site index s = x + Lx (y + Ly (z + Lz t))."""
    Lx, Ly, Lz, _ = dims
    return x + Lx * (y + Ly * (z + Lz * t))


def coords(dims):
    """Arrays (x, y, z, t) over the flat site index."""
    Lx, Ly, Lz, Lt = dims
    s = np.arange(Lx * Ly * Lz * Lt)
    return s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)


def parity_table(dims):
    """Parity (x + y + z + t) mod 2 of every flat site."""
    x, y, z, t = coords(dims)
    return (x + y + z + t) % 2


def eo_order(dims):
    """Site order of the even-odd layout: for each parity p, the sites of parity p listed by
    increasing flat index.  Returns (perm, cb) with perm[p*V/2 + k] = flat site of checkerboard
    index k in parity p, and cb[s] = position of site s within its parity."""
    par = parity_table(dims)
    even = np.nonzero(par == 0)[0]
    odd = np.nonzero(par == 1)[0]
    perm = np.concatenate([even, odd])
    cb = np.empty(par.shape[0], dtype=np.int64)
    cb[even] = np.arange(even.shape[0])
    cb[odd] = np.arange(odd.shape[0])
    return perm, cb


def domain_of_t(extents, Lt, t_start=0):
    """dom[t] for a tiling of the periodic time axis by consecutive domains of the given extents,
    domain 0 starting at t_start: domain d holds t_start + e_0 + ... + e_{d-1} + [0, e_d) mod Lt."""
    extents = [int(e) for e in extents]
    if any(e < 1 for e in extents) or sum(extents) != Lt:
        raise ValueError("domain extents must be >= 1 and tile the time extent")
    if not 0 <= int(t_start) < Lt:
        raise ValueError("t_start outside [0, Lt)")
    dom = np.empty(Lt, dtype=np.int64)
    t = int(t_start)
    for d, e in enumerate(extents):
        for k in range(e):
            dom[(t + k) % Lt] = d
        t += e
    return dom


def cut_after(extents, Lt, t_start=0):
    """cut[t] = True where the t-hop between t and t+1 (mod Lt) joins two different domains."""
    d = domain_of_t(extents, Lt, t_start)
    return d != np.roll(d, -1)


# ----------------------------------------------------------------------------- links
def fermion_links(U, bc_t=BC_ANTIPERIODIC, extents=None, t_start=0):
    """Links seen by the fermion hopping term: U with the time boundary phase on the t-links
    from t = Lt-1 and, for the domain operator, zero on every t-link that crosses a cut."""
    Ue = U.copy()
    Lt = U.shape[0]
    phase = {BC_PERIODIC: 1.0, BC_ANTIPERIODIC: -1.0, BC_OPEN: 0.0}[bc_t]
    Ue[Lt - 1, :, :, :, 3] *= phase
    if extents is not None:
        for t in np.nonzero(cut_after(extents, Lt, t_start))[0]:
            Ue[t, :, :, :, 3] = 0.0
    return Ue


def _shift(f, mu, n, axis_map):
    """g(x) = f(x + n mu) with periodic wrap-around."""
    return np.roll(f, -n, axis=axis_map[mu])


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _cmul(U, psi):
    """Colour matrix times spinor: (U psi)_{s a} = sum_b U_ab psi_{s b}, site-wise."""
    return np.matmul(psi, np.swapaxes(U, -1, -2))


def _smul(G, psi):
    """4x4 spin matrix on the spin index: (G psi)_{s c} = sum_t G_st psi_{t c}."""
    return np.matmul(G, psi)


def hopping(Ue, psi, dagger=False):
    """H psi (dagger=False) or H^dag psi (dagger=True) for fermion links Ue.

    H^dag has the projectors exchanged: (1 + gamma_mu) on the forward and (1 - gamma_mu) on the
    backward hop, with the same links.  psi: [..., t, z, y, x, 4, 3]."""
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    sgn = 1.0 if dagger else -1.0
    out = np.zeros_like(psi)
    for mu in range(4):
        Umu = Ue[:, :, :, :, mu]
        fwd = _cmul(Umu, _shift(psi, mu, 1, _SPINOR_AXIS))  # U_mu(x) psi(x+mu)
        out += _smul(one + sgn * g[mu], fwd)
        bwd = _shift(_cmul(_dag(Umu), psi), mu, -1, _SPINOR_AXIS)  # U_mu(x-mu)^dag psi(x-mu)
        out += _smul(one - sgn * g[mu], bwd)
    return out


# ----------------------------------------------------------------------------- clover
def clover_leaves(U, mu, nu):
    """Q_{mu nu}(x): sum of the four plaquettes in the (mu,nu) plane that start and end at x,
    all traversed in the same (mu then nu) orientation."""
    A = _LINK_AXIS
    Um = U[:, :, :, :, mu]
    Un = U[:, :, :, :, nu]
    sh = lambda f, m, n: _shift(f, m, n, A)
    mm = lambda *Ms: _mm_chain(Ms)
    l1 = mm(Um, sh(Un, mu, 1), _dag(sh(Um, nu, 1)), _dag(Un))
    l2 = mm(Un, _dag(sh(sh(Um, nu, 1), mu, -1)), _dag(sh(Un, mu, -1)), sh(Um, mu, -1))
    l3 = mm(_dag(sh(Um, mu, -1)), _dag(sh(sh(Un, mu, -1), nu, -1)), sh(sh(Um, mu, -1), nu, -1),
            sh(Un, nu, -1))
    l4 = mm(_dag(sh(Un, nu, -1)), sh(Um, nu, -1), sh(sh(Un, mu, 1), nu, -1), _dag(Um))
    return l1 + l2 + l3 + l4


def _mm_chain(Ms):
    out = Ms[0]
    for M in Ms[1:]:
        out = np.einsum("...ab,...bc->...ac", out, M)
    return out


def field_strength(U):
    """Fhat[t,z,y,x,plane,3,3] for the planes (x,y),(x,z),(x,t),(y,z),(y,t),(z,t)."""
    F = []
    for (mu, nu) in PLANES:
        Q = clover_leaves(U, mu, nu)
        F.append((Q - _dag(Q)) / 8.0)
    return np.stack(F, axis=4)


def clover_matrix(U, kappa, c_sw):
    """A(x) as a 12x12 matrix per site, index spin*3 + colour."""
    F = field_strength(U)
    A = np.zeros(U.shape[:4] + (12, 12), dtype=np.complex128)
    A += np.eye(12)
    for p, (mu, nu) in enumerate(PLANES):
        A += 1j * kappa * c_sw * np.einsum("st,...ab->...satb", sigma(mu, nu), F[..., p, :, :]
                                           ).reshape(U.shape[:4] + (12, 12))
    return A


def apply_site_matrix(A, psi):
    """Site-local 12x12 matrix on a spinor field."""
    sh = psi.shape
    flat = psi.reshape(sh[:-2] + (12, 1))
    return np.matmul(A, flat).reshape(sh)


# ----------------------------------------------------------------------------- operator
class WilsonClover:
    """D = A - kappa H on a fixed gauge field; ``extents`` (optional) makes it the Dirichlet
    domain operator D_Lambda (block diagonal over the domains of the tiling)."""

    def __init__(self, U, kappa, c_sw, bc_t=BC_ANTIPERIODIC, extents=None, t_start=0):
        self.U = U
        self.dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
        self.kappa = float(kappa)
        self.c_sw = float(c_sw)
        self.bc_t = bc_t
        self.extents = None if extents is None else [int(e) for e in extents]
        self.t_start = int(t_start)
        self.Ue = fermion_links(U, bc_t, self.extents, self.t_start)
        self.A = clover_matrix(U, kappa, c_sw)

    @property
    def volume(self):
        Lx, Ly, Lz, Lt = self.dims
        return Lx * Ly * Lz * Lt

    def apply(self, psi):
        return apply_site_matrix(self.A, psi) - self.kappa * hopping(self.Ue, psi, dagger=False)

    def apply_dagger(self, psi):
        Ah = np.conj(np.swapaxes(self.A, -1, -2))
        return apply_site_matrix(Ah, psi) - self.kappa * hopping(self.Ue, psi, dagger=True)

    def restricted(self, extents, t_start=0):
        """The domain operator D_Lambda of this operator for a tiling of the time axis whose
        domain 0 starts at t_start."""
        return WilsonClover(self.U, self.kappa, self.c_sw, self.bc_t, extents, t_start)

    def dense(self, chunk=512):
        """The full 12V x 12V matrix, columns ordered by (site, spin, colour)."""
        Lx, Ly, Lz, Lt = self.dims
        n = 12 * self.volume
        M = np.empty((n, n), dtype=np.complex128)
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            E = np.zeros((c1 - c0, n), dtype=np.complex128)
            E[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
            cols = self.apply(E.reshape(c1 - c0, Lt, Lz, Ly, Lx, 4, 3))
            M[:, c0:c1] = cols.reshape(c1 - c0, n).T
        return M


# ----------------------------------------------------------------------------- single sites
def apply_at_sites(U, kappa, c_sw, psi, sites, bc_t=BC_ANTIPERIODIC, extents=None, t_start=0):
    """(D psi)(x) at the listed sites only, from the definitions written out per site:

        (D psi)(x) = A(x) psi(x) - kappa sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                                                 + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
        A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) (Q_{mu nu}(x) - Q_{mu nu}(x)^dag) / 8,

    with the four clover leaves of Q built from explicit link coordinates, the time boundary phase
    on the t-hop between Lt-1 and 0, and (extents given) the t-hops between different domains
    removed.  For lattices too large to build the whole operator; it shares no code with
    WilsonClover beyond the gamma matrices.  psi: [t, z, y, x, 4, 3]; sites: iterable of (x, y, z, t).
    Returns [n_sites, 4, 3]."""
    Lt, Lz, Ly, Lx = U.shape[:4]
    L = (Lx, Ly, Lz, Lt)
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    phase = {BC_PERIODIC: 1.0, BC_ANTIPERIODIC: -1.0, BC_OPEN: 0.0}[bc_t]
    cut = cut_after(extents, Lt, t_start) if extents is not None else np.zeros(Lt, dtype=bool)

    def link(c, mu):
        return U[c[3] % Lt, c[2] % Lz, c[1] % Ly, c[0] % Lx, mu]

    def step(c, mu, n):
        d = list(c)
        d[mu] += n
        return d

    def dag(M):
        return M.conj().T

    def leaves(c, mu, nu):
        xpm, xpn, xmm, xmn = step(c, mu, 1), step(c, nu, 1), step(c, mu, -1), step(c, nu, -1)
        l1 = link(c, mu) @ link(xpm, nu) @ dag(link(xpn, mu)) @ dag(link(c, nu))
        l2 = link(c, nu) @ dag(link(step(xpn, mu, -1), mu)) @ dag(link(xmm, nu)) @ link(xmm, mu)
        l3 = dag(link(xmm, mu)) @ dag(link(step(xmm, nu, -1), nu)) @ link(step(xmm, nu, -1), mu) @ link(xmn, nu)
        l4 = dag(link(xmn, nu)) @ link(xmn, mu) @ link(step(xpm, nu, -1), nu) @ dag(link(c, mu))
        return l1 + l2 + l3 + l4

    def spinor(c):
        return psi[c[3] % Lt, c[2] % Lz, c[1] % Ly, c[0] % Lx]

    out = []
    for site in sites:
        c = [int(v) for v in site]
        A = np.eye(12, dtype=np.complex128)
        for (mu, nu) in PLANES:
            Q = leaves(c, mu, nu)
            F = (Q - dag(Q)) / 8.0
            A += 1j * kappa * c_sw * np.kron(sigma(mu, nu), F)
        res = (A @ spinor(c).reshape(12)).reshape(4, 3)
        for mu in range(4):
            cf = cb = 1.0
            if mu == 3:  # forward hop t -> t+1 and backward hop t-1 -> t
                t, tb = c[3], (c[3] - 1) % Lt
                cf = (phase if t == Lt - 1 else 1.0) * (0.0 if cut[t] else 1.0)
                cb = (phase if tb == Lt - 1 else 1.0) * (0.0 if cut[tb] else 1.0)
            fwd = spinor(step(c, mu, 1)) @ link(c, mu).T  # (U psi)_{s a} = sum_b U_ab psi_{s b}
            xm = step(c, mu, -1)
            bwd = spinor(xm) @ link(xm, mu).conj()        # (U^dag psi)_{s a} = sum_b conj(U_ba) psi_{s b}
            res = res - kappa * (cf * ((one - g[mu]) @ fwd) + cb * ((one + g[mu]) @ bwd))
        out.append(res)
    return np.array(out)
