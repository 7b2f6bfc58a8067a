"""Gauge-covariant parallel-transport network (oracle; test infrastructure).

The learned preconditioner has no counterpart in the paper: it is the oracle of the library's
network kernels.  Plain numpy, complex128.

A layer maps C_in channels of colour vectors h_c(x) to C_out channels:

    out_o(x) = sum_{p=0..8} sum_c W[p, o, c] (T_p h_c)(x)

with the paths  T_0 h(x) = h(x),  T_{1+mu} h(x) = U_mu(x) h(x+mu),  T_{5+mu} h(x) = U_mu(x-mu)^dag h(x-mu)
(mu = x, y, z, t), on the fermion links of ``oracle.dirac.fermion_links`` (time boundary phase
and, for the domain operator, the Dirichlet cuts).  Every path commutes with gauge
transformations, so the network is gauge covariant: N[U^G](G h) = G N[U](h).
The network is four linear layers with channel widths 4 -> 8 -> 8 -> 8 -> 4 (the four spin
components of a spinor in and out).  Loss of a batch: L = sum |N(h) - e|^2 / sum |e|^2 over the
sites selected by a mask.  Gradients are Wirtinger derivatives dL/d conj(W) (the real gradient
of the real and imaginary parts is twice their real and imaginary parts).

Pinned by (tests/test_oracle_nn.py): central finite differences of the loss, gauge covariance,
the adjoint identity <a, N b> = <N^dag a, b>, and the free-field momentum-space form of one layer.
"""
import numpy as np

WIDTHS = (4, 8, 8, 8, 4)
N_PATHS = 9

# numpy axis per mu for arrays [..., t, z, y, x, channel, colour]
_AX = {0: -3, 1: -4, 2: -5, 3: -6}


def _cmul(U, h):
    """(U h)_{c a} = sum_b U_ab h_{c b} site-wise; U [t,z,y,x,3,3], h [..., t,z,y,x,C,3]."""
    return np.matmul(h, np.swapaxes(U, -1, -2))


def transport(Ue, h, p):
    """T_p h for path p (see module docstring)."""
    if p == 0:
        return h
    mu = (p - 1) % 4
    Umu = Ue[:, :, :, :, mu]
    if p <= 4:
        return _cmul(Umu, np.roll(h, -1, axis=_AX[mu]))
    return np.roll(_cmul(np.conj(np.swapaxes(Umu, -1, -2)), h), 1, axis=_AX[mu])


def transport_adjoint(Ue, h, p):
    """T_p^dag: the forward hop of mu is adjoint to the backward hop of mu."""
    if p == 0:
        return h
    return transport(Ue, h, p + 4 if p <= 4 else p - 4)


def layer(W, Ue, h):
    """out_o = sum_p sum_c W[p, o, c] T_p h_c ; W [9, C_out, C_in]."""
    out = 0
    for p in range(N_PATHS):
        out = out + np.einsum("oc,...ca->...oa", W[p], transport(Ue, h, p))
    return out


def layer_adjoint(W, Ue, d):
    """The adjoint layer: sum_p sum_o conj(W[p, o, c]) T_p^dag d_o."""
    out = 0
    for p in range(N_PATHS):
        out = out + transport_adjoint(Ue, np.einsum("oc,...oa->...ca", np.conj(W[p]), d), p)
    return out


def forward(Ws, Ue, h):
    """All activations [h0, h1, ..., h4] of the network."""
    acts = [h]
    for W in Ws:
        acts.append(layer(W, Ue, acts[-1]))
    return acts


def loss_and_grad(Ws, Ue, h, target, mask):
    """Loss L and Wirtinger gradients dL/dconj(W_l) for each layer.  mask [t,z,y,x] selects sites."""
    acts = forward(Ws, Ue, h)
    m = mask[..., None, None]
    diff = (acts[-1] - target) * m
    norm = np.sum(np.abs(target * m) ** 2)
    L = np.sum(np.abs(diff) ** 2) / norm
    delta = diff / norm  # dL / d conj(out)
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        G = np.zeros_like(Ws[l])
        for p in range(N_PATHS):
            Th = transport(Ue, acts[l], p)
            sum_axes = tuple(range(delta.ndim - 2)) + (delta.ndim - 1,)
            G[p] = np.tensordot(delta, np.conj(Th), axes=(sum_axes, sum_axes))
        grads[l] = G
        if l > 0:
            delta = layer_adjoint(Ws[l], Ue, delta)
    return L, grads


def init_weights(seed, scale=0.1):
    """Deterministic initial weights: identity-like path 0 plus small random mixing."""
    rng = np.random.default_rng(seed)
    Ws = []
    for cin, cout in zip(WIDTHS[:-1], WIDTHS[1:]):
        W = scale * (rng.normal(size=(N_PATHS, cout, cin)) + 1j * rng.normal(size=(N_PATHS, cout, cin)))
        W[0] += np.eye(cout, cin)
        Ws.append(W)
    return Ws
