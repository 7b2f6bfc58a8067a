"""ctypes binding of the lqcd C ABI (include/lqcd.h): the same entry-point names, argument
marshalling only.  Arrays may be numpy arrays (host memory, LQCD_HOST) or torch CUDA tensors
(device memory, LQCD_DEVICE); complex arrays must be complex128 and C-contiguous.

Importing this module loads liblqcd.so from the package directory and raises if it is missing:
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblqcd.so")

LQCD_OK = 0
LQCD_ERR_INVALID_ARG = 1
LQCD_ERR_NOT_CONVERGED = 2
LQCD_ERR_CUDA = 3
LQCD_ERR_OOM = 4
LQCD_ERR_TIMEOUT = 5
LQCD_ERR_NAN = 6
LQCD_ERR_STATE = 7
LQCD_BC_PERIODIC, LQCD_BC_ANTIPERIODIC, LQCD_BC_OPEN = 0, 1, 2
LQCD_HOST, LQCD_DEVICE = 0, 1
LQCD_MODE_FULL, LQCD_MODE_DOMAIN = 0, 1
LQCD_SINKS_DIAG, LQCD_SINKS_ALL, LQCD_SINKS_DIAG_SRCV = 0, 1, 2
LQCD_SOLVER_BICGSTAB64, LQCD_SOLVER_MIXED, LQCD_SOLVER_FGCR_NN = 0, 1, 2
LQCD_PREC_F64, LQCD_PREC_F32, LQCD_PREC_F16, LQCD_PREC_DF = 0, 1, 2, 3

EXPORTED = [
    "lqcd_default_params", "lqcd_create", "lqcd_destroy", "lqcd_set_stream", "lqcd_last_error",
    "lqcd_gauge_upload", "lqcd_set_domains", "lqcd_set_domains_at", "lqcd_dirac_apply", "lqcd_solve_full",
    "lqcd_solve_domain", "lqcd_perambulator", "lqcd_loops", "lqcd_disc_correlator",
    "lqcd_dslash_bench", "lqcd_kernel_launches", "lqcd_laplace_eigs", "lqcd_disc_correlator_noalloc",
    "lqcd_phase_times", "lqcd_nn_num_weights", "lqcd_nn_set_weights", "lqcd_nn_get_weights", "lqcd_nn_apply",
    "lqcd_nn_loss_grad", "lqcd_nn_train", "lqcd_tune_dslash", "lqcd_set_dslash_variant", "lqcd_schur_apply",
    "lqcd_conn_correlator", "lqcd_nr_estimator", "lqcd_ape_smear", "lqcd_smeared_links",
    "lqcd_perambulator_cols", "lqcd_window_average", "lqcd_nn_apply_tc", "lqcd_nn_loss_grad_bf16",
    "lqcd_release_workspace",
]

NN_WIDTHS = (4, 8, 8, 8, 4)


def nn_flatten(Ws):
    """Network weights [W_l (9, C_out, C_in) complex] -> flat float32 (re, im) array of the C ABI."""
    return np.ascontiguousarray(np.concatenate([np.asarray(W, dtype=np.complex64).ravel() for W in Ws]).view(
        np.float32))


def nn_initial_weights(seed, scale=0.05):
    """Starting weights for training: the identity on the path-0 channel block plus small
    seeded Gaussian complex noise on every path (numpy; layers [9, C_out, C_in])."""
    rng = np.random.default_rng(seed)
    Ws = []
    for cin, cout in zip(NN_WIDTHS[:-1], NN_WIDTHS[1:]):
        W = scale * (rng.normal(size=(9, cout, cin)) + 1j * rng.normal(size=(9, cout, cin)))
        W[0] += np.eye(cout, cin)
        Ws.append(W)
    return Ws


def nn_unflatten(flat):
    c = np.asarray(flat, dtype=np.float32).view(np.complex64)
    out, o = [], 0
    for cin, cout in zip(NN_WIDTHS[:-1], NN_WIDTHS[1:]):
        n = 9 * cout * cin
        out.append(c[o:o + n].reshape(9, cout, cin).astype(np.complex128))
        o += n
    return out


def kernel_launches():
    """Kernels this library has queued in this process (direct launches + graph kernel nodes)."""
    return int(_lib.lqcd_kernel_launches())


class lqcd_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("solver", ctypes.c_int),
                ("inner_prec", ctypes.c_int), ("rhs_block", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("check_every", ctypes.c_int), ("gcr_nkrylov", ctypes.c_int),
                ("precond_iters", ctypes.c_int), ("pipeline", ctypes.c_int),
                ("projection", ctypes.c_int), ("residual", ctypes.c_int)]


class lqcd_solve_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.POINTER(ctypes.c_int)), ("true_resid", ctypes.POINTER(ctypes.c_double)),
                ("n_seg", ctypes.c_int), ("outer_cycles", ctypes.c_int), ("total_iters", ctypes.c_longlong),
                ("dslash_calls", ctypes.c_longlong), ("max_true_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("fallback", ctypes.c_int), ("device_loops", ctypes.c_int)]


class LqcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lqcd error %d: %s" % (code, msg))
        self.code = code


def load_library(path=_LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("liblqcd.so not built (run python paper_2609_37049_b300/build.py): %s" % path)
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    c_int_p = ctypes.POINTER(ctypes.c_int)
    sig = {
        "lqcd_default_params": (None, [ctypes.POINTER(lqcd_solve_params)]),
        "lqcd_create": (ip, [ctypes.POINTER(vp), c_int_p, ip, vp]),
        "lqcd_destroy": (ip, [vp]),
        "lqcd_set_stream": (ip, [vp, vp]),
        "lqcd_last_error": (ctypes.c_char_p, [vp]),
        "lqcd_gauge_upload": (ip, [vp, vp, ip, ctypes.c_double, ctypes.c_double]),
        "lqcd_set_domains": (ip, [vp, c_int_p, ip]),
        "lqcd_set_domains_at": (ip, [vp, ip, c_int_p, ip]),
        "lqcd_dirac_apply": (ip, [vp, vp, vp, ip, ip, ip]),
        "lqcd_schur_apply": (ip, [vp, ip, vp, vp, ip, ip, ip]),
        "lqcd_solve_full": (ip, [vp, vp, vp, ip, ip, ctypes.POINTER(lqcd_solve_params),
                                 ctypes.POINTER(lqcd_solve_stats)]),
        "lqcd_solve_domain": (ip, [vp, vp, vp, ip, ip, ctypes.POINTER(lqcd_solve_params),
                                   ctypes.POINTER(lqcd_solve_stats)]),
        "lqcd_perambulator": (ip, [vp, vp, ip, c_int_p, ip, ip, ip, ip, vp,
                                   ctypes.POINTER(lqcd_solve_params), ctypes.POINTER(lqcd_solve_stats)]),
        "lqcd_perambulator_cols": (ip, [vp, vp, ip, c_int_p, ip, ip, ip, ip, ip, ip, vp,
                                        ctypes.POINTER(lqcd_solve_params), ctypes.POINTER(lqcd_solve_stats)]),
        "lqcd_loops": (ip, [vp, vp, ip, ip, c_int_p, ip, vp, vp, vp, ip]),
        "lqcd_window_average": (ip, [vp, vp, vp, vp, ip, ip, ip, vp, vp, vp, vp, ip]),
        "lqcd_disc_correlator": (ip, [vp, vp, vp, vp, vp, ip, ip, ip, vp, vp, vp, vp, vp, vp, vp, vp, ip]),
        "lqcd_ape_smear": (ip, [vp, ctypes.c_double, ip]),
        "lqcd_smeared_links": (ip, [vp, vp, ip]),
        "lqcd_conn_correlator": (ip, [vp, vp, ip, c_int_p, ip, c_int_p, ip, vp, vp, ip]),
        "lqcd_nr_estimator": (ip, [vp, vp, vp, vp, ip, ip, c_int_p, vp, ip]),
        "lqcd_dslash_bench": (ip, [vp, ip, ip, ip, ip, dp, dp]),
        "lqcd_kernel_launches": (ctypes.c_longlong, []),
        "lqcd_laplace_eigs": (ip, [vp, ip, vp, vp, ip, ctypes.c_double, c_int_p]),
        "lqcd_disc_correlator_noalloc": (ip, [vp, vp, vp, vp, ip, ip, ip, vp, ip, vp, vp, vp, vp, vp, vp, vp, vp,
                                              vp]),
        "lqcd_phase_times": (ip, [vp, ctypes.c_char_p, ip, ip]),
        "lqcd_tune_dslash": (ip, [vp, ip, ip, c_int_p, ctypes.POINTER(ctypes.c_double)]),
        "lqcd_set_dslash_variant": (ip, [vp, ip, ip, ip]),
        "lqcd_nn_num_weights": (ip, []),
        "lqcd_nn_set_weights": (ip, [vp, vp]),
        "lqcd_nn_get_weights": (ip, [vp, vp]),
        "lqcd_nn_apply": (ip, [vp, vp, vp, ip, ip, ip]),
        "lqcd_nn_apply_tc": (ip, [vp, vp, vp, ip, ip, ip]),
        "lqcd_nn_loss_grad": (ip, [vp, vp, vp, ip, ip, ip, ip, ctypes.POINTER(ctypes.c_double), vp]),
        "lqcd_nn_train": (ip, [vp, ip, ip, ip, ctypes.c_double, ip, ctypes.c_uint, vp]),
        "lqcd_nn_loss_grad_bf16": (ip, [vp, vp, vp, ip, ip, ip, ip, ctypes.POINTER(ctypes.c_double), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load_library()


def lib():
    return _lib


# ----------------------------------------------------------------------------- marshalling
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _where(*arrays):
    kinds = {_is_torch(a) for a in arrays if a is not None}
    if len(kinds) > 1:
        raise TypeError("mix of host (numpy) and device (torch) arrays")
    if kinds == {True}:
        for a in arrays:
            if a is not None and not a.is_cuda:
                raise TypeError("torch tensors must live on the GPU")
        return LQCD_DEVICE
    return LQCD_HOST


def _ptr(a, dtype=np.complex128):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous %s" % np.dtype(dtype).name)
    return ctypes.c_void_p(a.ctypes.data)


def _int_array(vals):
    arr = (ctypes.c_int * len(vals))(*[int(v) for v in vals])
    return arr


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def default_params(**kw):
    p = lqcd_solve_params()
    _lib.lqcd_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Stats:
    """Host-side holder for lqcd_solve_stats plus its per-RHS arrays."""

    def __init__(self, nrhs, nseg):
        self.iters = np.zeros(nrhs, dtype=np.int32)
        self.true_resid = np.zeros(nrhs * nseg, dtype=np.float64)
        self.c = lqcd_solve_stats()
        self.c.iters = self.iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        self.c.true_resid = self.true_resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def __getattr__(self, k):
        return getattr(self.c, k)


class Context:
    """One lqcd context: a lattice of extents dims = (Lx, Ly, Lz, Lt) on the current GPU."""

    def __init__(self, dims, bc_t=LQCD_BC_ANTIPERIODIC, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.h = ctypes.c_void_p()
        L = _int_array(self.dims)
        rc = _lib.lqcd_create(ctypes.byref(self.h), L, int(bc_t), stream or _current_stream())
        if rc != LQCD_OK:
            raise LqcdError(rc, _lib.lqcd_last_error(None).decode())
        self.extents = [self.dims[3]]
        self.t_start = 0

    @property
    def volume(self):
        Lx, Ly, Lz, Lt = self.dims
        return Lx * Ly * Lz * Lt

    def close(self):
        if self.h:
            _lib.lqcd_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != LQCD_OK and rc not in allow:
            raise LqcdError(rc, _lib.lqcd_last_error(self.h).decode())
        return rc

    def set_stream(self, stream=None):
        return self._check(_lib.lqcd_set_stream(self.h, stream or _current_stream()))

    def gauge_upload(self, links, kappa, c_sw):
        return self._check(_lib.lqcd_gauge_upload(self.h, _ptr(links), _where(links), float(kappa),
                                                  float(c_sw)))

    def set_domains(self, extents, t_start=0):
        """Tile the time axis by domains of the given extents, domain 0 starting at t_start."""
        rc = self._check(_lib.lqcd_set_domains_at(self.h, int(t_start), _int_array(extents), len(extents)))
        self.extents = [int(e) for e in extents]
        self.t_start = int(t_start)
        return rc

    def dirac_apply(self, psi, out, domain_restricted=False):
        nrhs = psi.shape[0]
        return self._check(_lib.lqcd_dirac_apply(self.h, _ptr(psi), _ptr(out), nrhs, int(domain_restricted),
                                                 _where(psi, out)))

    def schur_apply(self, prec, psi, out, domain_restricted=False):
        """out_e = M psi_e, the even-odd Schur operator in storage precision prec (odd sites of out = 0)."""
        nrhs = psi.shape[0]
        return self._check(_lib.lqcd_schur_apply(self.h, int(prec), _ptr(psi), _ptr(out), nrhs,
                                                 int(domain_restricted), _where(psi, out)))

    def solve(self, b, x, params=None, domain=False, stats=None, allow_not_converged=False):
        nrhs = b.shape[0]
        p = params or default_params()
        f = _lib.lqcd_solve_domain if domain else _lib.lqcd_solve_full
        st = stats.c if stats is not None else None
        if stats is not None:
            nseg = len(self.extents) if domain else 1
            if stats.iters.size < nrhs or stats.true_resid.size < nrhs * nseg:
                raise ValueError("Stats arrays too small for %d right-hand sides x %d segments" % (nrhs, nseg))
        rc = f(self.h, _ptr(b), _ptr(x), nrhs, _where(b, x), ctypes.byref(p),
               ctypes.byref(st) if st is not None else None)
        return self._check(rc, allow=(LQCD_ERR_NOT_CONVERGED,) if allow_not_converged else ())

    def perambulator(self, Vt, n_ev, t_src, tau, mode=LQCD_MODE_FULL, sinks=LQCD_SINKS_DIAG, params=None,
                     stats=None):
        p = params or default_params()
        st = stats.c if stats is not None else None
        rc = _lib.lqcd_perambulator(self.h, _ptr(Vt), int(n_ev), _int_array(t_src), len(t_src), int(mode),
                                    int(sinks), _where(Vt, tau), _ptr(tau), ctypes.byref(p),
                                    ctypes.byref(st) if st is not None else None)
        return self._check(rc)

    def perambulator_cols(self, Vt, n_ev, t_src, tau, j0, nj, mode=LQCD_MODE_FULL, sinks=LQCD_SINKS_DIAG,
                          params=None, stats=None, allow=()):
        """Columns j in [j0, j0 + nj) (all four source spins) of the perambulators; other entries of
        tau are left as they were."""
        p = params or default_params()
        st = stats.c if stats is not None else None
        rc = _lib.lqcd_perambulator_cols(self.h, _ptr(Vt), int(n_ev), _int_array(t_src), len(t_src), int(mode),
                                         int(sinks), int(j0), int(nj), _where(Vt, tau), _ptr(tau), ctypes.byref(p),
                                         ctypes.byref(st) if st is not None else None)
        return self._check(rc, allow=allow)

    def loops(self, tau, n_ev, n_t, gamma_ids, L, Lt, weights=None):
        return self._check(_lib.lqcd_loops(self.h, _ptr(tau), int(n_ev), int(n_t), _int_array(gamma_ids),
                                           len(gamma_ids), _ptr(weights, np.float64), _ptr(L), _ptr(Lt),
                                           _where(tau, L, Lt, weights)))

    def disc_correlator(self, L, Lt, Ld, Ltd, vev, out, terms=None):
        """out: dict with C, Cdd, dC, C_avg, dC_avg (complex), valid, n_valid (int32)."""
        n_cfg, n_g = L.shape[0], L.shape[1]
        w = _where(L, Lt, Ld, Ltd, out["C"])
        return self._check(_lib.lqcd_disc_correlator(
            self.h, _ptr(L), _ptr(Lt), _ptr(Ld), _ptr(Ltd), n_cfg, n_g, int(vev), _ptr(out["C"]),
            _ptr(out["Cdd"]), _ptr(out["dC"]), _ptr(out["C_avg"]), _ptr(out["dC_avg"]),
            _ptr(out["valid"], np.int32), _ptr(out["n_valid"], np.int32), _ptr(terms), w))

    def window_average(self, C, dC, valid, t_lo, t_hi, out):
        """Bulk-window averages: out dict with C_avg, dC_avg (complex [n_gamma, Lt]) and n_pairs,
        n_valid (int32 [Lt]) over source and sink both in [t_lo, t_hi]."""
        return self._check(_lib.lqcd_window_average(
            self.h, _ptr(C), _ptr(dC), _ptr(valid, np.int32), C.shape[0], int(t_lo), int(t_hi), _ptr(out["C_avg"]),
            _ptr(out["dC_avg"]), _ptr(out["n_pairs"], np.int32), _ptr(out["n_valid"], np.int32),
            _where(C, dC, valid, out["C_avg"])))

    def ape_smear(self, alpha, n_iter):
        """Smear the spatial links (used by laplace_eigs); n_iter = 0 drops the smearing."""
        return self._check(_lib.lqcd_ape_smear(self.h, float(alpha), int(n_iter)))

    def smeared_links(self, out):
        """out[t, z, y, x, k, 3, 3] (k = x, y, z): the smeared spatial links."""
        return self._check(_lib.lqcd_smeared_links(self.h, _ptr(out), _where(out)))

    def conn_correlator(self, tau_all, n_ev, t_src, gamma_ids, C, C_avg=None):
        """C[g, x0, k] (and C_avg[g, dt]) from all-sink perambulators tau_all[k, t', i, a, j, b]."""
        n_t = len(t_src)
        return self._check(_lib.lqcd_conn_correlator(
            self.h, _ptr(tau_all), int(n_ev), _int_array(t_src), n_t, _int_array(gamma_ids), len(gamma_ids),
            _ptr(C), _ptr(C_avg), _where(tau_all, C)))

    def nr_estimator(self, C_conn_avg, C_disc_avg, dC_avg, delta_of_dt, out):
        """out[g, dt] = C_conn_avg + (dC_avg[delta_of_dt[dt]] or C_disc_avg where the index is -1)."""
        n_g = C_conn_avg.shape[0]
        n_delta = 0 if dC_avg is None else dC_avg.shape[0]
        return self._check(_lib.lqcd_nr_estimator(
            self.h, _ptr(C_conn_avg), _ptr(C_disc_avg), _ptr(dC_avg), n_delta, n_g, _int_array(delta_of_dt),
            _ptr(out), _where(C_conn_avg, C_disc_avg, out)))

    # ---- autotuning
    def tune_dslash(self, prec, nrhs):
        bt, ms = ctypes.c_int(), ctypes.c_double()
        self._check(_lib.lqcd_tune_dslash(self.h, int(prec), int(nrhs), ctypes.byref(bt), ctypes.byref(ms)))
        return bt.value, ms.value

    def release_workspace(self):
        """Free the library's work buffers (re-created on demand), e.g. before large torch allocations."""
        return self._check(_lib.lqcd_release_workspace(self.h))

    def set_dslash_variant(self, prec, nrhs, variant):
        return self._check(_lib.lqcd_set_dslash_variant(self.h, int(prec), int(nrhs), int(variant)))

    # ---- learned preconditioner
    def nn_set_weights(self, Ws):
        flat = nn_flatten(Ws)
        return self._check(_lib.lqcd_nn_set_weights(self.h, ctypes.c_void_p(flat.ctypes.data)))

    def nn_get_weights(self):
        flat = np.zeros(2 * _lib.lqcd_nn_num_weights(), dtype=np.float32)
        self._check(_lib.lqcd_nn_get_weights(self.h, ctypes.c_void_p(flat.ctypes.data)))
        return nn_unflatten(flat)

    def nn_apply(self, x, out, domain=False):
        return self._check(_lib.lqcd_nn_apply(self.h, _ptr(x, np.complex64), _ptr(out, np.complex64), x.shape[0],
                                              int(domain), _where(x, out)))

    def nn_apply_tc(self, x, out, domain=False):
        """The inference path of the preconditioner: BF16 weights and activations, channel mixing on
        the tensor cores, FP32 accumulation."""
        return self._check(_lib.lqcd_nn_apply_tc(self.h, _ptr(x, np.complex64), _ptr(out, np.complex64), x.shape[0],
                                                 int(domain), _where(x, out)))

    def nn_loss_grad(self, x, target, domain=False, even_only=False, bf16=False):
        """Loss and dL/dconj(W): FP32 kernels, or (bf16=True) the BF16 training kernels."""
        loss = ctypes.c_double()
        g = np.zeros(2 * _lib.lqcd_nn_num_weights(), dtype=np.float32)
        f = _lib.lqcd_nn_loss_grad_bf16 if bf16 else _lib.lqcd_nn_loss_grad
        self._check(f(self.h, _ptr(x, np.complex64), _ptr(target, np.complex64), x.shape[0], int(domain),
                      int(even_only), _where(x, target), ctypes.byref(loss), ctypes.c_void_p(g.ctypes.data)))
        return loss.value, nn_unflatten(g)

    def nn_train(self, n_pairs, epochs, batch, lr, domain=False, seed=1):
        hist = np.zeros(epochs, dtype=np.float64)
        self._check(_lib.lqcd_nn_train(self.h, int(n_pairs), int(epochs), int(batch), float(lr), int(domain),
                                       int(seed), ctypes.c_void_p(hist.ctypes.data)))
        return hist

    def phase_times(self, reset=False):
        """GPU milliseconds per solver phase (needs LQCD_PHASE_TIMING=1 at context creation)."""
        import json
        buf = ctypes.create_string_buffer(8192)
        self._check(_lib.lqcd_phase_times(self.h, buf, 8192, int(reset)))
        return json.loads(buf.value.decode())

    def laplace_eigs(self, n_ev, V, lam, tol=1e-10):
        """Lowest n_ev Laplacian eigenpairs per timeslice into V [Lt][n_ev][L3][3], lam [Lt][n_ev]."""
        it = ctypes.c_int()
        self._check(_lib.lqcd_laplace_eigs(self.h, int(n_ev), _ptr(V), _ptr(lam, np.float64), _where(V, lam),
                                           float(tol), ctypes.byref(it)))
        return it.value

    def dslash_bench(self, prec, nrhs, n_iter=20, flush_l2=True):
        """(ms per launch, algorithmic bytes per launch) of the eo hopping + clover-inverse kernel."""
        ms, by = ctypes.c_double(), ctypes.c_double()
        self._check(_lib.lqcd_dslash_bench(self.h, int(prec), int(nrhs), int(n_iter), int(flush_l2),
                                           ctypes.byref(ms), ctypes.byref(by)))
        return ms.value, by.value
