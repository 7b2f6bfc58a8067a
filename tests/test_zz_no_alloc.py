"""lqcd_disc_correlator_noalloc, the entry point for callers that cannot allocate GPU memory
(hosts that reserve all device memory up front, loops where an allocation would synchronise the
device): called through the C ABI
with caller-owned device buffers, twice in a row on different inputs, it must give the results of
the allocating lqcd_disc_correlator.  This file is collected last on purpose, so a failure here
does not hide the other tests of a run that stops at the first failure."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2609_37049_b300 import Context, lqcd  # noqa: E402


def _loops(n_cfg, n_g, T, seed):
    rng = np.random.default_rng(seed)
    mk = lambda: torch.from_numpy(rng.normal(size=(n_cfg, n_g, T)) + 1j * rng.normal(size=(n_cfg, n_g, T))).cuda()
    return mk(), mk(), mk(), mk()


def _outputs(n_g, T):
    z = lambda *s: torch.zeros(s, dtype=torch.complex128, device="cuda")
    return dict(C=z(n_g, T, T), Cdd=z(n_g, T, T), dC=z(n_g, T, T), C_avg=z(n_g, T), dC_avg=z(n_g, T),
                valid=torch.zeros((T, T), dtype=torch.int32, device="cuda"),
                n_valid=torch.zeros(T, dtype=torch.int32, device="cuda"))


def _noalloc(L, Lt, Ld, Ltd, T, dom, vev, out, terms):
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    n_cfg, n_g = L.shape[0], L.shape[1]
    return lqcd.lib().lqcd_disc_correlator_noalloc(
        p(L), p(Lt), p(Ld), p(Ltd), n_cfg, n_g, T, p(dom), int(vev), p(out["C"]), p(out["Cdd"]), p(out["dC"]),
        p(out["C_avg"]), p(out["dC_avg"]), p(out["valid"]), p(out["n_valid"]), p(terms),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    T, ext, n_g = 16, [4, 6, 6], 3
    ctx = Context((4, 4, 4, T))
    ctx.set_domains(ext)
    dom = torch.tensor(np.repeat(np.arange(len(ext)), ext), dtype=torch.int32, device="cuda")
    for n_cfg, seed, vev in ((5, 1, True), (3, 2, False)):
        L, Lt, Ld, Ltd = _loops(n_cfg, n_g, T, seed)
        ref = _outputs(n_g, T)
        ref_terms = torch.zeros((4, n_g, T, T), dtype=torch.complex128, device="cuda")
        ctx.disc_correlator(L, Lt, Ld, Ltd, vev, ref, terms=ref_terms)
        out = _outputs(n_g, T)
        terms = torch.full((4, n_g, T, T), float("nan"), dtype=torch.complex128, device="cuda")
        rc = _noalloc(L, Lt, Ld, Ltd, T, dom, vev, out, terms)
        assert rc == lqcd.LQCD_OK, lqcd.lib().lqcd_last_error(None)
        torch.cuda.synchronize()
        scale = ref["C"].abs().max().item()
        for k in ("C", "Cdd", "dC", "C_avg", "dC_avg"):
            assert (out[k] - ref[k]).abs().max().item() <= 1e-13 * scale, k
        assert (terms - ref_terms).abs().max().item() <= 1e-13 * scale
        assert torch.equal(out["valid"], ref["valid"]) and torch.equal(out["n_valid"], ref["n_valid"])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    T, n_g, n_cfg = 16, 16, 257  # 65792 loop entries > 65536
    L = torch.zeros((n_cfg, n_g, T), dtype=torch.complex128, device="cuda")
    dom = torch.zeros(T, dtype=torch.int32, device="cuda")
    out = _outputs(n_g, T)
    terms = torch.zeros((4, n_g, T, T), dtype=torch.complex128, device="cuda")
    rc = _noalloc(L, L, L, L, T, dom, True, out, terms)
    assert rc == lqcd.LQCD_ERR_INVALID_ARG
    assert b"65536" in lqcd.lib().lqcd_last_error(None)
