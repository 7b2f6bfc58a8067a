"""Benchmark of the distillation subtraction-estimator hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload scale|mixed|uneven|learned]

Default workload (scale run): 48^3 x 96 lattice, SU(3) links U = exp(i 0.6 H) (Philox-seeded
Gaussian traceless Hermitian H, seed 5001), clover-Wilson kappa = 0.126, c_sw = 1.7, antiperiodic
in time; N_ev = 128 seeded orthonormal colour vectors (seed 5002) on the 16 source timeslices
t = 0, 6, ..., 90; 24 time domains of extent 4 (extents 8 and 12 measured beside it);
Gamma = {gamma_5, 1}.  Synthetic data; it stands in for the paper's 96 x 32^3 ensemble with its
200 Laplacian eigenvectors.

One step = the whole hot path for one RHS block of each operator (rhs_block right-hand sides:
rhs_block / 4 source colour vectors x 4 spins):
  full-operator perambulator columns of a block at one source timeslice   rhs_block RHS
  domain-operator columns of a block for one source group (one source timeslice per domain) as
  one multi-site solve                                   rhs_block x (domains served) RHS
  loops of both, and the full / factorised / subtracted correlators of the configuration.
Consecutive steps walk the full operator's source timeslices, then its blocks, and the domain
operator's groups, then its blocks, so no step repeats the work of an earlier one.  Every solve reaches FP64 true
residual <= 1e-10 (FP64 defect correction around FP32 BiCGStab).
metric value = RHS solved per second (full + domain; each domain of a multi-site solve counts
once), inputs resident in HBM.

The JSON line also carries: e2e (the same steps through the C ABI with pinned host buffers: the
gauge field and the step's colour vectors uploaded and perambulators / loops / correlators
downloaded every step), the plain FP64 solver and the other solvers on one sample (the
"vs plain" ratio), the dslash roofline of the dominant kernel, domain extents 8 and 12, a CPU
baseline of the oracle, clocks sampled during the timed region and the number of library kernels
launched in it.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "scale": dict(
        title="48^3x96 scale run: batched mixed-precision distillation, full + domain solves",
        dims=(48, 48, 48, 96), eps=0.6, kappa=0.126, csw=1.7, n_ev=128, t_src=list(range(0, 96, 6)),
        extents=[4] * 24, sweep={8: [8] * 12, 12: [12] * 8}, gauge_seed=5001, cv_seed=5002,
        sources="seeded orthonormal colour vectors (Cholesky-QR twice)", rhs_block=16, pipeline=1,
        solver_sample_rhs=4),
    "mixed": dict(
        title="16^3x32 mixed-precision distillation, full + domain solves",
        dims=(16, 16, 16, 32), eps=0.5, kappa=0.125, csw=1.6, n_ev=32, t_src=list(range(32)),
        extents=[4] * 8, sweep={}, gauge_seed=2001, cv_seed=2002,
        sources="lowest Laplacian eigenvectors (GPU eigensolver)", rhs_block=64, pipeline=1,
        solver_sample_rhs=64),
    "uneven": dict(
        title="24^3x48 batched uneven domains 6/8/10/6/8/10",
        dims=(24, 24, 24, 48), eps=0.5, kappa=0.125, csw=1.6, n_ev=64, t_src=list(range(48)),
        extents=[6, 8, 10, 6, 8, 10], sweep={}, gauge_seed=3001, cv_seed=3002,
        sources="seeded orthonormal colour vectors (Cholesky-QR twice)", rhs_block=64, pipeline=1,
        solver_sample_rhs=16),
    "learned": dict(
        title="32^3x64 learned preconditioner: flexible GCR with the gauge-covariant network",
        dims=(32, 32, 32, 64), eps=0.6, kappa=0.126, csw=1.7, n_ev=64, t_src=list(range(0, 64, 4)),
        extents=[4] * 16, sweep={}, gauge_seed=4001, cv_seed=4002,
        sources="seeded orthonormal colour vectors (Cholesky-QR twice)", rhs_block=16, pipeline=1,
        solver_sample_rhs=16, learned=dict(pairs=2000, batch=4, epochs=2, lr=2e-3, seed=41)),
}
GAMMAS = [5, 0]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale", choices=sorted(WORKLOADS))
    ap.add_argument("--rhs-block", type=int, default=0, help="override the workload's RHS block")
    ap.add_argument("--pipeline", type=int, default=0, help="override the workload's batches in flight (1 or 2)")
    ap.add_argument("--projection", type=int, default=0, help="0: double-float projection (default), 1: FP64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="drive the solver loops from the host with plain launches (ncu does not profile the "
                         "kernel nodes of graphs with device-side loops; the kernels are the same)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement (tuning runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed steps and e2e (no solver comparison, sweep or roofline)")
    ap.add_argument("--profile-nn", action="store_true",
                    help="time the network preconditioner (FP32 CUDA-core and tensor-core forms) on the workload's "
                         "lattice with --dslash-nrhs samples (default 16), a few applications each (small command "
                         "for ncu)")
    ap.add_argument("--profile-dslash", action="store_true",
                    help="only time the dslash kernels of the workload (small command for ncu captures)")
    ap.add_argument("--profile-step", action="store_true",
                    help="set up the workload, run one warm step and one step inside the NVTX range "
                         "'bench_step' (for ncu --nvtx-include), print no bench line")
    ap.add_argument("--dslash-variant", type=int, default=-1,
                    help="with --profile-dslash: time only this launch variant (default: all)")
    ap.add_argument("--dslash-nrhs", type=int, default=0, help="with --profile-dslash: RHS count")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle baseline
def stored_cgnr_iterations(wl):
    """The oracle's CGNR iteration count to true residual 1e-10 at the workload's couplings, as
    measured by oracle/cgnr_iterations.py (largest lattice available with those couplings)."""
    path = os.path.join(ROOT, "oracle", "cgnr_iterations.json")
    try:
        with open(path) as f:
            data = json.load(f)
    except OSError:
        return None
    best = None
    for e in data.values():
        if abs(e["eps"] - wl["eps"]) < 1e-12 and abs(e["kappa"] - wl["kappa"]) < 1e-12 and \
                abs(e["c_sw"] - wl["csw"]) < 1e-12 and e["true_resid"] <= 1e-10:
            if best is None or np.prod(e["dims"]) > np.prod(best["dims"]):
                best = e
    return best


_ORACLE_POOL = None
_ORACLE_SETUP = {}


def _oracle_pool():
    """One process per host core (spawned: the parent holds a CUDA context), numpy single-threaded
    in each, created once and reused."""
    global _ORACLE_POOL
    if _ORACLE_POOL is None:
        import multiprocessing as mp
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            _ORACLE_POOL = mp.get_context("spawn").Pool(os.cpu_count() or 1)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return _ORACLE_POOL


def _oracle_rhs(task):
    """One oracle RHS on the 16^3 x 32 sample field: seconds per CGNR iteration over the budget, and
    the projection's seconds (runs in a pool worker)."""
    from lqcd_inputs import colour_vectors, gauge_field
    from oracle.dirac import WilsonClover
    from oracle.distill import project, sources
    from oracle.solve import cgnr
    wl, budget_s, j, n = task
    sdims = (16, 16, 16, 32)
    key = (wl["eps"], wl["kappa"], wl["csw"], wl["gauge_seed"], wl["cv_seed"], n)
    if key not in _ORACLE_SETUP:
        op = WilsonClover(gauge_field(sdims, wl["eps"], wl["gauge_seed"]), wl["kappa"], wl["csw"])
        V0 = colour_vectors(sdims, (n + 3) // 4, wl["cv_seed"], timeslices=[0])
        _ORACLE_SETUP.clear()
        _ORACLE_SETUP[key] = (op, V0)
    op, V0 = _ORACLE_SETUP[key]
    b = sources(V0[0], 0, sdims)[j: j + 1]  # colour vector j // 4, spin j % 4
    k, x = 0, None
    t1 = time.time()
    while True:
        x, _ = cgnr(op, b, tol=1e-30, max_iter=2, x0=x)
        k += 2
        if time.time() - t1 > budget_s or k >= 40:
            break
    t_iter = (time.time() - t1) / k
    t2 = time.time()
    project(V0[0], x, 0)
    return t_iter, time.time() - t2, k


def cpu_baseline(wl, budget_s=20.0, setup=None):
    """The oracle, as it stands, on a bounded sample of the workload, on every host core.

    Sample: one process per host core, each running the oracle's CGNR on its own right-hand side
    (t = 0, colour vector j // 4, spin j % 4) of a 16^3 x 32 field with the workload's couplings for
    a fixed time budget; each process's time per iteration is scaled by the volume ratio to the
    workload's lattice (every oracle step is a site loop) and by the iteration count the oracle
    needs for true residual 1e-10 at these couplings (measured once by oracle/cgnr_iterations.py on
    the largest lattice listed there), plus the projection on the source timeslice scaled the same
    way.  RHS/s = the sum over processes of 1 / (seconds per RHS)."""
    t0 = time.time()
    pool = _oracle_pool()
    n = os.cpu_count() or 1
    res = pool.map(_oracle_rhs, [(dict(wl), budget_s, j, n) for j in range(n)])
    ratio = float(np.prod(wl["dims"])) / float(16 * 16 * 16 * 32)
    ref = stored_cgnr_iterations(wl)
    n_iter = ref["iters"] if ref else None
    value = sum(1.0 / ((ti * n_iter + tp) * ratio) for ti, tp, _ in res) if n_iter else None
    t_iter = float(np.median([r[0] for r in res]))
    k = min(r[2] for r in res)
    return {"value": value, "unit": "RHS/s", "cores": n, "kind": "oracle", "nproc": os.cpu_count(),
            "sample": ("oracle CGNR, one RHS per host core (%d processes, numpy single-threaded in each), on a "
                       "16^3x32 field with the workload's couplings for >= %d iterations (median %.3f s/iter), "
                       "scaled by the volume ratio %.0f to %s and by the %s CGNR iterations the oracle needs for "
                       "1e-10 at these couplings (measured by oracle/cgnr_iterations.py on the %s field)"
                       % (n, k, t_iter, ratio, "x".join(map(str, wl["dims"])), n_iter,
                          "x".join(map(str, ref["dims"])) if ref else "?")),
            "seconds": time.time() - t0}, setup


# ----------------------------------------------------------------------------- workload set-up
class Workload:
    """Inputs, context, buffers and the step of one workload on this rank's GPU."""

    def __init__(self, name, rhs_block=0, rank=0, world=1, pipeline=0, projection=0):
        import torch
        from lqcd_inputs import colour_vectors, gauge_field
        from paper_2609_37049_b300 import Context, lqcd
        from paper_2609_37049_b300.shard import domain_groups

        self.name, self.wl = name, WORKLOADS[name]
        wl = self.wl
        self.rank, self.world = rank, world
        self.dims, self.T = wl["dims"], wl["dims"][3]
        self.L3 = self.dims[0] * self.dims[1] * self.dims[2]
        self.n_ev = wl["n_ev"]
        self.rhs_block = rhs_block or wl["rhs_block"]
        self.pipeline = pipeline or wl["pipeline"]
        self.projection = projection
        self.nj = self.rhs_block // 4
        assert self.rhs_block % 4 == 0 and self.n_ev % self.nj == 0
        self.n_blocks = self.n_ev // self.nj
        self.t_src = list(wl["t_src"])
        self.slot = {t: k for k, t in enumerate(self.t_src)}
        t0 = time.time()
        self.U = gauge_field(self.dims, wl["eps"], wl["gauge_seed"])
        self.ctx = Context(self.dims)
        self.ctx.gauge_upload(self.U, wl["kappa"], wl["csw"])
        self.ctx.set_domains(wl["extents"])
        self.t_gauge = time.time() - t0
        t0 = time.time()
        if wl["sources"].startswith("lowest Laplacian"):
            Vall = torch.zeros((self.T, self.n_ev, self.L3, 3), dtype=torch.complex128, device="cuda")
            lam = torch.zeros((self.T, self.n_ev), dtype=torch.float64, device="cuda")
            self.ctx.laplace_eigs(self.n_ev, Vall, lam)
            self.V = Vall[self.t_src].contiguous()
            del Vall
        else:
            Vh = colour_vectors(self.dims, self.n_ev, wl["cv_seed"], timeslices=self.t_src)
            self.V = torch.from_numpy(Vh.reshape(len(self.t_src), self.n_ev, self.L3, 3)).cuda()
            del Vh
        torch.cuda.synchronize()
        self.t_vectors = time.time() - t0
        # source groups for the multi-site domain solves: at most one source timeslice per domain
        self.groups = domain_groups(self.t_src, self.T, wl["extents"])
        n_t = len(self.t_src)
        c128 = dict(dtype=torch.complex128, device="cuda")
        self.tau_f = torch.zeros((n_t, self.n_ev, 4, self.n_ev, 4), **c128)
        # per source group: its colour vectors (a view where the slots are consecutive) and tau
        self.Vg, self.tau_g = [], []
        for grp in self.groups:
            ks = [self.slot[t] for t in grp]
            contiguous = ks == list(range(ks[0], ks[0] + len(ks)))
            self.Vg.append(self.V[ks[0]:ks[0] + len(ks)] if contiguous else self.V[ks].contiguous())
            self.tau_g.append(torch.zeros((len(grp), self.n_ev, 4, self.n_ev, 4), **c128))
        self.Lb = {k: torch.zeros((len(GAMMAS), max(len(g) for g in self.groups)), **c128) for k in ("a", "b")}
        self.loops = {k: torch.zeros((1, len(GAMMAS), self.T), **c128) for k in ("f", "ft", "d", "dt")}
        self.corr = dict(C=torch.zeros((len(GAMMAS), self.T, self.T), **c128))
        self.corr["Cdd"], self.corr["dC"] = torch.zeros_like(self.corr["C"]), torch.zeros_like(self.corr["C"])
        self.corr["C_avg"] = torch.zeros((len(GAMMAS), self.T), **c128)
        self.corr["dC_avg"] = torch.zeros_like(self.corr["C_avg"])
        self.corr["valid"] = torch.zeros((self.T, self.T), dtype=torch.int32, device="cuda")
        self.corr["n_valid"] = torch.zeros(self.T, dtype=torch.int32, device="cuda")
        self.params = None
        self.lqcd = lqcd
        self.stats = []

    def tune(self):
        import tempfile
        from paper_2609_37049_b300 import autotune, default_params
        lq = self.lqcd
        self.tuning = autotune.tune(self.ctx, cache=os.path.join(tempfile.gettempdir(), "lqcd_tuning.json"),
                                    precisions=(lq.LQCD_PREC_F32, lq.LQCD_PREC_F64, lq.LQCD_PREC_DF),
                                    blocks=(self.rhs_block // self.pipeline,))
        self.params = default_params(solver=lq.LQCD_SOLVER_MIXED, inner_prec=lq.LQCD_PREC_F32,
                                     rhs_block=self.rhs_block // self.pipeline, pipeline=self.pipeline,
                                     projection=self.projection)
        self.training = None
        if self.wl.get("learned"):  # train the network on solver-generated pairs, then solve with it
            import torch
            L = self.wl["learned"]
            self.ctx.nn_set_weights(lq.nn_initial_weights(5, 0.05))
            torch.cuda.synchronize()
            t0 = time.time()
            hist = self.ctx.nn_train(n_pairs=L["pairs"], epochs=L["epochs"], batch=L["batch"], lr=L["lr"],
                                     seed=L["seed"])
            torch.cuda.synchronize()
            self.training = {"pairs": L["pairs"], "batch": L["batch"], "epochs": L["epochs"], "lr": L["lr"],
                             "seconds": time.time() - t0, "loss_per_epoch": [float(h) for h in hist],
                             "pairs_from": "the solver without the network (FP64 defect correction around FP32 "
                                           "BiCGStab, true residual 1e-8), random even-site r"}
            self.params = default_params(solver=lq.LQCD_SOLVER_FGCR_NN, rhs_block=self.rhs_block,
                                         projection=self.projection)

    def unit(self, step):
        from paper_2609_37049_b300.shard import plan_unit
        return plan_unit(step * self.world + self.rank, len(self.t_src), len(self.groups), self.n_blocks)

    def rhs_of_unit(self, u):
        k, bf, g, bd = u
        return self.rhs_block + self.rhs_block * len(self.groups[g])

    def step(self, s, host=None):
        """One step on device buffers, or (host = dict of pinned numpy arrays) through host buffers.
        Returns the right-hand sides solved."""
        from paper_2609_37049_b300 import Stats
        lq = self.lqcd
        k, bf, g, bd = u = self.unit(s)
        grp = self.groups[g]
        B = self if host is None else None
        V = self.V if B else host["V"]
        Vg = self.Vg[g] if B else host["Vg"][g]
        tau_f = self.tau_f if B else host["tau_f"]
        tau_g = self.tau_g[g] if B else host["tau_g"][g]
        Lb, loops, corr = (self.Lb, self.loops, self.corr) if B else (host["Lb"], host["loops"], host["corr"])
        if host is not None:
            self.ctx.gauge_upload(host["U"], self.wl["kappa"], self.wl["csw"])
        st = Stats(1, 1)
        self.ctx.perambulator_cols(V[k:k + 1], self.n_ev, [self.t_src[k]], tau_f[k:k + 1], bf * self.nj, self.nj,
                                   mode=lq.LQCD_MODE_FULL, sinks=lq.LQCD_SINKS_DIAG_SRCV, params=self.params,
                                   stats=st)
        self.stats.append(("full", st.total_iters, st.max_true_resid, st.outer_cycles))
        st = Stats(1, 1)
        self.ctx.perambulator_cols(Vg, self.n_ev, grp, tau_g, bd * self.nj, self.nj, mode=lq.LQCD_MODE_DOMAIN,
                                   sinks=lq.LQCD_SINKS_DIAG_SRCV, params=self.params, stats=st)
        self.stats.append(("dom", st.total_iters, st.max_true_resid, st.outer_cycles))
        # loops of the timeslices this step touched, then the correlators of the configuration
        La, Lta = Lb["a"][:, :1], Lb["b"][:, :1]
        if B:
            La, Lta = La.contiguous(), Lta.contiguous()
        else:
            La, Lta = np.ascontiguousarray(La), np.ascontiguousarray(Lta)
        self.ctx.loops(tau_f[k:k + 1], self.n_ev, 1, GAMMAS, La, Lta)
        loops["f"][0][:, self.t_src[k]] = La[:, 0]
        loops["ft"][0][:, self.t_src[k]] = Lta[:, 0]
        n = len(grp)
        Ld, Ltd = Lb["a"][:, :n], Lb["b"][:, :n]
        if B:
            Ld, Ltd = Ld.contiguous(), Ltd.contiguous()
        else:
            Ld, Ltd = np.ascontiguousarray(Ld), np.ascontiguousarray(Ltd)
        self.ctx.loops(tau_g, self.n_ev, n, GAMMAS, Ld, Ltd)
        loops["d"][0][:, grp] = Ld
        loops["dt"][0][:, grp] = Ltd
        self.ctx.disc_correlator(loops["f"], loops["ft"], loops["d"], loops["dt"], 0, corr)
        return self.rhs_of_unit(u)

    def host_buffers(self):
        """Pinned host copies of the step's inputs and outputs for the end-to-end measurement."""
        import torch
        pin = lambda t: torch.zeros(t.shape, dtype=t.dtype).pin_memory().numpy()
        V = self.V.cpu().pin_memory().numpy()
        Vg = []
        for grp in self.groups:
            ks = [self.slot[t] for t in grp]
            contiguous = ks == list(range(ks[0], ks[0] + len(ks)))
            Vg.append(V[ks[0]:ks[0] + len(ks)] if contiguous else
                      torch.from_numpy(V[ks]).pin_memory().numpy())
        h = {"U": torch.from_numpy(self.U).pin_memory().numpy(), "V": V, "Vg": Vg, "tau_f": pin(self.tau_f),
             "tau_g": [pin(t) for t in self.tau_g], "Lb": {k: pin(v) for k, v in self.Lb.items()},
             "loops": {k: pin(v) for k, v in self.loops.items()}, "corr": {k: pin(v) for k, v in self.corr.items()}}
        return h

    def e2e_bytes(self, s):
        """Host<->device bytes of one end-to-end step (counted from the arrays the calls copy)."""
        k, bf, g, bd = self.unit(s)
        vslice = self.n_ev * self.L3 * 3 * 16
        tau1 = self.n_ev * 4 * self.n_ev * 4 * 16
        grp = len(self.groups[g])
        ng = len(GAMMAS)
        # gauge field; colour vectors; tau read back first (untouched columns) and written out;
        # loops (tau in, loops out); correlator inputs (four loop arrays) and outputs
        h2d = self.U.nbytes + vslice * (1 + grp) + tau1 * (1 + grp) + tau1 * (1 + grp) + 4 * ng * self.T * 16
        d2h = tau1 * (1 + grp) + 2 * ng * (1 + grp) * 16
        d2h += sum(v.numel() * v.element_size() for v in self.corr.values())
        return int(h2d), int(d2h)


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch
    from paper_2609_37049_b300 import Stats, default_params, lqcd

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    peak, peak_kind = peaks()
    W = Workload(args.workload, args.rhs_block, rank, world, args.pipeline, args.projection)
    W.tune()
    if args.no_graph:
        W.params.use_graph = 0
    if args.profile_step:  # one warm step, then one step inside an NVTX range for an ncu launch list
        W.step(0)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_step")
        W.step(1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_step": "done", "rhs": W.rhs_of_unit(W.unit(1))}), flush=True)
        return None
    for s in range(args.warmup):
        W.step(s)
    torch.cuda.synchronize()
    dist_barrier(world)
    W.stats.clear()
    l0 = lqcd.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rhs = 0
    with ClockSampler(dev) as clk:
        torch.cuda.synchronize()
        e0.record()
        for s in range(args.steps):
            rhs += W.step(args.warmup + s)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = lqcd.kernel_launches() - l0
    ms_max = dist_max(ms, world)
    rhs_all = dist_sum(rhs, world)
    dist_barrier(world)
    value = rhs_all / (ms_max / 1e3)
    full_rhs = args.steps * W.rhs_block * world
    step_stats = list(W.stats)

    res = {"metric": "distillation RHS/s at FP64 resid 1e-10 (mixed FP64/FP32 solver)", "value": value,
           "unit": "RHS/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
           "config": {"workload": W.wl["title"], "lattice": "x".join(map(str, W.dims)), "eps": W.wl["eps"],
                      "kappa": W.wl["kappa"], "c_sw": W.wl["csw"], "n_ev": W.n_ev, "t_src": W.t_src,
                      "domains": "%d x %s" % (len(W.wl["extents"]), sorted(set(W.wl["extents"]))),
                      "rhs_block": W.rhs_block, "batches_in_flight": W.pipeline,
                      "projection": "FP64" if W.projection else "double-float (FP32 pipe)", "sources": W.wl["sources"],
                      "step": "one RHS block: full-operator columns at one source timeslice + domain-operator "
                              "columns of one source group (multi-site solve)",
                      "l2": "inputs larger than L2 (126 MB): each FP64 full-lattice batch vector is %.1f GB"
                            % (W.rhs_block * np.prod(W.dims) * 192 / 1e9),
                      "parallelism": "rhs-sharded x%d" % world},
           "gpu_launches": launches, "clocks": clk.summary(),
           "rates": {"full_rhs_per_s": full_rhs / (ms_max / 1e3),
                     "domain_rhs_per_s": (rhs_all - full_rhs) / (ms_max / 1e3)},
           "solver_stats": {"full_iters_per_rhs": statistics.mean(x[1] for x in step_stats if x[0] == "full") / W.rhs_block,
                            "dom_iters_per_rhs": statistics.mean(x[1] for x in step_stats if x[0] == "dom") / W.rhs_block,
                            "max_true_resid": max(x[2] for x in step_stats),
                            "outer_cycles": max(x[3] for x in step_stats)},
           "setup_s": {"gauge": W.t_gauge, "vectors": W.t_vectors}, "tuning": W.tuning}
    if W.training:
        res["training"] = W.training
        res["metric"] = "distillation RHS/s at FP64 resid 1e-10 (learned-preconditioned FGCR)"
    if not args.no_extras:  # before the end-to-end run, whose host staging buffers stay allocated
        res.update(extras(W, peak, peak_kind, dev))
    if os.environ.get("LQCD_PHASE_TIMING") == "1":  # diagnostic runs: GPU ms per solver phase
        res["phase_ms"] = W.ctx.phase_times()
    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    if args.no_e2e:
        return res
    H = W.host_buffers()
    W.step(args.warmup, host=H)
    torch.cuda.synchronize()
    dist_barrier(world)
    t0 = time.time()
    rhs_e, h2d, d2h = 0, 0, 0
    for s in range(args.steps):
        rhs_e += W.step(args.warmup + s, host=H)
        bi, bo = W.e2e_bytes(args.warmup + s)
        h2d, d2h = h2d + bi, d2h + bo
    torch.cuda.synchronize()
    e2e_s = dist_max(time.time() - t0, world)
    e2e = {"value": dist_sum(rhs_e, world) / e2e_s, "unit": "RHS/s", "h2d_bytes_per_step": h2d // args.steps,
           "d2h_bytes_per_step": d2h // args.steps, "steps": args.steps}
    del H

    res["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"], _ = cpu_baseline(W.wl)
    return res


def captured_traffic(variant, site_rhs):
    """DRAM bytes of one FP32 dslash launch of the captured variant, scaled from the committed ncu
    capture (profiles/dslash_f32_24x24x24x48_nrhs16.md: bytes per (site, RHS)) to site_rhs pairs;
    None when another variant runs or the kernel's sources changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "dslash_f32_24x24x24x48_nrhs16.md")) as f:
            rec = dict(line.split(":", 1) for line in f.read().splitlines()
                       if line.startswith(("source_sha256_16:", "traffic_bytes_per_site_rhs:", "traffic_variant:")))
    except OSError:
        return None
    if rec.get("traffic_variant", "").strip() != str(variant):
        return None
    h = hashlib.sha256()
    for name in ("dslash_staged.cu", "dslash_ops.cuh", "lqcd_common.cuh"):
        with open(os.path.join(ROOT, "paper_2609_37049_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    if rec.get("source_sha256_16", "").split()[0:1] != [h.hexdigest()[:16]]:
        return None
    return float(rec["traffic_bytes_per_site_rhs"]) * float(site_rhs)


def extras(W, peak, peak_kind, dev):
    """Solvers on one sample, domain extents 8 and 12, and the dslash rooflines (outside the timed
    region)."""
    import torch
    from paper_2609_37049_b300 import Stats, default_params, lqcd
    out = {}
    ctx = W.ctx
    n = W.wl["solver_sample_rhs"]
    nj = max(1, n // 4)
    tau1 = torch.zeros((1, W.n_ev, 4, W.n_ev, 4), dtype=torch.complex128, device="cuda")

    def sample(p):
        ctx.perambulator_cols(W.V[0:1], W.n_ev, [W.t_src[0]], tau1, 0, nj, mode=lqcd.LQCD_MODE_FULL,
                              sinks=lqcd.LQCD_SINKS_DIAG_SRCV, params=p)  # graphs, buffers
        torch.cuda.synchronize()
        t0 = time.time()
        st = Stats(1, 1)
        ctx.perambulator_cols(W.V[0:1], W.n_ev, [W.t_src[0]], tau1, 0, nj, mode=lqcd.LQCD_MODE_FULL,
                              sinks=lqcd.LQCD_SINKS_DIAG_SRCV, params=p, stats=st)
        torch.cuda.synchronize()
        return {"rhs_per_s": 4 * nj / (time.time() - t0), "iters_per_rhs": st.total_iters / (4 * nj),
                "max_true_resid": st.max_true_resid, "fallback": st.fallback, "outer_cycles": st.outer_cycles}

    solvers = {}
    blk = 4 * nj
    solvers["plain_fp64_bicgstab"] = sample(default_params(solver=lqcd.LQCD_SOLVER_BICGSTAB64, rhs_block=blk))
    solvers["mixed_fp32_bicgstab"] = sample(default_params(solver=lqcd.LQCD_SOLVER_MIXED,
                                                           inner_prec=lqcd.LQCD_PREC_F32, rhs_block=blk))
    if np.prod(W.dims) <= 24 ** 3 * 48:  # its 16 extra Krylov vectors do not fit beside the 48^3x96 batch
        solvers["mixed_fgcr_fp16_mr4"] = sample(default_params(solver=lqcd.LQCD_SOLVER_MIXED,
                                                               inner_prec=lqcd.LQCD_PREC_F16, precond_iters=4,
                                                               rhs_block=blk))
    if W.training:
        solvers["mixed_fgcr_learned"] = sample(default_params(solver=lqcd.LQCD_SOLVER_FGCR_NN, rhs_block=blk))
        solvers["mixed_fgcr_none"] = sample(default_params(solver=lqcd.LQCD_SOLVER_FGCR_NN, precond_iters=-1,
                                                           rhs_block=blk))
    plain = solvers["plain_fp64_bicgstab"]["rhs_per_s"]
    out["solvers"] = solvers
    out["solver_sample"] = "full-operator perambulator columns of %d RHS (t=%d, colour vectors 0..%d, 4 spins)" % (
        4 * nj, W.t_src[0], nj - 1)
    out["speedup_vs_plain"] = {k: v["rhs_per_s"] / plain for k, v in solvers.items()}
    # domain extents swept beside the timed tiling: one source group, the first block (the solver
    # samples' work buffers released first: the sweep's inputs are torch allocations)
    ctx.release_workspace()
    torch.cuda.empty_cache()
    sweep = {}
    for ext, tiling in W.wl["sweep"].items():
        ctx.set_domains(tiling)
        from paper_2609_37049_b300.shard import domain_groups
        grp = domain_groups(W.t_src, W.T, tiling)[0]
        ks = [W.slot[t] for t in grp]
        Vg = W.V[ks].contiguous()
        tg = torch.zeros((len(grp), W.n_ev, 4, W.n_ev, 4), dtype=torch.complex128, device="cuda")
        ctx.perambulator_cols(Vg, W.n_ev, grp, tg, 0, W.nj, mode=lqcd.LQCD_MODE_DOMAIN,
                              sinks=lqcd.LQCD_SINKS_DIAG_SRCV, params=W.params)
        torch.cuda.synchronize()
        st = Stats(1, 1)
        t0 = time.time()
        ctx.perambulator_cols(Vg, W.n_ev, grp, tg, 0, W.nj, mode=lqcd.LQCD_MODE_DOMAIN,
                              sinks=lqcd.LQCD_SINKS_DIAG_SRCV, params=W.params, stats=st)
        torch.cuda.synchronize()
        dt = time.time() - t0
        sweep[str(ext)] = {"domains": len(tiling), "sources_in_group": len(grp),
                           "domain_rhs_per_s": W.rhs_block * len(grp) / dt, "iters_per_rhs": st.total_iters / W.rhs_block,
                           "max_true_resid": st.max_true_resid}
        del Vg, tg
    ctx.set_domains(W.wl["extents"])
    if sweep:
        out["domain_sweep"] = sweep
    # dslash rooflines of the dominant kernel (FP32 hopping + inverse clover at the RHS block)
    ctx.release_workspace()
    torch.cuda.empty_cache()
    dsl = {}
    nbat = W.rhs_block // W.pipeline  # right-hand sides of one launch
    n64 = min(nbat, 4 if np.prod(W.dims) > 24 ** 3 * 48 else nbat)
    for name, prec, nr in (("f32", lqcd.LQCD_PREC_F32, nbat), ("f64", lqcd.LQCD_PREC_F64, n64)):
        ms_l, by = ctx.dslash_bench(prec, nr, 10, True)
        dsl[name] = {"ms": ms_l, "GBs": by / ms_l / 1e6, "bytes": by, "nrhs": nr}
    achieved = dsl["f32"]["GBs"]
    v32 = int(W.tuning["variant"].get(str(lqcd.LQCD_PREC_F32), {}).get(str(nbat), 0))
    kname = {3: "dslash_sl_kernel", 4: "dslash_pipe_kernel", 5: "dslash_sl2_kernel", 6: "dslash_sl3_kernel",
             7: "dslash_rb2_kernel"}.get(v32, "dslash_kernel")
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "traffic": captured_traffic(v32, np.prod(W.dims) // 2 * nbat), "peak_kind": peak_kind,
                       "kernel": "%s<P32,EPI_CH> (launch variant %d: eo hopping + A^-1, %d RHS)" % (kname, v32,
                                                                                                  nbat),
                       "algo_bytes_per_launch": dsl["f32"]["bytes"]}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    f64_flops = 1824.0 * (np.prod(W.dims) // 2) * n64
    f64_peak = n_sm * 2 * 2 * 2.032e9 / 1e12
    out["roofline_fp64"] = {"bound": "alu", "kernel": "dslash_kernel<P64,EPI_CH> (%d RHS)" % n64,
                            "unit": "TFLOP/s", "achieved": f64_flops / (dsl["f64"]["ms"] * 1e-3) / 1e12,
                            "peak": f64_peak, "peak_kind": "derived: SMs x 2 FP64 FMA/clk x 2 flops x 2.032 GHz",
                            "algo_flops_per_launch": f64_flops}
    out["roofline_fp64"]["frac"] = out["roofline_fp64"]["achieved"] / f64_peak
    out["dslash"] = dsl
    return out


def profile_dslash(args):
    """The FP32 / FP16 / FP64 even-odd hopping + inverse-clover kernels of the workload's lattice,
    a few launches each per launch variant, L2 flushed between launches (small command for ncu)."""
    import torch
    from lqcd_inputs import gauge_field
    from paper_2609_37049_b300 import Context, lqcd
    wl = WORKLOADS[args.workload]
    torch.cuda.set_device(0)
    ctx = Context(wl["dims"])
    ctx.gauge_upload(gauge_field(wl["dims"], wl["eps"], wl["gauge_seed"]), wl["kappa"], wl["csw"])
    nr = args.dslash_nrhs or (args.rhs_block or wl["rhs_block"])
    out = {}
    for name, prec in (("f32", lqcd.LQCD_PREC_F32), ("f16", lqcd.LQCD_PREC_F16), ("f64", lqcd.LQCD_PREC_F64),
                       ("df_res", lqcd.LQCD_PREC_DF)):
        for v in (range(3) if prec in (lqcd.LQCD_PREC_F64, lqcd.LQCD_PREC_DF) else range(8)):
            if args.dslash_variant >= 0 and v != args.dslash_variant:
                continue
            ctx.set_dslash_variant(prec, nr, v)
            ms, by = ctx.dslash_bench(prec, nr, 3, True)
            out["%s_v%d" % (name, v)] = {"nrhs": nr, "ms": ms, "GBs": by / ms / 1e6, "algo_bytes": by}
    print(json.dumps(out), flush=True)


def profile_nn(args):
    """The gauge-covariant network on the workload's lattice: FP32 CUDA-core layers and the
    tensor-core layers, 2 + 3 applications each on N random samples (device buffers)."""
    import torch
    from lqcd_inputs import gauge_field
    from paper_2609_37049_b300 import Context, lqcd
    wl = WORKLOADS[args.workload]
    torch.cuda.set_device(0)
    ctx = Context(wl["dims"])
    ctx.gauge_upload(gauge_field(wl["dims"], wl["eps"], wl["gauge_seed"]), wl["kappa"], wl["csw"])
    ctx.nn_set_weights(lqcd.nn_initial_weights(3))
    n = args.dslash_nrhs or 16
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.randn((n, int(np.prod(wl["dims"])), 4, 3), dtype=torch.complex64, device="cuda", generator=g)
    out = {}
    for name, f in (("fp32", ctx.nn_apply), ("tensor_core", ctx.nn_apply_tc)):
        o = torch.zeros_like(x)
        for _ in range(2):
            f(x, o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            f(x, o)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"samples": n, "ms_per_application": e0.elapsed_time(e1) / 3}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle as it stands, timed per step on a bounded sample (see cpu_baseline)."""
    wl = WORKLOADS[args.workload]
    vals, setup = [], None
    for _ in range(args.warmup):
        _, setup = cpu_baseline(wl, budget_s=2.0, setup=setup)
    t0 = time.time()
    for _ in range(args.steps):
        r, setup = cpu_baseline(wl, budget_s=4.0, setup=setup)
        vals.append(r)
    total = time.time() - t0
    v = statistics.median(x["value"] for x in vals) if vals[0]["value"] else None
    return {"impl": "reference", "metric": "distillation RHS/s at FP64 resid 1e-10 (mixed FP64/FP32 solver)",
            "value": v, "unit": "RHS/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["title"], "lattice": "x".join(map(str, wl["dims"])), "eps": wl["eps"],
                       "kappa": wl["kappa"], "c_sw": wl["csw"], "n_ev": wl["n_ev"], "t_src": wl["t_src"],
                       "domains": "%d x %s" % (len(wl["extents"]), sorted(set(wl["extents"]))),
                       "sources": wl["sources"], "parallelism": "oracle on the host cores"},
            "cpu_baseline": {"value": v, "unit": "RHS/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- distributed glue
_PG = None


def dist_init():
    global _PG
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
        _PG = dist
    return rank, world


def dist_barrier(world):
    if world > 1 and _PG is not None:
        _PG.barrier()


def _reduce(x, world, op):
    if world > 1 and _PG is not None:
        import torch
        t = torch.tensor([float(x)], device="cuda" if torch.cuda.is_available() else "cpu")
        _PG.all_reduce(t, op=op)
        return float(t.item())
    return x


def dist_max(x, world):
    return _reduce(x, world, _PG.ReduceOp.MAX if _PG is not None else None)


def dist_sum(x, world):
    return _reduce(x, world, _PG.ReduceOp.SUM if _PG is not None else None)


def main():
    args = parse()
    if args.profile_dslash:
        profile_dslash(args)
        return
    if args.profile_nn:
        profile_nn(args)
        return
    rank, world = dist_init()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    res = run_ours(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
