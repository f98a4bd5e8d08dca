#!/usr/bin/env python3
"""Benchmark of the nested shift-invert MINRES eigensolver (Kutsuzawa & Todo,
arXiv:2203.09732) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the L = 28 random-field Heisenberg chain (dimension 40,116,600),
h = 3.7, seeds 0, 1, 2, the 10 eigenpairs nearest sigma = (E_min + E_max)/2,
FP32 MINRES with FP64 iterative refinement inside an FP64 shift-invert
Lanczos with full reorthogonalisation (Sec. IV A; Algorithms 1 and 2).

A full solve at this size needs about 5e7 MINRES iterations per Lanczos step
(the iteration count grows as n, Sec. IV A), hours per step, so a timed step
runs every part of the pipeline at full size with each MINRES solve capped:
one call of hs_lanczos_eigs with K Lanczos steps whose solves stop after
--minres-cap iterations, the Ritz pairs certified by FP64 residuals, and the
twist overlaps. The realisations rotate over the steps. The reported value is
eigenpairs per second PROJECTED from what the timed steps measure at L = 28
(seconds per MINRES iteration, per Lanczos step outside MINRES, per Ritz
certification) and an iteration model measured on the GPU in the same run:
full MINRES solves at L = 16, 18, 20 (iterations per solve ~ n^b, fitted) and
full eigensolves at L = 12 (Lanczos steps for K pairs):

    T_pair_set = m * (N(L=28) * t_iter + t_lanczos_step) + t_ritz,
    value = K / T_pair_set.

The plain FP64 method is measured the same way (fewer steps) and projected
with its own iteration model; `fp32_refine_over_fp64` is the ratio. The H x
kernel at L = 28 is timed alone for the roofline. A batch of 24 L = 16
realisations solved to convergence gives a measured (not projected)
eigenpairs/s beside it.

Several GPUs (torchrun): each rank runs its own realisations (replicas, weak
scaling, no collective on the data path); value = sum over ranks.
"""
import os

# Concurrent realisations (the L = 16 batch) run on separate streams; with
# more than 8 busy streams, CUDA's default of 8 hardware queues makes a short
# kernel wait behind another stream's persistent solve. This must be set
# before the CUDA context exists (a process setting, not a GPU setting).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse
import hashlib
import json
import math
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigenpairs/s near sigma at L=28 (FP32+refine vs FP64); H*v GB/s vs HBM peak"
UNIT = "eigenpairs/s"
L28_H = 3.7
L28_SEEDS = (0, 1, 2)
BATCH = 24
SHARE_CAP = 38   # SMs per L = 16 solve when few realisations are left
FALLBACK_HBM_GBS = 6800.0
CAL_L = (16, 18, 20)      # full MINRES solves for the iteration model
CAL_M_L = 12              # full eigensolves for the Lanczos step count


class Shares:
    """SM shares of the realisations running in one L = 16 batch. Every
    realisation starts on `base` SMs; when one finishes, the others get
    nsm // (number still running) SMs each (at most `cap`, never less than
    `base`) from their next Lanczos step on: the library reads a handle's share
    at every MINRES solve. The shares of running solves never sum to more than
    nsm. `static` keeps every share at `base`."""

    def __init__(self, n, base, nsm, cap=SHARE_CAP, static=False):
        self.lock = threading.Lock()
        self.live = {}
        self.active = n
        self.base, self.nsm, self.cap, self.static = base, nsm, cap, static
        self.current = None

    def share(self):
        if self.static:
            return self.base
        return max(self.base, min(self.cap, self.nsm // max(1, self.active)))

    def start(self, key, chain):
        with self.lock:
            self.live[key] = chain
            self.current = self.share()
            chain.set_sm_budget(self.current)

    def done(self, key):
        with self.lock:
            self.live.pop(key, None)
            self.active -= 1
            b = self.share()
            if b != self.current:
                self.current = b
                for other in self.live.values():
                    other.set_sm_budget(b)


def realisation(idx, L):
    """Realisation idx of the batched sweep: h ~ U[0.5, 6], h_j ~ U[-h, h]."""
    from paper_2203_09732_gb300 import inputs
    h, hv = inputs.disorder_mixed(L, 1000 * L + idx)
    return h, 1000 * L + idx, hv


def rank_realisations(rank, world, step, batch):
    """Realisation indices of one step on one rank: disjoint across ranks and
    steps (replicas, weak scaling)."""
    base = (rank + world * step) * batch
    return [base + i for i in range(batch)]


def rank_seeds(rank, world):
    """Disorder seeds of the L = 28 realisations on one rank: 0, 1, 2 on rank 0,
    then the next three on each further rank (replicas)."""
    return [len(L28_SEEDS) * rank + s for s in L28_SEEDS]


def fit_power(ns, its):
    """Least-squares fit of log(iterations) = a + b log(n)."""
    b, a = np.polyfit(np.log(np.asarray(ns, float)), np.log(np.asarray(its, float)), 1)
    return float(a), float(b)


def project(a, b, n):
    return float(math.exp(a + b * math.log(n)))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--L", type=int, default=28)
    ap.add_argument("--K", type=int, default=10)
    ap.add_argument("--minres-cap", type=int, default=192, dest="minres_cap",
                    help="MINRES iterations per solve in a timed step")
    ap.add_argument("--minres-tol", type=float, default=1e-10, dest="minres_tol")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-l16", action="store_true", help="skip the L = 16 batch")
    ap.add_argument("--no-calibration", action="store_true",
                    help="skip the iteration-model solves (value then null)")
    ap.add_argument("--static-budget", action="store_true", dest="static_budget")
    ap.add_argument("--detail", default=None, help="write per-step records to this JSON file")
    ap.add_argument("--sweep", default="24,0",
                    help="--only sweep: realisations at L = 16 and L = 18 (C3 recipe)")
    ap.add_argument("--only", choices=["hv", "minres", "forms", "smem", "sweep"], default=None,
                    help="profiling cases: only the H x timing at --L; one capped MINRES "
                         "solve (FP32 + refinement) of --minres-iters iterations at --L; the "
                         "products and MINRES iterations of every row form at L = 24, 26, 28; "
                         "--minres-iters FP64 and FP32 iterations of the one- and "
                         "two-reduction shared-memory forms at --L (L <= 20); or one batched "
                         "sweep (hs_sweep) of the --sweep realisations, K = 8, beside the "
                         "24-stream batch of the same L = 16 realisations")
    ap.add_argument("--minres-iters", type=int, default=200, dest="minres_iters")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------------------
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback (profiling recipe 6.8 TB/s)"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("common.cuh", "sb.cuh", "sb_kern.cuh", "sb4.cuh", "sb4_kern.cuh", "hv_sb.cu"):
        h.update(open(os.path.join(ROOT, "paper_2203_09732_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(name):
    """dram bytes per launch recorded in profiles/<name>.md, if the kernel
    sources still match the hash stored there."""
    p = os.path.join(ROOT, "profiles", name + ".md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def hv_kernel_name(L):
    e = os.environ.get("HS_HV_SB")
    on = (e == "1" and L >= 22) if e is not None else L >= 24
    if not on:
        return "k_matvec<float> (block form)"
    if os.environ.get("HS_SB4") == "1":
        return "k_sb4<float, MODE_HV> (four-low-bit superblock form, one lane per sub-block)"
    return "k_sbhv<float, MODE_HV> (ten-low-bit superblock form, one warp per sub-block)"


def hv_roofline(torch, hs, L, stream):
    """H x at L (FP32 and FP64), timed with CUDA events on the launching
    stream over 20 (FP32) / 5 (FP64) launches; inputs (2 x 160 MB in FP32 at
    L = 28) exceed L2."""
    from paper_2203_09732_gb300 import inputs
    out = {}
    with hs.Chain(L, inputs.disorder(L, L28_H, 0), sigma=0.0, stream=stream) as c:
        n = c.n
        for name, dt, w in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
            x = torch.randn(n, dtype=dt, device="cuda")
            y = torch.empty_like(x)
            for _ in range(3):
                c.matvec(x, y, shifted=True)
            torch.cuda.synchronize()
            reps = 20 if name == "f32" else 5
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                c.matvec(x, y, shifted=True)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3 / reps
            out[name] = {"n": n, "seconds": sec, "bytes": 2 * n * w}
            del x, y
    return out


# ---------------------------------------------------------------------------
# the oracle (CPU): per-iteration cost of Algorithm 2 and its own iteration
# model; used by the cpu_baseline object and by --impl reference
ORACLE_SAMPLE_L = 22


class OracleModel:
    """The oracle as it stands (scipy CSR FP64 Algorithm 2 inside Algorithm 1),
    projected to L = 28 like the GPU arm: iterations per solve from full
    oracle solves at L = 12, 14, 16 (fitted ~ n^b), Lanczos steps for K pairs
    from the oracle's eigensolves at L = 12 (as the GPU arm), and seconds per iteration from a
    bounded run at L = 22, scaled to L = 28 by the nonzeros (n L)."""

    def __init__(self, K, tol):
        self.K, self.tol = K, tol
        self.model = None
        self.sample = None

    def calibrate(self):
        import scipy.sparse as sp

        from oracle import hamiltonian, lanczos, minres, rng
        from paper_2203_09732_gb300 import inputs
        ns, its = [], []
        for L in (12, 14, 16):
            h = inputs.disorder(L, L28_H, 0)
            H, diag, st = hamiltonian.build(L, h)
            sigma = lanczos.sigma_midpoint(H)
            A = (H - sigma * sp.identity(H.shape[0])).tocsr()
            Minv = 1.0 / hamiltonian.precond_diag(H, diag, sigma, "row")
            b = inputs.gaussian(H.shape[0], 7)
            b /= np.linalg.norm(b)
            x, k, phi = minres.pminres(A, b, Minv, tol=self.tol, kmax=60 * H.shape[0])
            ns.append(H.shape[0])
            its.append(k)
        a, b = fit_power(ns, its)
        steps = []
        for s in L28_SEEDS:
            h = inputs.disorder(CAL_M_L, L28_H, s)
            H, diag, st = hamiltonian.build(CAL_M_L, h)
            sigma = lanczos.sigma_midpoint(H)
            v0 = rng.uniform_pm1(1000 + s, H.shape[0])
            steps.append(_oracle_lanczos_steps(H, diag, sigma, self.K, v0, self.tol))
        self.model = {"fit_a": a, "fit_b": b, "ns": ns, "iters": its,
                      "lanczos_steps": steps, "m": float(np.mean(steps))}
        return self.model

    def sample_iteration(self, seconds=8.0):
        """Seconds per Algorithm-2 iteration at L = 28, from a bounded run at
        L = 22 scaled by n L."""
        import scipy.sparse as sp

        from oracle import hamiltonian, minres
        from paper_2203_09732_gb300 import inputs
        L = ORACLE_SAMPLE_L
        if self.sample is None:
            h = inputs.disorder(L, L28_H, 0)
            H, diag, st = hamiltonian.build(L, h)
            A = (H - 0.0 * sp.identity(H.shape[0])).tocsr()
            Minv = 1.0 / hamiltonian.precond_diag(H, diag, 0.0, "row")
            b = inputs.gaussian(H.shape[0], 1)
            self.sample = (A, Minv, b)
        A, Minv, b = self.sample
        it = 4
        minres.pminres(A, b, Minv, kmax=2, tol=0.0)
        while True:
            t0 = time.perf_counter()
            minres.pminres(A, b, Minv, kmax=it, tol=0.0)
            dt = time.perf_counter() - t0
            if dt > seconds / 3 or it >= 4096:
                break
            it *= 3
        n22 = A.shape[0]
        n28 = math.comb(28, 14)
        return dt / it * (n28 * 28) / (n22 * L), it, dt


def _oracle_lanczos_steps(H, diag, sigma, K, v0, tol):
    """Lanczos steps the oracle's Algorithm 1 (Algorithm 2 inside) needs for K
    pairs: it runs its fixed m = max(130, 3K + 30) steps, and the count is the
    first k whose Ritz estimates beta_{k+1} |y_{k,i}| (oracle lanczos.ritz on
    the leading T_k) meet tol |theta_i| for every wanted pair, the library's
    stopping rule."""
    import scipy.sparse as sp

    from oracle import hamiltonian, lanczos, minres
    n = H.shape[0]
    A = (H - sigma * sp.identity(n, format="csr")).tocsr()
    Minv = 1.0 / hamiltonian.precond_diag(H, diag, sigma, "row")
    m = min(max(130, 3 * K + 30), n)
    alpha, beta, V = lanczos.si_lanczos(
        lambda v: minres.pminres(A, v, Minv, tol=tol, kmax=50 * n)[0], v0, m)
    for k in range(K, len(alpha) + 1):
        E, psi, theta, est = lanczos.ritz(alpha[:k], beta[: k + 1], V[:, :k], sigma, K)
        if (est <= tol * np.abs(theta)).all():
            return k
    return len(alpha)


def cpu_projection(om, t_it):
    n28 = math.comb(28, 14)
    N = project(om.model["fit_a"], om.model["fit_b"], n28)
    T = om.model["m"] * N * t_it
    return om.K / T, N, T


def run_reference(args):
    """--impl reference: the CPU oracle, timed on this host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    K = args.K
    om = OracleModel(K, args.minres_tol)
    t0 = time.perf_counter()
    om.calibrate()
    cal_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        om.sample_iteration(1.0)
    t0 = time.perf_counter()
    vals, its = [], []
    for s in range(args.steps):
        t_it, it, dt = om.sample_iteration(3.0)
        vals.append(t_it)
        its.append(it)
    wall = time.perf_counter() - t0
    t_it = float(np.median(vals))
    v, N, T = cpu_projection(om, t_it)
    sample = (f"oracle Algorithm 2 (scipy CSR FP64, one core) at L={ORACLE_SAMPLE_L} for "
              f"{its[-1]} iterations per step, scaled to L=28 by n L: {t_it:.3f} s/iteration; "
              f"x {N:.3g} iterations per solve (fit of oracle solves at L=12,14,16) x "
              f"{om.model['m']:.1f} Lanczos steps (oracle eigensolves at L=12); projection")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded disorder realisations)",
        "config": {"workload": f"L=28 random-field Heisenberg chain, Sz=0 (dim {math.comb(28, 14)}), "
                               f"h={L28_H}, seeds 0-2, {K} eigenpairs nearest sigma=(Emin+Emax)/2",
                   "L": 28, "K": K, "minres_tol": args.minres_tol},
        "value_kind": "projected eigenpairs/s (measured seconds per oracle iteration x oracle iteration model)",
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_model": {k: om.model[k] for k in ("fit_a", "fit_b", "m")},
        "calibration_s": cal_s,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def calibrate_gpu(torch, hs, K, tol):
    """The GPU's iteration model: full MINRES solves at L = 16, 18, 20 (FP64
    and FP32 + refinement) and full FP64 eigensolves at L = 12 for the
    Lanczos step count (roughly independent of L, Sec. IV A); every input as in the L = 28 workload (h = 3.7,
    sigma at the midpoint, a unit random right-hand side)."""
    from paper_2203_09732_gb300 import inputs
    rec = {"L": [], "n": [], "fp64": [], "mixed": []}
    for L in CAL_L:
        with hs.Chain(L, inputs.disorder(L, L28_H, 0)) as c:
            b = inputs.gaussian(c.n, 7)
            b = torch.from_numpy(b / np.linalg.norm(b)).cuda()
            rec["L"].append(L)
            rec["n"].append(c.n)
            for key, mixed in (("fp64", False), ("mixed", True)):
                x, info = c.minres(b, tol=tol, kmax=60 * c.n, mixed=mixed, inner_tol=1e-5,
                                   allow_not_converged=True)
                rec[key].append(info["iters"])
    steps = []
    for s in L28_SEEDS:
        with hs.Chain(CAL_M_L, inputs.disorder(CAL_M_L, L28_H, s)) as c:
            ev, vecs, res, info = c.eigs(K, seed=1000 + s, minres_tol=tol, vectors=False,
                                         allow_not_converged=True)
            steps.append(info["steps"])
    rec["lanczos_steps"] = steps
    rec["m"] = float(np.mean(steps))
    for key in ("fp64", "mixed"):
        a, b = fit_power(rec["n"], rec[key])
        rec[key + "_fit"] = {"a": a, "b": b}
    return rec


def run_ours(args):
    import torch

    from paper_2203_09732_gb300 import hs, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    hs.load()
    L, K, cap = args.L, args.K, args.minres_cap
    n = math.comb(L, L // 2)
    stream = torch.cuda.Stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # the realisations of this rank, sigma set by the extremal Lanczos inside hs_create
    t0 = time.perf_counter()
    chains = []
    with torch.cuda.stream(stream):
        for s in rank_seeds(rank, world):
            chains.append(hs.Chain(L, inputs.disorder(L, L28_H, s), stream=stream))
    torch.cuda.synchronize()
    create_s = (time.perf_counter() - t0) / len(chains)

    def step(i, mixed, out):
        c = chains[i % len(chains)]
        with torch.cuda.stream(stream):
            ev, vecs, res, info = c.eigs(K, m_max=K, mixed=mixed, minres_tol=args.minres_tol,
                                         minres_kmax=cap, seed=1000 + i, allow_not_converged=True)
            z = c.twist(vecs)
        out.append({"seed_idx": i % len(chains), "minres_iters": info["minres_iters"],
                    "lanczos_steps": info["steps"], "sweeps": info["sweeps"],
                    "s_solve": info["seconds_solve"], "s_ritz": info["seconds_ritz"],
                    "s_total": info["seconds_total"], "max_resid": float(res.max()),
                    "zabs2_mean": float(np.mean(np.abs(z) ** 2))})

    for w in range(args.warmup):
        step(10_000 + w, True, [])
    recs = []
    launches0 = hs.kernel_launches()
    barrier()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for s_ in range(args.steps):
            step(s_, True, recs)
        e1.record(stream)
        barrier()
        wall = time.perf_counter() - t0
    dev_sec = e0.elapsed_time(e1) / 1e3
    launches = hs.kernel_launches() - launches0
    tmax = dev_sec
    if dist is not None:
        t = torch.tensor([dev_sec], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax = float(t.item())

    def parts(rs, total):
        """Split the event-timed total of a set of steps into seconds per
        MINRES iteration, per Lanczos step outside MINRES and per certification
        (the shares of the library's own host timers)."""
        its = sum(r["minres_iters"] for r in rs)
        st = sum(r["lanczos_steps"] for r in rs)
        s_tot = sum(r["s_total"] for r in rs)
        f = total / s_tot if s_tot > 0 else 1.0
        t_it = f * sum(r["s_solve"] for r in rs) / its
        t_lz = f * sum(r["s_total"] - r["s_solve"] - r["s_ritz"] for r in rs) / st
        t_rz = f * sum(r["s_ritz"] for r in rs) / len(rs)
        return {"t_iter_s": t_it, "t_lanczos_step_s": t_lz, "t_ritz_s": t_rz,
                "minres_iters": its, "lanczos_steps": st, "seconds": total}

    mix = parts(recs, tmax)

    # the plain FP64 method, same steps (fewer of them)
    rec64 = []
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    n64 = max(1, min(3, args.steps))
    step(20_000, False, [])
    torch.cuda.synchronize()
    e2.record(stream)
    for s_ in range(n64):
        step(s_, False, rec64)
    e3.record(stream)
    torch.cuda.synchronize()
    f64 = parts(rec64, e2.elapsed_time(e3) / 1e3)
    for c in chains:
        c.close()
    chains.clear()

    # iteration model (GPU, same run)
    cal = None if args.no_calibration else calibrate_gpu(torch, hs, K, args.minres_tol)

    def proj(p, key):
        if cal is None:
            return None
        N = project(cal[key + "_fit"]["a"], cal[key + "_fit"]["b"], n)
        T = cal["m"] * (N * p["t_iter_s"] + p["t_lanczos_step_s"]) + p["t_ritz_s"]
        return {"eigenpairs_per_s": K / T, "seconds_per_K_pairs": T, "minres_iters_per_solve": N,
                "lanczos_steps": cal["m"]}

    pj_mix, pj_64 = proj(mix, "mixed"), proj(f64, "fp64")
    value = world * pj_mix["eigenpairs_per_s"] if pj_mix else None

    # end to end through the C ABI with host buffers only (hs_eigs_host): the
    # disorder goes in from host memory, the handle, sigma (extremal Lanczos),
    # the capped Lanczos steps, certification and twist run on the device, and
    # the K eigenvectors (K n doubles), eigenvalues, residuals and overlaps come
    # back into pinned host memory, all inside the timed region
    barrier()
    pinned = torch.empty((K, n), dtype=torch.float64, pin_memory=True)
    hv0 = inputs.disorder(L, L28_H, rank_seeds(rank, world)[0])
    t0 = time.perf_counter()
    ev, vec, res, z, einfo = hs.eigs_host(L, hv0, K, m_max=K, mixed=True, minres_tol=args.minres_tol,
                                          minres_kmax=cap, seed=1000, out=pinned.numpy())
    e2e_wall = time.perf_counter() - t0
    barrier()
    fixed_e2e = e2e_wall - einfo["seconds_total"]      # create + sigma + copies + twist
    e2e_val = None
    if pj_mix:
        e2e_val = world * K / (pj_mix["seconds_per_K_pairs"] + max(0.0, fixed_e2e))
    h2d = 8 * L
    d2h = K * n * 8 + K * 8 + K * 8 + 2 * K * 8
    del pinned

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # H x bandwidth at L = 28 (the product inside MINRES pass A)
    peak, peak_src = peaks()
    rf = hv_roofline(torch, hs, L, torch.cuda.current_stream())
    f32r = rf["f32"]
    achieved = f32r["bytes"] / f32r["seconds"] / 1e9
    traffic = profiled_traffic(f"hv_l{L}_f32")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": f"{hv_kernel_name(L)}: (H - sigma) x at L={L}, n={f32r['n']}; MINRES pass A "
                          f"is the same kernel template with the alpha dot fused",
                "algorithmic_bytes_per_launch": f32r["bytes"], "launch_us": f32r["seconds"] * 1e6,
                "peak_source": peak_src,
                "f64": {"achieved": rf["f64"]["bytes"] / rf["f64"]["seconds"] / 1e9,
                        "launch_us": rf["f64"]["seconds"] * 1e6}}
    iter_bytes32 = 11 * n * 4
    minres_iter = {"fp32_us": mix["t_iter_s"] * 1e6, "fp64_us": f64["t_iter_s"] * 1e6,
                   "algorithmic_bytes_fp32": iter_bytes32,
                   "fp32_GBps": iter_bytes32 / mix["t_iter_s"] / 1e9,
                   "fp32_frac": iter_bytes32 / mix["t_iter_s"] / 1e9 / peak,
                   "fp64_GBps": 2 * iter_bytes32 / f64["t_iter_s"] / 1e9,
                   "per_iteration_speedup_fp32": f64["t_iter_s"] / mix["t_iter_s"]}

    # the L = 16 batch, solved to convergence (measured, not projected)
    l16 = None
    if not args.no_l16:
        l16 = l16_batch(torch, hs, args)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        om = OracleModel(K, args.minres_tol)
        t0 = time.perf_counter()
        om.calibrate()
        t_it, it, dt = om.sample_iteration(8.0)
        v, N, T = cpu_projection(om, t_it)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"oracle Algorithm 2 (scipy CSR FP64, one core) at L={ORACLE_SAMPLE_L}, "
                          f"{it} iterations in {dt:.1f} s, scaled to L=28 by n L; iteration model from "
                          f"oracle solves at L=12,14,16 and eigensolves at L=12; projection like value"),
               "wall_s": time.perf_counter() - t0}
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (MINRES, H*v) + f64 (refinement, Lanczos)",
        "data": "synthetic (seeded disorder, h_j ~ U[-3.7, 3.7])",
        "value_kind": ("projected: K / (m (N t_iter + t_lanczos_step) + t_ritz); t_* measured at L=28 "
                       "in the timed steps, N and m measured on this GPU (MINRES solves at L=16,18,20 "
                       "fitted ~ n^b; eigensolves at L=12)"),
        "config": {"workload": f"L={L} random-field Heisenberg chain, Sz=0 (dim {n}), h={L28_H}, seeds "
                               f"{rank_seeds(rank, world)}, {K} eigenpairs nearest sigma=(Emin+Emax)/2; "
                               f"FP32 MINRES + FP64 refinement, FP64 Lanczos (CGS2); a step = "
                               f"hs_lanczos_eigs with {K} Lanczos steps, each solve capped at {cap} "
                               f"iterations, FP64 certification, twist",
                   "L": L, "K": K, "minres_cap": cap, "minres_tol": args.minres_tol,
                   "precond": "row-norm", "l2": "inputs larger than L2 (one vector 160-321 MB)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "wall_s": e2e_wall, "fixed_s": fixed_e2e},
        "gpu_launches": launches,
        "roofline": roofline,
        "minres_iteration": minres_iter,
        "projection": {"fp32_refine": pj_mix, "fp64": pj_64},
        "fp32_refine_over_fp64": (pj_mix["eigenpairs_per_s"] / pj_64["eigenpairs_per_s"])
        if pj_mix and pj_64 else None,
        "measured_L28": {"fp32_refine": mix, "fp64": f64, "create_sigma_s": create_s,
                         "max_resid_last": recs[-1]["max_resid"] if recs else None},
        "calibration": None if cal is None else {k: cal[k] for k in (
            "L", "fp64", "mixed", "m", "fp64_fit", "mixed_fit")},
        "l16_batch": l16,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "wall_seconds_timed": wall,
    }
    print(json.dumps(line), flush=True)
    if args.detail:
        json.dump({"steps": recs, "fp64_steps": rec64, "calibration": cal}, open(args.detail, "w"))
    if dist is not None:
        dist.destroy_process_group()


def l16_batch(torch, hs, args):
    """One batch of 24 L = 16 realisations of the disorder sweep (h ~ U[0.5, 6]),
    8 eigenpairs each, solved to convergence concurrently (FP64 MINRES)."""
    L, K, B = 16, 8, BATCH
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    budget = max(1, nsm // B)
    out = []

    def solve_one(idx, shares):
        h, seed, hv = realisation(idx, L)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with hs.Chain(L, hv, stream=s) as c:
                shares.start(idx, c)
                try:
                    ev, vecs, res, info = c.eigs(K, minres_tol=args.minres_tol, seed=seed,
                                                 allow_not_converged=True)
                    c.twist(vecs)
                finally:
                    shares.done(idx)
            s.synchronize()
        out.append(info)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    shares = Shares(B, budget, nsm, static=args.static_budget)
    th = [threading.Thread(target=solve_one, args=(i, shares)) for i in range(B)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return {"value": K * B / sec, "unit": UNIT, "seconds": sec, "realisations": B, "K": K,
            "converged": sum(1 for i in out if i["converged"] == K),
            "minres_iters": sum(i["minres_iters"] for i in out)}


def forms_table(torch, hs, inputs):
    """Microseconds per product and per MINRES iteration for each row form
    (block, ten-low-bit and four-low-bit superblock; HS_HV_SB and HS_SB4 select
    them) at L = 24, 26, 28, FP32 and FP64, CUDA events on the current stream."""
    out = {}

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e3

    saved = {k: os.environ.get(k) for k in ("HS_HV_SB", "HS_SB4")}
    try:
        for L in (24, 26, 28):
            with hs.Chain(L, inputs.disorder(L, L28_H, 0), sigma=0.0) as c:
                for name, dt, reps in (("f32", torch.float32, 10), ("f64", torch.float64, 3)):
                    x = torch.randn(c.n, dtype=dt, device="cuda")
                    y = torch.empty_like(x)
                    for form, env in (("block", ("0", "0")), ("sb10", ("1", "0")), ("sb4", ("1", "1"))):
                        os.environ["HS_HV_SB"], os.environ["HS_SB4"] = env
                        for _ in range(2):
                            c.matvec(x, y, shifted=True)
                        out[f"hv L={L} {name} {form}"] = timed(lambda: c.matvec(x, y, shifted=True), reps)
                    del x, y
                os.environ["HS_HV_SB"] = "1"
                b = torch.randn(c.n, dtype=torch.float64, device="cuda")
                for name, lo, hi in (("f32", 20, 120), ("f64", 10, 30)):
                    for form in ("0", "1"):
                        os.environ["HS_SB4"] = form
                        if name == "f32":
                            run = lambda k: c.minres_f32(b.float(), tol=0.0, kmax=k, allow_not_converged=True)
                        else:
                            run = lambda k: c.minres(b, tol=0.0, kmax=k, allow_not_converged=True)
                        t_lo, t_hi = timed(lambda: run(lo), 1), timed(lambda: run(hi), 1)
                        key = "sb4" if form == "1" else "sb10"
                        out[f"minres L={L} {name} pass A {key}"] = (t_hi - t_lo) / (hi - lo)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out


def smem_forms(torch, hs, inputs, L, iters):
    """Microseconds per MINRES iteration (row norm, tolerance 0, `iters`
    iterations in one launch) of the one-reduction (HS_MINRES_PIPE=1) and the
    two-reduction (=0) shared-memory forms, FP64 then FP32, on all SMs, CUDA
    events on the current stream; one launch of each kernel per case."""
    out = {}
    saved = os.environ.get("HS_MINRES_PIPE")
    try:
        with hs.Chain(L, inputs.disorder(L, L28_H, 0), sigma=0.05) as c:
            b = torch.randn(c.n, dtype=torch.float64, device="cuda")
            for name in ("f64", "f32"):
                for form in ("1", "0"):
                    os.environ["HS_MINRES_PIPE"] = form
                    bb = b if name == "f64" else b.float()
                    run = c.minres if name == "f64" else c.minres_f32
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    x, info = run(bb, tol=0.0, kmax=iters, precond="row", allow_not_converged=True)
                    e1.record()
                    torch.cuda.synchronize()
                    key = f"L={L} {name} {'one' if form == '1' else 'two'}-reduction"
                    out[key] = {"us_per_iter": e0.elapsed_time(e1) * 1e3 / info["iters"],
                                "form": info["form"]}
    finally:
        if saved is None:
            os.environ.pop("HS_MINRES_PIPE", None)
        else:
            os.environ["HS_MINRES_PIPE"] = saved
    return out


def sweep_case(torch, hs, args):
    """One hs_sweep call over the C3-recipe realisations (h ~ U[0.5, 6],
    h_j ~ U[-h, h]; the same realisations as the 24-stream batch), K = 8,
    FP64 inner solves to --minres-tol: eigenpairs per second of the whole call
    and of its rounds, with the schedule the library chose."""
    n16, n18 = (int(v) for v in args.sweep.split(","))
    K = 8
    Ls, hl = [], []
    for L, cnt in ((16, n16), (18, n18)):
        for idx in range(cnt):
            Ls.append(L)
            hl.append(realisation(idx, L)[2])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, res, z, zz, info = hs.sweep(Ls, hl, K, minres_tol=args.minres_tol)
    sec = time.perf_counter() - t0
    return {"value": K * len(Ls) / sec, "unit": UNIT, "seconds": sec,
            "eigenpairs_per_s_rounds": K * len(Ls) / info["seconds_solve"],
            "realisations": {"16": n16, "18": n18}, "K": K,
            "max_resid": float(res.max()), "info": info}


def run_only(args):
    """Single-kernel cases for profiler captures."""
    import torch

    from paper_2203_09732_gb300 import hs, inputs
    torch.cuda.set_device(0)
    if args.only == "forms":
        print(json.dumps(forms_table(torch, hs, inputs)))
        return
    if args.only == "smem":
        print(json.dumps(smem_forms(torch, hs, inputs, args.L, args.minres_iters)))
        return
    if args.only == "sweep":
        out = {"sweep": sweep_case(torch, hs, args)}
        n16 = int(args.sweep.split(",")[0])
        if n16 == BATCH and int(args.sweep.split(",")[1]) == 0:
            out["streams_24"] = l16_batch(torch, hs, args)
        print(json.dumps(out))
        return
    if args.only == "hv":
        rf = hv_roofline(torch, hs, args.L, torch.cuda.current_stream())
        print(json.dumps({k: {"GB/s": v["bytes"] / v["seconds"] / 1e9, "us": v["seconds"] * 1e6}
                          for k, v in rf.items()}))
        return
    # a fixed shift (no extremal Lanczos), so that a profiler's launch list
    # holds the solve's kernels only
    with hs.Chain(args.L, inputs.disorder(args.L, L28_H, 0), sigma=0.05) as c:
        b = torch.randn(c.n, dtype=torch.float64, device="cuda")
        b /= b.norm()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info = c.minres(b, tol=0.0, kmax=args.minres_iters, mixed=True, allow_not_converged=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    print(json.dumps({"L": args.L, "iters": info["iters"], "us_per_iter": dt / info["iters"] * 1e6}))


def main():
    args = parse()
    if args.only:
        run_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
