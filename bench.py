#!/usr/bin/env python
"""Throughput of the IMEX time step (Mgridpoint-steps/s = n_r * n_phi * steps / s).

Default workload (large_n2049_p6144): n_r = 2049, n_phi = 6144 (N_m = 2048,
N_c = 1365), E = 1e-8, Pr = 1, Ra = 20 Ra_c, radius ratio 0.35, Chebyshev
integration / tau, SBDF3, dt = 1e-10, FP64, seeded initial temperature
perturbation of amplitude 1e-3 -- the largest single-GPU configuration.  The
same line carries the mixed-precision form of the same workload (FP32 explicit
stage, FP64 solves and history) with its distance from the FP64 path.
--workload selects another (sparse_n257_p768: n_r = 257, ARS443;
coll_n257_p768: the same problem in the collocation formulation; batch64: 64
uneven runs in one CUDA graph; ...).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload W]

Timing: W untimed steps, then K steps, each bracketed by CUDA events on the
library's stream, with a 256 MiB write between steps to flush the 129 MB L2
(outside the events).  A second pass of K steps records events around every
kernel launch for the per-kernel (roofline) numbers.  The end-to-end figure
times set_state (pinned host buffers) + step + get_state per step.
Multi-GPU (torchrun): independent replicas, one per rank; value = all ranks'
grid-point-steps / max time over ranks.  --shard slabs instead splits one run
over the ranks by the m-slab decomposition (NCCL all-to-alls inside the step;
strong scaling), and checks the decomposed step bitwise against the whole one.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1902_07092_gb300 import inputs  # noqa: E402

METRIC = "Mgridpoint-steps/s (n_r*n_phi*steps/s), FP64 vs mixed/batched at <=1e-6 rel err"
UNIT = "Mgridpoint-steps/s"
# GB300 FP64 from unit counts and clock: 152 SMs x 2 DFMA/clk (ncu's
# sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 304/cycle)
# x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
KERNELS = ("spec_to_grid", "phi_products", "grid_to_spec", "solve")


def critical_rayleigh(E):
    """Ra_c from the oracle's table; between tabulated E, log-log interpolation."""
    t = json.load(open(os.path.join(ROOT, "tests", "golden", "critical_rayleigh.json")))
    key = "%g" % E
    if key in t:
        return t[key]["Ra_c"]
    pts = sorted((float(k), v["Ra_c"]) for k, v in t.items())
    for (e0, r0), (e1, r1) in zip(pts, pts[1:]):
        if e0 <= E <= e1:
            f = (math.log(E) - math.log(e0)) / (math.log(e1) - math.log(e0))
            return math.exp(math.log(r0) + f * (math.log(r1) - math.log(r0)))
    raise KeyError("no critical Rayleigh number for E = %g" % E)


# ----------------------------------------------------------- flop counts ----
def algorithmic_flops(n_r, n_phi, scheme, radial="integration"):
    """FP64 flops per launch of each kernel (formulas and unit counts in the design
    notes): a complex FFT of length L counts 5 L log2 L, a complex-data DCT-I of
    K+1 points 5 K log2 K (a length-K complex FFT), a banded apply 2 flops per
    real x complex tap pair, the unpivoted band solve its multiply-adds; the
    collocation solve 8 flops per complex x complex and 4 per real x complex
    inverse entry."""
    K = n_r - 1
    M = n_phi // 3 + 1
    if radial == "collocation":
        dct = 5.0 * K * math.log2(K)
        fft = 5.0 * n_phi * math.log2(n_phi)
        f_s2g = M * (2 * dct + 20.0 * n_r)
        f_phi = n_r * (4 * fft + 8.0 * n_phi)
        f_g2s = M * (4 * dct + 40.0 * n_r)
        nterms = 6
        f_solve = M * (20.0 * n_r * (n_r - 2) + nterms * 3 * 4.0 * n_r)
        return dict(zip(KERNELS, (f_s2g, f_phi, f_g2s, f_solve)))
    nc = (2 * (n_r - 1)) // 3
    dct = 5.0 * K * math.log2(K)
    fft = 5.0 * n_phi * math.log2(n_phi)
    f_s2g = M * (4 * dct + 40.0 * n_r)
    f_phi = n_r * (4 * fft + 8.0 * n_phi)
    band = lambda h: 4.0 * (2 * h + 1) * nc            # real band x complex vector
    f_g2s = M * (6 * dct + 30.0 * n_r + band(8) + 2 * band(4))
    np_, nt = nc - 4, nc - 2
    if radial == "galerkin":
        # pivoted band sweeps: 8 + 20 complex multiply-adds per Psi row (8 flops),
        # 4 + 10 real x complex per temperature row (4 flops); the basis expansion
        solve_psi = np_ * (8 + 20 + 1) * 8.0 + 4.0 * 5 * nc
        solve_th = nt * (4 + 10 + 1) * 4.0 + 4.0 * 2 * nc
    else:
        solve_psi = np_ * (8 * 8 + 8 * 8 + 6) + 4 * 4 * np_ + 4 * 8 * np_   # LU sweeps + Schur
        solve_th = nt * (4 * 4 + 4 * 4 + 2) + 2 * 4 * nt + 2 * 4 * nt
    epi = band(8) * 2 + band(6) * 3 + band(8) + band(4) + 2 * band(2)
    f_solve = M * (solve_psi + solve_th + 6 * 8.0 * nc + epi)
    return dict(zip(KERNELS, (f_s2g, f_phi, f_g2s, f_solve)))


# DRAM bytes (read + write) per launch of the roofline kernel from one ncu capture
# of this workload (summaries under profiles/); null for kernels not captured.
NCU_TRAFFIC = {
    ("sparse_n257_p768", "solve"): (44.36e6 + 0.03e6, "profiles/imex_step_kernels_n257_p768.md"),
    ("large_n2049_p6144", "solve"): (5672.7e6 + 171.6e6, "profiles/imex_step_kernels_n2049_p6144.md"),
    ("large_n2049_p6144", "spec_to_grid"): (106.3e6 + 226.2e6, "profiles/imex_step_kernels_n2049_p6144.md"),
    ("large_n2049_p6144", "phi_products"): (269.1e6 + 216.3e6, "profiles/imex_step_kernels_n2049_p6144.md"),
    ("large_n2049_p6144", "grid_to_spec"): (360.1e6 + 71.0e6, "profiles/imex_step_kernels_n2049_p6144.md"),
    ("coll_n257_p768", "solve"): (735.4e6 + 6.9e6, "profiles/collocation_step_kernels_n257_p768.md"),
    ("galerkin_n257_p768", "solve"): (34.58e6 + 0.003e6, "profiles/galerkin_step_kernels_n257_p768.md"),
}


def launches_per_step(scheme):
    return {"CNAB2": 4, "SBDF2": 4, "SBDF3": 4, "ARS443": 16, "BPR353": 13}[scheme]


# --------------------------------------------------------------- clocks -----
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 4 + i and r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------ oracle arm ----
def oracle_kind(wl):
    if wl.get("radial") == "collocation":
        return "oracle.collocation: dense grid-valued inverses"
    if wl.get("radial") == "galerkin":
        return "oracle.galerkin: LAPACK banded LU of the Galerkin systems"
    return "oracle.banded: band-stored operators, Appendix A bordered solves with a banded LU"


def oracle_sample(wl, Ra, budget_s, max_steps):
    """Time the oracle (as it stands) on the workload: steps until budget_s.
    Returns (steps, seconds, set-up seconds, average busy cores), the last from
    the process's CPU time over the wall time of the timed steps."""
    from oracle.banded import BandedIntegrationStepper
    from oracle.collocation import CollocationStepper
    from oracle.galerkin import GalerkinStepper
    from oracle import schemes
    n_r, n_phi = wl["n_r"], wl["n_phi"]
    nc = inputs.n_c_of(wl)
    t0 = time.perf_counter()
    th = inputs.theta_init(n_r, n_phi, wl["amp"], wl["seed"], cfg=wl["cfg"], n_c=nc)
    z, zu = inputs.zero_state(n_r, n_phi, n_c=nc)
    if wl.get("radial") == "collocation":
        st = CollocationStepper(n_r, n_phi, wl["E"], Ra, wl["Pr"], wl["eta"], wl["scheme"], wl["dt"])
        st.set_state(z, z.copy(), th, zu)
    else:
        cls = GalerkinStepper if wl.get("radial") == "galerkin" else BandedIntegrationStepper
        st = cls(n_r, n_phi, wl["E"], Ra, wl["Pr"], wl["eta"], wl["scheme"], wl["dt"])
        st.set_state(z, th, zu)
    if hasattr(st, "lu"):
        for g in schemes.implicit_weights(wl["scheme"]):   # every factorisation (set-up, untimed)
            st.lu(g)
    st.step()                                  # first step (start-up; untimed)
    setup = time.perf_counter() - t0
    n, t = 0, 0.0
    r0 = os.times()
    while n < max_steps and (t < budget_s or n == 0):
        a = time.perf_counter()
        st.step()
        t += time.perf_counter() - a
        n += 1
    r1 = os.times()
    busy = ((r1.user - r0.user) + (r1.system - r0.system)) / max(t, 1e-9)
    return n, t, setup, round(busy, 1)


def max_over_ranks(x, world, device=None):
    """Largest value of x over the ranks of the default process group (x on a
    single rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(gridpoints, steps, world, total_ms):
    """Whole-job throughput in Mgridpoint-steps/s: every rank advances its own
    replica by ``steps`` steps; the job takes the slowest rank's time."""
    return world * gridpoints * steps / (total_ms / 1e3) / 1e6


def cores_used():
    """Threads the oracle's numpy/scipy can use: the BLAS/OpenMP pools (when
    threadpoolctl is there), else the CPU count, capped by the thread-count
    variables of the environment."""
    try:
        from threadpoolctl import threadpool_info
        n = max([p.get("num_threads", 1) for p in threadpool_info()] + [1])
    except Exception:
        n = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var, "")
        if v.isdigit() and int(v) > 0:
            n = min(n, int(v))
    return n


def run_reference(args, wl, Ra, rank):
    if rank != 0:
        return
    per_step_budget = 150.0 / max(args.steps + args.warmup, 1)
    n, t, setup, busy = oracle_sample(wl, Ra, budget_s=min(150.0, per_step_budget * args.steps),
                                      max_steps=args.steps)
    gp = wl["n_r"] * wl["n_phi"]
    val = gp * n / t / 1e6
    sample = ("%d of %d requested steps of the full %s workload (oracle set-up, factorisation and first step "
              "%.1f s untimed; %s; %d BLAS threads available)" % (n, args.steps, args.workload, setup,
                                                                 oracle_kind(wl), cores_used()))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "warmup": 1, "ms_per_step": 1e3 * t / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, wl, Ra),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": busy, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(args, wl, Ra):
    return {"workload": args.workload, "n_r": wl["n_r"], "n_phi": wl["n_phi"], "N_m": wl["n_phi"] // 3,
            "N_c": inputs.n_c_of(wl), "E": wl["E"], "Ra": Ra, "Ra_over_Ra_c": wl["ra_factor"],
            "Pr": wl["Pr"], "radius_ratio": wl["eta"], "scheme": wl["scheme"], "dt": wl["dt"],
            "radial": {"collocation": "chebyshev-collocation", "galerkin": "chebyshev-integration-galerkin"}.get(
                wl.get("radial"), "chebyshev-integration-tau"),
            "l2": "flushed (256 MiB write) between timed steps",
            "parallelism": "replicas" if args.gpus > 1 else "single",
            "precision": ("fp64 throughout (the oracle)" if getattr(args, "impl", "native") == "reference" else
                          precision_label(wl) if getattr(args, "precision", "fp64") == "fp64"
                          else "mixed: FP32 explicit stage, FP64 state/history/couplings/solves")}


def precision_label(wl):
    """What the FP64 path computes in which arithmetic (double-float: pairs of
    FP32 words, ~48-bit significands, on the FP32 pipe)."""
    big = wl["n_r"] >= 513 and wl.get("radial", "integration") == "integration"
    nc = inputs.n_c_of(wl)
    parts = ["fp64: state, history, stored grid values, linear couplings, banded applies, "
             "Schur steps, residuals and refinements in FP64" + ("" if big else "; field arithmetic at each "
                                                                 "radius in FP64"),
             "azimuthal FFTs and products in double-float with the m = 0 means of the products in FP64"]
    if big:
        parts.append("radial DCT-I, derivative scans and field arithmetic at each radius in double-float "
                     "(lean layout, n_r >= 513)")
    if wl.get("radial", "integration") == "integration" and nc > 64:
        parts.append("block chains of the streamfunction solve in double-float (N_c > 64)")
    if nc > 600:
        parts.append("temperature solves by FP32 chains with two FP64-residual corrections (N_c > 600)")
    return "; ".join(parts)


# ------------------------------------------------------------ native arm ----
def mixed_error(args, B, wl, Ra, sol, th, z, zu):
    """Relative L2 distance of the mixed-precision state from an FP64 twin started
    from the same state, after each of min(steps, 50) steps."""
    ref = B.Solver(wl["n_r"], wl["n_phi"], wl["E"], Ra, wl["Pr"], wl["eta"], wl["scheme"], wl["dt"],
                   radial=wl.get("radial", "integration"))
    sol.set_state(th, z, zu)
    ref.set_state(th, z, zu)
    errs, bad = [], []
    for k in range(min(args.steps, 50)):
        sol.step(1)
        ref.step(1)
        a = np.concatenate([np.ravel(x) for x in sol.get_state()])
        b = np.concatenate([np.ravel(x) for x in ref.get_state()])
        if not (np.all(np.isfinite(a)) and np.all(np.isfinite(b))):
            bad.append([k + 1, bool(np.all(np.isfinite(a))), bool(np.all(np.isfinite(b)))])
        errs.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
    ref.close()
    out = {"per_step_max": float(np.max(errs)), "final": errs[-1], "steps": len(errs),
           "against": "FP64 GPU path (parity-tested against the oracle) from the same state"}
    if bad:
        out["nonfinite"] = bad[:5]  # [step, mixed finite, FP64 finite]
    return out


def adjoint_cost(args, B, wl, Ra, sol, th, z, zu):
    """Discrete adjoint of a CNAB2 run of args.steps steps (J = time-averaged
    Nusselt number): wall time of the taped forward run and of the checkpointed
    reverse sweep (which recomputes the forward states segment by segment)."""
    import torch
    K = args.steps
    every = int(wl.get("checkpoint_every", 20))
    w = sol.nusselt_weights()
    g = np.zeros((sol.M, sol.n_c), np.complex128)
    g[0] = w / K
    g = torch.from_numpy(g).cuda()  # the objective's gradient, resident like the state
    sol.set_state(th, z, zu)
    sol.tape_begin(every)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sol.step(K)
    B.pizza_synchronize(sol.ctx)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    for i in range(K):
        dRa = sol.adjoint_step(g_theta=g, want_dRa=(i == K - 1))
    B.pizza_synchronize(sol.ctx)
    t_rev = time.perf_counter() - t0
    return {"steps": K, "checkpoint_every": every, "forward_ms_per_step": 1e3 * t_fwd / K,
            "reverse_ms_per_step": 1e3 * t_rev / K, "reverse_over_forward": t_rev / t_fwd,
            "dJ_dRa": dRa, "objective": "J = (1/K) sum_n (Nu_n - 1)",
            "timing": "wall clock, synchronised, inputs and the objective's gradient resident; dJ/dRa read after "
                      "the last step; reverse includes the segment recomputation"}


def run_batch(args, wl, rank, world, local_rank):
    """64 independent CNAB2 runs of uneven sizes advanced args.steps steps by one
    CUDA graph (pizza_batch_step), each context autotuned first; timed against
    the same contexts stepped one after another."""
    import torch
    from paper_1902_07092_gb300 import binding as B
    torch.cuda.set_device(local_rank)
    runs = inputs.batch_runs(wl["batch"])
    sols, states = [], []
    t0 = time.perf_counter()
    for r in runs:
        Ra = r["ra_factor"] * critical_rayleigh(r["E"])
        s = B.Solver(r["n_r"], r["n_phi"], r["E"], Ra, r["Pr"], r["eta"], r["scheme"], r["dt"])
        th = inputs.theta_init(r["n_r"], r["n_phi"], r["amp"], r["seed"] + 1000 * rank, cfg=r["cfg"])
        z, zu = inputs.zero_state(r["n_r"], r["n_phi"])
        s.set_state(th, z, zu)
        s.step(1)                      # factor set-up outside the timing
        sols.append(s)
        states.append((th, z, zu))
    setup_s = time.perf_counter() - t0
    tuned = [s.autotune() for s in sols]
    K = args.steps if args.steps_given else wl["steps"]
    gp_steps = sum(r["n_r"] * r["n_phi"] for r in runs) * K
    # plain: one context after another
    for s, st in zip(sols, states):
        s.set_state(*st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in sols:
        s.step(K)
        B.pizza_synchronize(s.ctx)
    plain_s = time.perf_counter() - t0
    # one graph for all runs: capture + first launch, then the timed relaunch
    batch = B.Batch(sols)
    for s, st in zip(sols, states):
        s.set_state(*st)
    t0 = time.perf_counter()
    batch.step(K)
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t0
    for s, st in zip(sols, states):
        s.set_state(*st)
    torch.cuda.synchronize()
    stream = torch.cuda.ExternalStream(batch.stream)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        a.record(stream)
        batch.step(K)
        b.record(stream)
        torch.cuda.synchronize()
    graph_ms = a.elapsed_time(b)
    graph_ms = max_over_ranks(graph_ms, world, torch.device("cuda", local_rank))
    finite = all(np.all(np.isfinite(x)) for s in sols for x in s.get_state())
    if rank == 0:
        line = {"metric": METRIC, "value": world * gp_steps / (graph_ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": 1, "ms_per_step": graph_ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "batch64", "runs": len(runs), "scheme": "CNAB2", "radial": "chebyshev-integration-tau",
                           "sizes": "n_r in {65,129,257,513} x n_phi in {192,384,768,1536}, seeds 1000..1063",
                           "l2": "working set of all runs larger than L2 (no flush)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "batch": {"graph_ms": graph_ms, "plain_ms": 1e3 * plain_s, "speedup_vs_plain": 1e3 * plain_s / graph_ms,
                          "capture_and_first_launch_ms": 1e3 * capture_s, "setup_s": setup_s,
                          "autotuned": sorted(set(map(tuple, tuned))), "finite": bool(finite),
                          "timing": "CUDA events on the batch stream around one graph launch of all runs"},
                "e2e": {"value": gp_steps / plain_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0, "note": "plain: contexts stepped one after another"},
                "gpu_launches": launches_per_step("CNAB2") * K * len(runs),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    batch.close()
    for s in sols:
        s.close()


def algorithmic_bytes(n_r, n_phi, scheme, radial="integration"):
    """HBM bytes per launch of each kernel that a fused pipeline must move (the
    grid stays on chip inside a kernel; formulas in the design notes):
    a1 reads 2 spectral fields and writes 4 radius-major grid fields, 16 B each;
    a2 reads 4 and writes 4 grid fields; a3 reads 4 grid fields, the 2 spectral
    state fields for its linear couplings and writes 2 spectral fields; the solve
    reads its right-hand-side terms and factors and writes the new state and its
    mass (and implicit) terms: 32 B per (m, n) per vector pair (Psi, theta), the
    paper's bordered factor storage 16 x 33 B (Psi) + 8 x 17 B (theta) per (m, n).
    Multistep counts are the steady-state ones; DIRK counts average the stages."""
    M = n_phi // 3 + 1
    if radial == "collocation":
        nc = n_r
        f_solve = M * (16 * 2 * n_r * (n_r - 2) + 8 * n_r * (n_r - 2) + 32 * 6 * n_r)
        return dict(zip(KERNELS, (16.0 * M * (2 * nc + 4 * n_r), 16.0 * 8 * M * n_r, 16.0 * M * (4 * n_r + 2 * nc),
                                  float(f_solve))))
    nc = (2 * (n_r - 1)) // 3
    terms_out = {"CNAB2": (4, 3), "SBDF2": (4, 2), "SBDF3": (6, 2), "ARS443": (4.5, 1.5), "BPR353": (5.0, 1.5)}[scheme]
    per_mn = 32.0 * (terms_out[0] + terms_out[1]) + 16 * 33 + 8 * 17
    return dict(zip(KERNELS, (16.0 * M * (2 * nc + 4 * n_r), 16.0 * 8 * M * n_r, 16.0 * M * (4 * n_r + 4 * nc),
                              per_mn * M * nc)))


def measure_context(args, B, sol, stream, flush, world, dev, barrier, local_rank):
    """W warm-up steps, K timed steps (events around each step, L2 flushed between
    steps), then K steps with events around every launch."""
    import torch
    for _ in range(args.warmup):
        sol.step(1)
    torch.cuda.synchronize()

    def timed_pass(profile):
        evs = []
        if profile:
            B.pizza_profile_begin(sol.ctx, 0xF)
        for _ in range(args.steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sol.step(1)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        prof = B.pizza_profile_end(sol.ctx) if profile else None
        return sum(a.elapsed_time(b) for a, b in evs), prof

    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        total_ms, _ = timed_pass(False)
    barrier()
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms, world, dev)
    _, (kt, kn) = timed_pass(True)
    return total_ms, kt, kn, clk.summary()


def e2e_rate(args, B, sol, gp):
    """set_state from pinned host buffers + one step + get_state into them, per step."""
    import torch
    M, nc = sol.M, sol.n_c
    h_th = torch.empty((M, nc), dtype=torch.complex128, pin_memory=True).numpy()
    h_ps = torch.empty((M, nc), dtype=torch.complex128, pin_memory=True).numpy()
    h_u = torch.empty(nc, dtype=torch.float64, pin_memory=True).numpy()
    B.pizza_get_state(sol.ctx, h_th, h_ps, h_u)
    k_e2e = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        B.pizza_set_state(sol.ctx, h_th, h_ps, h_u, nc)
        B.pizza_step(sol.ctx, 1)
        B.pizza_get_state(sol.ctx, h_th, h_ps, h_u)
    e2e_s = time.perf_counter() - t0
    nbytes = 2 * M * nc * 16 + nc * 8
    return {"value": gp * k_e2e / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": k_e2e}


def kernel_table(kt, kn, flops, nbytes, hbm_peak):
    share = {k: float(kt[i]) / max(float(kt.sum()), 1e-30) for i, k in enumerate(KERNELS)}
    out = {}
    for i, k in enumerate(KERNELS):
        us = 1e3 * float(kt[i]) / max(int(kn[i]), 1)
        out[k] = {"launches": int(kn[i]), "avg_us": us, "share": share[k], "gflop_per_launch": flops[k] / 1e9,
                  # FP64-grade algorithmic flops per second, whichever pipe ran them
                  # (the double-float transforms and chains run on the FP32 pipe)
                  "tflops_algorithmic": flops[k] / (us * 1e-6) / 1e12 if us > 0 else None,
                  "mb_per_launch": nbytes[k] / 1e6,
                  "hbm_frac": nbytes[k] / (us * 1e-6) / 1e9 / hbm_peak if us > 0 else None}
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_native(args, wl, Ra, rank, world, local_rank):
    import torch
    from paper_1902_07092_gb300 import binding as B
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n_r, n_phi = wl["n_r"], wl["n_phi"]
    gp = n_r * n_phi
    radial = wl.get("radial", "integration")
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    # FP64 FMA rate measured here, with the clocks sampled during the probe
    with ClockSampler(local_rank) as pclk:
        fp64_meas, fp64_ms = B.pizza_fp64_fma_rate(40000)
    pclk = pclk.summary()

    # a dedicated stream: the library launches, the L2 flush and the timing events
    # all go to it (torch's default stream handle is 0, which the library reads
    # as "use your own stream")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    nc = inputs.n_c_of(wl)
    th = inputs.theta_init(n_r, n_phi, wl["amp"], wl["seed"] + 1000 * rank, cfg=wl["cfg"], n_c=nc)
    z, zu = inputs.zero_state(n_r, n_phi, n_c=nc)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def make(precision):
        s = B.Solver(n_r, n_phi, wl["E"], Ra, wl["Pr"], wl["eta"], wl["scheme"], wl["dt"], radial=radial)
        if precision == "mixed":
            B.pizza_set_option(s.ctx, "precision", 1)
        B.pizza_set_stream(s.ctx, stream.cuda_stream)
        s.set_state(th, z, zu)
        return s

    sol = make(args.precision)
    total_ms, kt, kn, clocks = measure_context(args, B, sol, stream, flush, world, dev, barrier, local_rank)
    e2e = e2e_rate(args, B, sol, gp)
    mixed = None
    want_mixed = (args.precision == "fp64" and radial == "integration" and not wl.get("adjoint")
                  and not args.no_mixed)
    if want_mixed:
        mix = make("mixed")
        m_ms, m_kt, m_kn, m_clk = measure_context(args, B, mix, stream, flush, world, dev, barrier, local_rank)
        m_e2e = e2e_rate(args, B, mix, gp)
        err = mixed_error(args, B, wl, Ra, mix, th, z, zu)
        mixed = {"value": job_value(gp, args.steps, world, m_ms), "unit": UNIT, "ms_per_step": m_ms / args.steps,
                 "speedup_vs_fp64": total_ms / m_ms, "e2e": m_e2e, "error_vs_fp64": err, "clocks": m_clk,
                 "precision": "FP32 explicit stage (radial transforms, azimuthal FFTs, products); FP64 state, "
                              "history, linear couplings, boundary rows and solves",
                 "kernels": {k: {"avg_us": 1e3 * float(m_kt[i]) / max(int(m_kn[i]), 1),
                                 "share": float(m_kt[i]) / max(float(m_kt.sum()), 1e-30)}
                             for i, k in enumerate(KERNELS)}}
        mix.close()
    err = mixed_error(args, B, wl, Ra, sol, th, z, zu) if args.precision == "mixed" else None
    adj = adjoint_cost(args, B, wl, Ra, sol, th, z, zu) if wl.get("adjoint") else None

    if rank != 0:
        sol.close()
        return
    value = job_value(gp, args.steps, world, total_ms)
    flops = algorithmic_flops(n_r, n_phi, wl["scheme"], radial)
    nbytes = algorithmic_bytes(n_r, n_phi, wl["scheme"], radial)
    kernels = kernel_table(kt, kn, flops, nbytes, hbm_peak)
    dom = max(range(4), key=lambda i: kt[i])
    kd = KERNELS[dom]
    avg_s = float(kt[dom]) / max(int(kn[dom]), 1) / 1e3
    achieved = flops[kd] / avg_s / 1e12
    traffic = NCU_TRAFFIC.get((args.workload, kd), (None, None))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": config_of(args, wl, Ra),
        "e2e": e2e,
        "gpu_launches": launches_per_step(wl["scheme"]) * args.steps,
        "roofline": {"bound": "alu", "kernel": kd, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "frac_of_measured_fp64": achieved / fp64_meas,
                     "traffic": traffic[0], "traffic_source": traffic[1],
                     "peak_source": "FP64 unit count x max SM clock (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz); "
                                    "MEASURED_PEAKS.json has no FP64 figure",
                     "timing": "CUDA events around each launch, second pass of the same K steps"},
        "roofline_hbm": {"bound": "hbm", "kernel": kd, "achieved": nbytes[kd] / avg_s / 1e9, "peak": hbm_peak,
                         "unit": "GB/s", "frac": nbytes[kd] / avg_s / 1e9 / hbm_peak,
                         "algorithmic_bytes": nbytes[kd], "peak_source": hbm_src + ", of measured"},
        "fp64_peak_measured": {"tflops": fp64_meas, "ms": fp64_ms, "clocks": pclk,
                               "tflops_at_max_clock": (fp64_meas * 2070.0 / pclk["sm_mhz"]
                                                       if pclk.get("sm_mhz") else None),
                               "how": "pizza_fp64_fma_rate: 8 independent FMA chains x 2048 threads per SM, "
                                      "one launch timed with CUDA events"},
        "kernels": kernels,
        "clocks": clocks,
    }
    if mixed is not None:
        line["mixed"] = mixed
    if err is not None:
        line["error_vs_fp64"] = err
    if adj is not None:
        line["adjoint"] = adj
    if not args.no_cpu_baseline and world == 1:
        n, t_cpu, setup, busy = oracle_sample(wl, Ra, budget_s=args.cpu_budget, max_steps=1000)
        line["cpu_baseline"] = {"value": gp * n / t_cpu / 1e6, "unit": UNIT, "cores": busy,
                                "kind": "oracle",
                                "sample": "%d full step(s) of the workload on the host CPU (%.1f s; set-up, "
                                          "factorisation and first step %.1f s untimed; %s; cores = average "
                                          "busy cores, of %d BLAS threads)" % (n, t_cpu, setup, oracle_kind(wl),
                                                                              cores_used())}
    print(json.dumps(line), flush=True)
    sol.close()


def run_slabs(args, wl, Ra, rank, world, local_rank):
    """One run of the workload split over the ranks by the m-slab decomposition
    (Section 5): each rank advances its slab of modes and transforms its slab of
    radii, two NCCL all-to-alls per explicit evaluation.  Total work is fixed as
    the rank count grows: strong scaling."""
    import torch
    import torch.distributed as dist
    from paper_1902_07092_gb300 import binding as B
    from paper_1902_07092_gb300.slabs import DistTransport, Plan, SlabSolver
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n_r, n_phi = wl["n_r"], wl["n_phi"]
    gp = n_r * n_phi
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    nc = inputs.n_c_of(wl)
    th = inputs.theta_init(n_r, n_phi, wl["amp"], wl["seed"], cfg=wl["cfg"], n_c=nc)
    z, zu = inputs.zero_state(n_r, n_phi, n_c=nc)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def make():
        s = B.Solver(n_r, n_phi, wl["E"], Ra, wl["Pr"], wl["eta"], wl["scheme"], wl["dt"])
        B.pizza_set_stream(s.ctx, stream.cuda_stream)
        s.set_state(th, z, zu)
        return s

    sol = make()
    plan = Plan(sol.M, n_r, world, rank)
    slab = SlabSolver(sol, plan, DistTransport(), dev)
    total_ms, kt, kn, clocks = measure_context(args, B, sol, stream, flush, world, dev, dist.barrier, local_rank)
    if slab.error:
        raise RuntimeError(slab.error)
    # the decomposed step against the whole step on one context: two steps from
    # the initial state, this rank's modes compared bit for bit
    sol.set_state(th, z, zu)
    sol.step(2)
    mine = sol.get_state()
    ref = make()
    ref.step(2)
    whole = ref.get_state()
    ref.close()
    m0, m1 = plan.m_range
    same = all(np.array_equal(a[m0:m1], b[m0:m1]) for a, b in zip(mine[:2], whole[:2]))
    if m0 == 0:
        same = same and np.array_equal(mine[2], whole[2])
    ok = torch.tensor([1.0 if same else 0.0], device=dev)
    dist.all_reduce(ok, op=dist.ReduceOp.MIN)
    if rank == 0:
        flops = algorithmic_flops(n_r, n_phi, wl["scheme"])
        nbytes = algorithmic_bytes(n_r, n_phi, wl["scheme"])
        peaks = measured_peaks()
        line = {
            "metric": METRIC, "value": gp * args.steps / (total_ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_of(args, wl, Ra), parallelism="m-slabs x%d" % world,
                           slabs={"modes": plan.ms, "radii": plan.ks}),
            "gpu_launches": launches_per_step(wl["scheme"]) * args.steps,
            "kernels": kernel_table(kt, kn, flops, nbytes, float(peaks.get("hbm_gbs", 6800.0))),
            "slabs": {"bitwise_equal_to_whole_step": bool(ok.item() == 1.0),
                      "exchange": "torch.distributed all_to_all_single (NCCL), two per explicit evaluation, "
                                  "inside the step through pizza_set_slab's callback",
                      "rank0_kernels_note": "kernel times of rank 0's slab"},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    slab.close()
    sol.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="large_n2049_p6144", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision record")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "slabs"],
                    help="replicas: one run per rank (weak scaling); slabs: one run split over the ranks "
                         "by the m-slab decomposition (strong scaling)")
    args = ap.parse_args()
    args.steps_given = args.steps is not None
    if args.steps is None:
        args.steps = 100 if inputs.WORKLOADS[args.workload]["n_r"] < 1025 else 20
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    wl = inputs.WORKLOADS[args.workload]
    if wl.get("batch"):
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle has no batched mode; "
                                  "its per-run rate is the cpu_baseline of the single-run workloads"}))
            return
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        run_batch(args, wl, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    Ra = wl["ra_factor"] * critical_rayleigh(wl["E"])
    if args.impl == "reference":
        run_reference(args, wl, Ra, rank)
        return
    if args.shard == "slabs":
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29541")
        os.environ.setdefault("NCCL_DEBUG", "WARN")  # keep stdout to the one JSON line
        dist.init_process_group("nccl", rank=rank, world_size=world)
        run_slabs(args, wl, Ra, rank, world, local_rank)
        dist.destroy_process_group()
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_native(args, wl, Ra, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
