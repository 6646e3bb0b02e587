"""Benchmark: treecode BEM solve of the ~40k-panel synthetic protein on one B300.

One step = one pass of the whole hot path on the synthetic globular protein
(2,000 atoms, ~40k panels, K = 3 Gauss points, theta = 0.5, Taylor order 6,
ncrit 300, FP32-mixed, GMRES tol 1e-4): geometry, Morton octree, interaction
lists, near-singular corrections, right-hand side, device GMRES with one
treecode matrix-vector product per iteration, reaction potential and
solvation energy.  Inputs are resident in device memory when the timed region
starts (pb_add_surface / pb_set_charges copy them to HBM); L2 is flushed
between steps.

Metric: matvec Ginteractions/s = direct (P2P) target-source pairs evaluated
by all matvecs of the timed steps / timed device time.  The solve time, the
per-phase matvec times, the FP64 treecode solve on the same GPU and the
mixed-vs-FP64 energy error are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the plain FP64 CPU oracle (dense matrix-free C/OpenMP
operator) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import datetime
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matvec Ginteractions/s & solve time to 1e-4 ΔG err: batched FP32-mixed vs FP64"
WORKLOAD = "synthetic globular protein, 2000 atoms, ~40k panels, K=3, theta=0.5, P=6, ncrit=300"
PARAMS = dict(K=3, K_fine=19, N_k=5, thres=2.0, P=6, theta=0.5, ncrit=300, gmres_tol=1e-4, restart=50,
              max_iter=1000)
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_LANES_PER_SM = 128


# ---------------------------------------------------------------- arithmetic counts
def p2p_ops_per_pair(kernels):
    """FP32 and MUFU instructions (each one issue slot) of one P2P pair in the mixed kernel.

    Shared part: 3 differences, r^2 (3), rsqrt (1 MUFU), s*inv (1), d.(x-y) (3),
    kv = rd * inv^3 (3) = 14.  Per Laplace kernel: 2 adds.  Per Yukawa kernel:
    rho, exponent scale, ex2 (1 MUFU), s*e fma, kv*e, 1+kappa*rho, fma = 7.
    """
    return 14 + sum(2 if k == 0.0 else 7 for k in kernels)


def radial_terms(P):
    return sum(((P - a) // 2 + 1) * (a + 1) * (a + 2) // 2 for a in range(P + 1))


def m2p_ops_per_box(P):
    """FP32 and MUFU instructions of one (target, box) evaluation of the fused
    Laplace + Yukawa M2P in radial form at order P (mirrors the kernel).

    u (3), r^2 (3), rsqrt (1), 1/r^2 (1); Laplace radial functions (2 per
    order); rho, exponent and ex2 (3); Yukawa F_0, F_1, kappa^2 (5) and 3 per
    further order; coordinate powers (3 (P - 1)); monomials (one multiply per
    nontrivial factor); two fmas per radial moment (M and D); four fmas per
    order for (V, K) of both kernels.  Loads of the radial moments not counted.
    """
    if P == 0:
        return 3 + 3 + 1 + 1 + 3 + 1 + 2 + 4
    mono = 0
    for a1 in range(P + 1):
        for a2 in range(P + 1 - a1):
            mono += 1 if (a1 and a2) else 0
            mono += sum(1 for a3 in range(P + 1 - a1 - a2) if a3)
    return (3 + 3 + 1 + 1 + 2 * P + 3 + 5 + 3 * (P - 1) + 3 * (P - 1) + mono + 2 * radial_terms(P)
            + 4 * (P + 1))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 20 ms from the start of the run; summary() keeps
    the samples taken between mark_start() and mark_end() (the timed steps)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def __exit__(self, *a):
        if self.proc is None:
            return
        proc, self.proc = self.proc, None
        proc.terminate()
        try:
            out, _ = proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            proc.kill()
            out, _ = proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def _parse(self):
        out = []
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                clk, cmax = float(f[2]), float(f[3])
            except ValueError:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                ts = None   # an unexpected timestamp format: the sample counts as inside the window
            out.append((ts, clk, cmax, f[6:10]))
        return out

    def summary(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        rows = self._parse()
        window = "timed steps"
        def inside(r, lo, hi):
            return r[0] is None or lo is None or (lo <= r[0] <= (hi or r[0]))
        sel = [r for r in rows if inside(r, self.t0, self.t1)]
        if not sel and self.t0 is not None:
            # a timed region shorter than the sampling interval: the last second before it (the warm-up)
            sel = [r for r in rows if inside(r, self.t0 - datetime.timedelta(seconds=1), self.t1)]
            window = "warm-up (no sample fell inside the timed steps)"
        reasons = set()
        for r in sel:
            for name, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(name)
        sm = [r[1] for r in sel]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": sel[-1][2] if sel else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_total": len(rows), "interval_ms": 20,
                "window": window}


# ---------------------------------------------------------------- helpers
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _peaks():
    try:
        with open(MEASURED) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def _traffic_record(kernel_file, kernel_name):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    src = os.path.join(ROOT, "paper_1309_4018_b300", "csrc", kernel_file)
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    for fn in sorted(os.listdir(os.path.join(ROOT, "profiles"))) if os.path.isdir(os.path.join(ROOT, "profiles")) else []:
        if not fn.endswith(".md"):
            continue
        txt = open(os.path.join(ROOT, "profiles", fn)).read()
        if f"kernel: {kernel_name}" not in txt:
            continue
        m = re.search(r"source_sha256: ([0-9a-f]{64})", txt)
        b = re.search(r"dram_bytes_per_launch: ([0-9.eE+]+)", txt)
        if m and b and m.group(1) == digest:
            return float(b.group(1))
    return None


def _problem():
    from synth.configs import protein_problem
    return protein_problem()


def _oracle_golden(d):
    """The oracle's stored energy of the benchmark protein (tests/golden/protein40k.json),
    if the file is there and was made on the same mesh."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "protein40k.json")) as f:
            g = json.load(f)
    except OSError:
        return None
    return g if g["mesh"][0]["n_panels"] == int(d["surfaces"][0]["tris"].shape[0]) else None


FLEET = 64          # ligands of the batched-solve measurement
TRIPLET = (8000, 1500)


def _fleet_member(args):
    """Ligand i: its atoms, its CPU-meshed problem and the single-core meshing time."""
    from synth.configs import fleet_atoms, molecule_problem
    i, n = args
    at = fleet_atoms(i, n)
    t0 = time.perf_counter()
    d = molecule_problem(at["xyz"], at["radius"], at["q"])
    return d, at, time.perf_counter() - t0


def _triplet_member(which):
    from synth.configs import binding_triplet
    return binding_triplet(*TRIPLET)[which]


def _variants(_):
    from synth.configs import model_variants
    return model_variants()


def _batch_inputs():
    """The ligand fleet and the binding triplet, generated in a spawned process pool."""
    import multiprocessing as mp
    from synth.configs import fleet_sizes
    sizes = fleet_sizes(FLEET)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        var = pool.map_async(_variants, [0])
        tri = pool.map_async(_triplet_member, [0, 1, 2])
        fleet = pool.map(_fleet_member, list(enumerate(sizes)))
        triplet = tri.get()
        variants = var.get()[0]
    return fleet, triplet, variants


# ---------------------------------------------------------------- reference arm (CPU oracle)
def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from oracle.cdense import DenseOperator
    d = _problem()
    op = DenseOperator(d, PARAMS)
    n = op.sd[0].n
    ns = n * PARAMS["K"]
    sample = np.linspace(0, n - 1, 2048).astype(np.int64)
    rows = {0: sample}
    x = np.random.default_rng(0).normal(size=op.n)
    cores = len(os.sched_getaffinity(0))
    for _ in range(args.warmup):
        op.apply(x, rows)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        op.apply(x, rows)
        times.append(time.perf_counter() - t0)
    pairs = sample.size * ns
    t = float(np.sum(times))
    value = pairs * args.steps / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Ginteractions/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "panels": n, "sources": ns, "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": "Ginteractions/s", "cores": cores, "kind": "oracle",
                             "sample": f"dense FP64 matrix-free operator rows for {sample.size} of {n} targets "
                                       f"against all {ns} Gauss points, both kernels, per step"},
            "e2e": {"value": value, "unit": "Ginteractions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(d):
    """The oracle (dense FP64 C/OpenMP operator) on a bounded sample, in Ginteractions/s."""
    from oracle.cdense import DenseOperator
    op = DenseOperator(d, PARAMS)
    n = op.sd[0].n
    ns = n * PARAMS["K"]
    sample = np.linspace(0, n - 1, 8192).astype(np.int64)
    x = np.random.default_rng(0).normal(size=op.n)
    op.apply(x, {0: sample[:8]})
    t0 = time.perf_counter()
    op.apply(x, {0: sample})
    t = time.perf_counter() - t0
    value = sample.size * ns / t / 1e9
    out = {"value": value, "unit": "Ginteractions/s",
           "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
           "sample": f"dense FP64 matrix-free operator: {sample.size} of {n} target rows against all {ns} "
                     f"Gauss points, Laplace and Yukawa kernels ({t:.1f} s)"}
    out["one_core"] = _oracle_one_core(512)
    g = _oracle_golden(d)
    if g:
        # one operator application per GMRES iteration plus one per cycle start
        applications = g["iterations"] + (g["iterations"] + PARAMS["restart"] - 1) // PARAMS["restart"] + 1
        out["full_solve"] = {
            "recorded_s": g["seconds"], "recorded_cores": g["host_cores"], "gmres_tol": g["gmres_tol"],
            "iterations": g["iterations"],
            "estimated_s_on_these_cores": applications * n * ns / (value * 1e9),
            "note": "setup + GMRES + energy of the dense oracle; recorded when tests/golden/protein40k.json "
                    "was written, estimated here from the sampled all-core rate"}
    return out


_ONE_CORE = r"""
import sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle.cdense import DenseOperator
from synth.configs import protein_problem
op = DenseOperator(protein_problem(), {params!r})
n = op.sd[0].n
rows = np.linspace(0, n - 1, {m}).astype(np.int64)
x = np.random.default_rng(0).normal(size=op.n)
op.apply(x, {{0: rows[:4]}})
t0 = time.perf_counter()
op.apply(x, {{0: rows}})
print(rows.size * n * {K} / (time.perf_counter() - t0) / 1e9)
"""


def _oracle_one_core(m):
    """The oracle's sampled operator rate on one host core (OMP_NUM_THREADS=1, child process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = _ONE_CORE.format(root=ROOT, params=PARAMS, m=m, K=PARAMS["K"])
    try:
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        return {"value": float(p.stdout.strip().splitlines()[-1]), "unit": "Ginteractions/s", "cores": 1,
                "sample": f"{m} target rows against all Gauss points"}
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"value": None, "error": str(e)[:200]}


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    fleet, triplet, variants = _batch_inputs() if args.extras else (None, None, None)
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1309_4018_b300.build import build
    # the clock sampler starts first, so that it is sampling well before the
    # timed steps; its summary keeps the timed steps' samples
    clk = ClockSampler(local).__enter__()
    atexit.register(clk.__exit__, None, None, None)   # the sampler ends with the process whatever happens
    build()
    from paper_1309_4018_b300 import pbbem

    d = _problem()
    surf = d["surfaces"][0]
    ch = d["charges"]
    ctx = pbbem.Context(local)
    stream = torch.cuda.ExternalStream(ctx.stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    def make_problem():
        return pbbem.Problem.from_dict(ctx, d)

    pb = make_problem()
    nsrc = surf["tris"].shape[0] * PARAMS["K"]

    def step(prob):
        prob.setup(precision="mixed", **PARAMS)
        return prob.solve()

    for _ in range(args.warmup):
        r = step(pb)
    # timed steps (device time on the library stream, L2 flushed before each)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    launches0 = pbbem.launch_count()
    _barrier(ws)
    torch.cuda.synchronize()
    clk.mark_start()
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev[i][0].record(stream)
        results.append(step(pb))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk.mark_end()
    clk.__exit__(None, None, None)
    launches = pbbem.launch_count() - launches0
    _barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = _max_over_ranks(float(np.sum(step_ms)) / 1e3, ws)
    r = results[-1]
    pairs_per_step = r.p2p_pairs * r.matvecs
    value = ws * pairs_per_step * args.steps / t_total / 1e9

    # per-phase matvec profile, dominant kernel and its roofline
    x = np.random.default_rng(0).normal(size=pb.n_unknowns)
    prof = pb.profile(x, reps=20)
    peaks, peak_kind = _peaks()
    clocks = clk.summary()
    fmax = float(peaks.get("sm_max_mhz", 2032.0)) * 1e6
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = nsm * FP32_LANES_PER_SM * fmax / 1e12      # FP32 Tinstr/s
    kernels = [d["regions"][0]["kappa"], d["regions"][1]["kappa"]]
    p2p_ops = r.p2p_pairs * p2p_ops_per_pair(kernels)
    m2p_ops = (r.m2p_pairs // 2) * m2p_ops_per_box(PARAMS["P"])
    cand = {"p2p32": (prof["p2p"], p2p_ops), "m2p32": (prof["m2p"], m2p_ops)}
    dom = max(cand, key=lambda k: cand[k][0])
    dom_ms, dom_ops = cand[dom]
    achieved = dom_ops / (dom_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": alu_peak, "unit": "FP32 Tinstr/s",
                "frac": achieved / alu_peak, "peak_source": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                                             f"{fmax / 1e6:.0f} MHz ({peak_kind} sm_max_mhz)",
                "traffic": _traffic_record("treecode.cu", dom),
                "frac_at_measured_clock": (achieved / (alu_peak * clocks["sm_mhz"] * 1e6 / fmax))
                if clocks["sm_mhz"] else None,
                "other": {k: {"ms": v[0], "Tinstr_s": v[1] / (v[0] / 1e3) / 1e12,
                              "frac": v[1] / (v[0] / 1e3) / 1e12 / alu_peak} for k, v in cand.items()}}

    # the M2P contraction on the tensor pipe (pb_params.m2p_variant = 1): phase time and energy (an extra)
    m2p_tc, rtc = None, None
    if args.extras:
        ptc = make_problem()
        ptc.setup(precision="mixed", m2p_variant=1, **PARAMS)
        rtc = ptc.solve()
        prof_tc = ptc.profile(x, reps=20)
        ptc.close()
        m2p_tc = {"m2p_ms": prof_tc["m2p"], "m2p_ms_fp32_pipe": prof["m2p"], "matvec_ms": prof_tc["total"],
                  "dG_kJ_mol": rtc.dG_solv, "iterations": rtc.iterations,
                  "note": "radial-form contraction as mma.sync m16n8k8 TF32 with split operands (3 products), "
                          "FP32 accumulation; monomials, radial functions and final sums on the FP32 pipe"}

    # end to end through the public API with host buffers (H2D inside the timed region),
    # the inputs held in page-locked host memory
    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(np.ascontiguousarray(a)).dtype, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    d_pin = dict(d)
    d_pin["surfaces"] = [dict(sf, verts=pinned(sf["verts"]), tris=pinned(sf["tris"])) for sf in d["surfaces"]]
    d_pin["charges"] = dict(d["charges"], xyz=pinned(d["charges"]["xyz"]), q=pinned(d["charges"]["q"]))
    e2e_t = []
    # untimed new problems first, as many as the device warm-up steps (the first fills the allocator's cache)
    for i in range(max(1, args.warmup)):
        p2 = pbbem.Problem.from_dict(ctx, d_pin)
        step(p2)
        p2.close()
    for i in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = pbbem.Problem.from_dict(ctx, d_pin)
        r2 = step(p2)
        e2e_t.append(time.perf_counter() - t0)
        p2.close()
    h2d = surf["verts"].size * 8 + surf["tris"].size * 4 + ch["xyz"].size * 8 + ch["q"].size * 8
    cycles = (r2.iterations + PARAMS["restart"] - 1) // PARAMS["restart"] + 1
    d2h = 8 * (2 + cycles + r2.iterations)
    e2e_val = ws * r2.p2p_pairs * r2.matvecs / float(np.mean(e2e_t)) / 1e9

    # The metric's second half: the plain FP64 treecode on the same GPU at the
    # same tolerance (1e-4, equal energy error: the same tree, lists and
    # truncation), timed like the mixed steps; the oracle's energy decides
    # whether both meet the 1e-4 bar.  The FP64 solve at tol 1e-8 is kept as a
    # separately labelled extra.
    mixed_s = t_total / args.steps
    p64 = make_problem()
    step64 = lambda: (p64.setup(precision="fp64", **PARAMS), p64.solve())[1]
    step64()
    t64 = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        r64 = step64()
        t64.append((r64.setup_ms + r64.solve_ms) / 1e3)
    p64.setup(precision="fp64", **dict(PARAMS, gmres_tol=1e-8))
    r64t = p64.solve()
    p64.close()
    rel_err = abs(r.dG_solv - r64t.dG_solv) / abs(r64t.dG_solv)
    golden = _oracle_golden(d)
    dG_or = golden["dG"] if golden else None
    rel_or = (lambda e: abs(e - dG_or) / abs(dG_or)) if golden else (lambda e: None)
    if m2p_tc is not None:
        m2p_tc["dG_rel_err_vs_oracle"] = rel_or(rtc.dG_solv)

    extras = {}
    if args.extras:
        extras = _extras(pbbem, ctx, pb, r, d, fleet, triplet, variants)

    if rank == 0:
        cpu = cpu_baseline(d)
        line = {
            "metric": METRIC, "value": value, "unit": "Ginteractions/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "panels": int(surf["tris"].shape[0]), "sources": nsrc,
                       "charges": int(ch["q"].size), "precision": "FP32-mixed (Krylov, near field, energy FP64)",
                       "gmres_tol": PARAMS["gmres_tol"], "l2": "flushed (256 MB write) before every step",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "solve_time_s": r.solve_ms / 1e3 + r.setup_ms / 1e3,
            "setup_ms": r.setup_ms, "gmres_ms": r.solve_ms, "iterations": r.iterations, "matvecs": r.matvecs,
            "dG_kJ_mol": r.dG_solv, "dG_rel_err_vs_fp64": rel_err, "dG_rel_err_vs_oracle": rel_or(r.dG_solv),
            "oracle": {"dG_kJ_mol": dG_or, "gmres_tol": golden["gmres_tol"] if golden else None,
                       "source": "tests/golden/protein40k.json (dense FP64 oracle, GMRES, written by "
                                 "tests/golden/make_golden.py)" if golden else "missing"},
            "p2p_pairs_per_matvec": r.p2p_pairs, "m2p_evals_per_matvec": r.m2p_pairs,
            "matvec_phase_ms": prof,
            "matvec_gint_per_s": r.p2p_pairs / (prof["total"] / 1e3) / 1e9,
            "dense_equivalent_gint_per_s": surf["tris"].shape[0] * nsrc / (prof["total"] / 1e3) / 1e9,
            "fp64": {"solve_time_s": float(np.mean(t64)), "iterations": r64.iterations,
                     "gmres_tol": PARAMS["gmres_tol"], "dG_kJ_mol": r64.dG_solv,
                     "dG_rel_err_vs_oracle": rel_or(r64.dG_solv), "mixed_solve_time_s": mixed_s,
                     "speedup_mixed_vs_fp64": float(np.mean(t64)) / mixed_s,
                     "meets_1e-4_vs_oracle": {"mixed": rel_or(r.dG_solv) is not None and rel_or(r.dG_solv) <= 1e-4,
                                              "fp64": rel_or(r64.dG_solv) is not None and rel_or(r64.dG_solv) <= 1e-4},
                     "extra_tol_1e-8": {"solve_time_s": (r64t.solve_ms + r64t.setup_ms) / 1e3,
                                        "iterations": r64t.iterations, "dG_kJ_mol": r64t.dG_solv,
                                        "dG_rel_err_vs_oracle": rel_or(r64t.dG_solv)}},
            "roofline": roofline, "cpu_baseline": cpu, "m2p_tensor_pipe": m2p_tc,
            "e2e": {"value": e2e_val, "unit": "Ginteractions/s", "inputs": "page-locked host memory",
                    "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "seconds_per_step": float(np.mean(e2e_t))},
            "gpu_launches": int(launches), "clocks": clocks,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_phases(reps, m2p_variant=0):
    """One setup and solve of the workload, then `reps` operator applications timed phase by phase."""
    from paper_1309_4018_b300.build import build
    build()
    from paper_1309_4018_b300 import pbbem
    d = _problem()
    ctx = pbbem.Context(0)
    pb = pbbem.Problem.from_dict(ctx, d)
    pb.setup(precision="mixed", m2p_variant=m2p_variant, **PARAMS)
    r = pb.solve()
    x = np.random.default_rng(0).normal(size=pb.n_unknowns)
    print(json.dumps({"setup_ms": r.setup_ms, "solve_ms": r.solve_ms, "phases_ms": pb.profile(x, reps=reps)}))


def _extras(pbbem, ctx, pb, r, d, fleet_members, triplet, variants):
    """Adjoint gradient of the bench problem, a batched fleet solve, a binding energy, a
    Richardson study, the model variants, an accuracy/time sweep and device surface generation."""
    fleet = [f[0] for f in fleet_members]
    t0 = time.perf_counter()
    g1 = pb.gradient()
    first = time.perf_counter() - t0
    g = pb.gradient()
    q = d["charges"]["q"]
    grad = {"workload": WORKLOAD, "grad_ms": g["grad_ms"], "first_call_ms": 1e3 * first,
            "solve_ms": r.solve_ms + r.setup_ms, "adjoint_iterations": g["iterations"],
            "q_dq_over_2E": float(q @ g["dq"]) / (2 * r.dG_solv),
            "dE_deps": g["deps"].tolist(), "dE_dkappa": g["dkappa"].tolist()}
    probs = [pbbem.Problem.from_dict(ctx, f) for f in fleet]
    for p in probs:
        p.setup(precision="mixed", **PARAMS)
    pbbem.solve_batch(ctx, probs)
    ts = time.perf_counter()
    seq = [p.solve() for p in probs]
    t_seq = time.perf_counter() - ts
    ts = time.perf_counter()
    bat = pbbem.solve_batch(ctx, probs)
    t_bat = time.perf_counter() - ts
    # the same batch as one persistent launch per GMRES step (the opt-in path)
    ctx.set_option(pbbem.PB_OPT_BATCH_PERSISTENT, 1)
    pbbem.solve_batch(ctx, probs)
    ts = time.perf_counter()
    bat_p = pbbem.solve_batch(ctx, probs)
    t_bat_p = time.perf_counter() - ts
    ctx.set_option(pbbem.PB_OPT_BATCH_PERSISTENT, 0)
    pairs = sum(x.p2p_pairs * x.matvecs for x in bat)
    panels = [int(f["surfaces"][0]["tris"].shape[0]) for f in fleet]
    batch = {"workload": f"{FLEET} synthetic ligands, 300-3000 atoms, {min(panels)}-{max(panels)} panels",
             "panels_total": int(sum(panels)), "sequential_s": t_seq, "batch_s": t_bat,
             "speedup_batch_vs_sequential": t_seq / t_bat, "ginteractions_per_s": pairs / t_bat / 1e9,
             "same_energies": all(a.dG_solv == b.dG_solv for a, b in zip(seq, bat)),
             "mode": "per-problem device-driven GMRES cycle graphs on 8 pool streams",
             "persistent_launch_s": t_bat_p,
             "speedup_persistent_vs_default": t_bat / t_bat_p,
             "same_energies_persistent": all(a.dG_solv == b.dG_solv for a, b in zip(seq, bat_p))}
    for p in probs:
        p.close()
    batch["autotuned"] = _autotuned_fleet(pbbem, ctx, fleet, bat)
    batch["mixed_vs_fp64"] = _batched_fp64(pbbem, ctx, fleet[:16])
    tri = [pbbem.Problem.from_dict(ctx, t) for t in triplet]
    ts = time.perf_counter()
    for p in tri:
        p.setup(precision="mixed", **PARAMS)
    ddG = pbbem.binding_energy(ctx, *tri)
    t_bind = time.perf_counter() - ts
    binding = {"workload": f"receptor {TRIPLET[0]} atoms, ligand {TRIPLET[1]} atoms, complex",
               "panels": [int(t["surfaces"][0]["tris"].shape[0]) for t in triplet], "ddG_kJ_mol": ddG,
               "setup_and_solve_s": t_bind}
    for p in tri:
        p.close()
    from paper_1309_4018_b300.richardson import study
    from synth.configs import sphere_problem
    spheres = [sphere_problem(level=l, charges="both") for l in (3, 4, 5)]
    st = study(spheres, 4.0, ctx, precision="fp64", theta=0.4, P=10, ncrit=100, gmres_tol=1e-10)
    rich = {"workload": "Kirkwood sphere r=4 A, charges at 0 and 2 A, 512/2048/8192 panels, FP64 treecode "
                        "(the tests compare the extrapolation with the closed form)",
            "energies": st.energies, "observed_order": st.order, "extrapolated": st.extrapolated,
            "solve_s": st.solve_s}
    names = list(variants)
    vp = [pbbem.Problem.from_dict(ctx, variants[k]) for k in names]
    ts = time.perf_counter()
    for p in vp:
        p.setup(precision="mixed", **PARAMS)
    vr = pbbem.solve_batch(ctx, vp)
    t_var = time.perf_counter() - ts
    models = {"workload": "2000-atom molecule with two 3 A solvent cavities and a 2 A Stern layer "
                          "(Single / Cavity / Stern / Full models)",
              "panels": {k: int(sum(s["tris"].shape[0] for s in variants[k]["surfaces"])) for k in names},
              "dG_kJ_mol": {k: x.dG_solv for k, x in zip(names, vr)},
              "iterations": {k: x.iterations for k, x in zip(names, vr)}, "setup_and_batch_solve_s": t_var}
    for p in vp:
        p.close()
    from paper_1309_4018_b300.pareto import pareto_front, sweep
    # reference: every knob at its most accurate setting on the same mesh
    best = dict(PARAMS, precision="mixed", K=7, K_fine=19, thres=4.0, theta=0.3, P=10, gmres_tol=1e-7)
    ref_pb = pbbem.Problem.from_dict(ctx, d)
    ref_pb.setup(**best)
    ref = ref_pb.solve().dG_solv
    ref_pb.close()
    grid = []
    for theta, P in ((0.7, 3), (0.6, 4), (0.5, 6), (0.4, 8)):
        for tol in (1e-3, 1e-4, 1e-6):
            grid.append((f"theta={theta} P={P} tol={tol:g}", d,
                         dict(PARAMS, precision="mixed", theta=theta, P=P, gmres_tol=tol)))
    for k, v in (("K", 1), ("K", 7), ("K_fine", 3), ("K_fine", 7), ("thres", 0.5), ("thres", 1.0),
                 ("thres", 4.0), ("no_precond", 1)):
        grid.append((f"theta=0.5 P=6 tol=0.0001 {k}={v}", d, dict(PARAMS, precision="mixed", **{k: v})))
    res = sweep(grid, ref, ctx)
    pareto = {"workload": WORKLOAD.split(",")[0] + ", same mesh; base K=3 K_fine=19 thres=2; reference: "
                                                   "K=7 K_fine=19 thres=4 theta=0.3 P=10 tol 1e-7",
              "reference_dG_kJ_mol": ref,
              "cases": [{"label": c.label, "time_s": c.time_s, "rel_error": c.rel_error,
                         "iterations": c.iterations} for c in res],
              "front": [c.label for c in pareto_front(res)]}
    surface = _surface_extra(pbbem, ctx, fleet_members)
    from synth.configs import large_protein_problem
    dl = large_protein_problem()
    ts = time.perf_counter()
    pl = pbbem.Problem.from_dict(ctx, dl)
    info = pl.surface_info(0)
    pl.setup(precision="mixed", **PARAMS)
    rl = pl.solve()
    gl = pl.gradient()
    t_large = time.perf_counter() - ts
    ql = dl["charges"]["q"]
    large = {"workload": "30,000-atom synthetic globule, surface meshed on the device at 0.8 A "
                         "(the tests check 32 sampled coordinates and eps/kappa against central differences)",
             "panels": info["nt"], "mesh_ms": info["gen_ms"], "setup_ms": rl.setup_ms, "solve_ms": rl.solve_ms,
             "iterations": rl.iterations, "dG_kJ_mol": rl.dG_solv, "grad_ms": gl["grad_ms"],
             "adjoint_iterations": gl["iterations"], "q_dq_over_2E": float(ql @ gl["dq"]) / (2 * rl.dG_solv),
             "wall_s": t_large}
    pl.close()
    return {"gradient": grad, "batch": batch, "binding": binding, "richardson": rich, "model_variants": models,
            "pareto": pareto, "surface": surface, "large_gradient": large}


def _batched_fp64(pbbem, ctx, ligands):
    """Batched solve time to the 1e-4 energy bar: setup + pb_solve_batch of the same
    ligands in FP32-mixed and in plain FP64 at the same tolerance, tree and lists
    (so the same truncation error), wall time after one untimed round each."""
    def run(prec):
        t = None
        for _ in range(2):
            probs = [pbbem.Problem.from_dict(ctx, f) for f in ligands]
            ts = time.perf_counter()
            for p in probs:
                p.setup(precision=prec, **PARAMS)
            res = pbbem.solve_batch(ctx, probs)
            t = time.perf_counter() - ts
            for p in probs:
                p.close()
        return t, res

    tm, rm = run("mixed")
    t64, r64 = run("fp64")
    return {"workload": f"the first {len(ligands)} ligands of the fleet "
                        f"({sum(int(f['surfaces'][0]['tris'].shape[0]) for f in ligands)} panels)",
            "gmres_tol": PARAMS["gmres_tol"], "mixed_setup_and_batch_s": tm, "fp64_setup_and_batch_s": t64,
            "speedup_mixed_vs_fp64": t64 / tm,
            "iterations_mixed": [x.iterations for x in rm], "iterations_fp64": [x.iterations for x in r64],
            "max_rel_dG_diff_mixed_vs_fp64": float(max(abs(a.dG_solv - b.dG_solv) / abs(b.dG_solv)
                                                       for a, b in zip(rm, r64)))}


def _autotuned_fleet(pbbem, ctx, fleet, default_results):
    """The fleet with (theta, P, ncrit) from the autotuner's per-size-class schedule, against the
    configuration's fixed setting: setup + batched solve wall time and the energies."""
    from paper_1309_4018_b300.autotune import Schedule
    base = {k: v for k, v in PARAMS.items() if k not in ("theta", "P", "ncrit")}
    base["precision"] = "mixed"
    t0 = time.perf_counter()
    sched = Schedule.build(ctx, fleet, target=1e-4, base=base)
    t_tune = time.perf_counter() - t0

    def run(tuned):
        probs = [pbbem.Problem.from_dict(ctx, f) for f in fleet]
        ts = time.perf_counter()
        for p, f in zip(probs, fleet):
            p.setup(**(dict(base, **sched.params_for(f)) if tuned else dict(PARAMS, precision="mixed")))
        res = pbbem.solve_batch(ctx, probs)
        t = time.perf_counter() - ts
        for p in probs:
            p.close()
        return t, res

    run(True)
    t_tuned, res = run(True)
    t_def, _ = run(False)
    return {"schedule": {str(k): dict(c.params(), rel_error=c.rel_error, time_s=c.time_s)
                         for k, c in sched.choices.items()},
            "tuning_s": t_tune, "setup_and_batch_s_tuned": t_tuned, "setup_and_batch_s_default": t_def,
            "speedup": t_def / t_tuned,
            "max_rel_dG_diff_vs_default": float(max(abs(a.dG_solv - b.dG_solv) / abs(b.dG_solv)
                                                    for a, b in zip(res, default_results)))}


def _surface_extra(pbbem, ctx, fleet_members):
    """Device surface generation: the protein's mesh on the GPU against the CPU mesher, and the
    ligand fleet's pipeline from atoms (GPU meshes, setup, batched solve) against the same
    pipeline fed with CPU meshes."""
    from synth.configs import PROTEIN_SPACING, protein_atoms
    from synth.molecule import gaussian_surface
    at = protein_atoms(2000, 2)
    t0 = time.perf_counter()
    _, t_cpu = gaussian_surface(at["xyz"], at["radius"], PROTEIN_SPACING)
    t_cpu_mesh = time.perf_counter() - t0
    gen = []
    for _ in range(5):
        p = pbbem.Problem(ctx)
        p.add_region(4.0, 0.0)
        p.add_region(80.0, 0.125)
        sid = p.add_gaussian_surface(at["xyz"], at["radius"], 0, 1, spacing=PROTEIN_SPACING)
        info = p.surface_info(sid)
        gen.append(info["gen_ms"])
        p.close()
    prot = {"workload": f"2,000-atom synthetic protein, {PROTEIN_SPACING} A grid", "panels_gpu": info["nt"],
            "panels_cpu_mesher": int(t_cpu.shape[0]), "gpu_ms_median": float(np.median(gen)),
            "cpu_mesher_s_one_core": t_cpu_mesh, "speedup": t_cpu_mesh / (float(np.median(gen)) / 1e3),
            "grid": list(info["grid"]), "rounds": info["rounds"]}

    def pipeline(from_atoms):
        probs = []
        ts = time.perf_counter()
        for dd, a, _ in fleet_members:
            if from_atoms:
                p = pbbem.Problem(ctx)
                for reg in dd["regions"]:
                    p.add_region(reg["eps"], reg["kappa"])
                p.add_gaussian_surface(a["xyz"], a["radius"], 0, 1, spacing=PROTEIN_SPACING)
                p.set_charges(a["xyz"], a["q"], 0)
            else:
                p = pbbem.Problem.from_dict(ctx, dd)
            p.setup(precision="mixed", **PARAMS)
            probs.append(p)
        res = pbbem.solve_batch(ctx, probs)
        t = time.perf_counter() - ts
        for p in probs:
            p.close()
        return t, [x.dG_solv for x in res]

    pipeline(True)
    t_gpu, e_gpu = pipeline(True)
    t_up, e_up = pipeline(False)
    mesh_core = float(sum(m[2] for m in fleet_members))
    fleet_out = {"workload": f"{len(fleet_members)} synthetic ligands from atoms, {PROTEIN_SPACING} A grid",
                 "gpu_pipeline_s": t_gpu, "uploaded_cpu_meshes_pipeline_s": t_up,
                 "cpu_mesher_s_one_core_total": mesh_core,
                 "cpu_pipeline_s_one_core": mesh_core + t_up,
                 "speedup_vs_cpu_meshing_one_core": (mesh_core + t_up) / t_gpu,
                 "max_rel_dG_diff_gpu_vs_cpu_meshes": float(max(abs(a - b) / abs(b) for a, b in zip(e_gpu, e_up)))}
    return {"protein": prot, "fleet": fleet_out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the gradient, batched-fleet and binding-energy measurements")
    ap.add_argument("--phases", type=int, default=0, metavar="R",
                    help="only set up and solve the workload once, then time R operator applications phase by "
                         "phase (pb_profile_operator) and print them: a short run for profilers")
    ap.add_argument("--m2p-variant", type=int, default=0, help="with --phases: pb_params.m2p_variant")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.phases:
        run_phases(args.phases, args.m2p_variant)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
