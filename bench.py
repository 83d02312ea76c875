"""Benchmark: SM-AMG preconditioned Wilson-Dirac solves on one B300 (or N replicas).

Workload (one "step" = one pass of the whole solve path over one batch of
synthetic input): a 256x256 lattice, quenched U(1) gauge field at beta = 6
(Metropolis, 500 sweeps from a cold start, seed 2); three bare masses
m0 = m_crit + {0.1, 0.02, 0.005}, each with its own resident 3-level hierarchy
(tile sides 4 then 2, coarsest 32x32 solved by its FP64 inverse); per step one
Gaussian right-hand side per mass, FGMRES(30) to a true relative residual of
1e-10.  Setup is timed separately.  Between steps the L2 cache is flushed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AM-AMG solves/s at 1e-10 rel. residual, mixed vs FP64; D-apply GB/s; p50/p99"
L = 256
BETA = 6.0
FIELD_SEED = 2
SWEEPS = 500
MASS_OFFSETS = [0.1, 0.02, 0.005]
AGGS = [4, 2]
RESTART = 30
TOL = 1e-10
RHS_SEED0 = 1000
FP64_PEAK_GFLOPS = 1250.0      # nominal B300 FP64 rate
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# FP64 level-1 coarse Gauss-Seidel (k_coarse_sweeps_owner<double>, two sweeps of
# a 64x64 level with 21 offsets, the shape of this workload's level 1), from one
# ncu capture of that kernel on the smooth1 probe; set to None when that kernel
# changes
COARSE_SMOOTH_F64_DRAM_BYTES = 5818368
WORKLOAD = ("256x256 Wilson-Dirac (periodic x, antiperiodic t), quenched U(1) beta=6 seed 2, "
            "m0 = m_crit + {0.1, 0.02, 0.005}, 3-level SM-AMG (tiles 4, 2), FGMRES(30) to 1e-10, 1 RHS per mass")


def arm_config(world):
    """The workload description both arms print."""
    return {"workload": WORKLOAD, "lattice": f"{L}x{L}", "levels": 3, "tiles": AGGS, "restart": RESTART,
            "tol": TOL, "rhs_per_mass": 1, "masses": len(MASS_OFFSETS), "parallelism": f"replicas x{world}",
            "l2": "flushed (256 MB write) between steps"}


def replica_rhs_seed(rank: int, i: int) -> int:
    """Seed of the i-th right-hand side of replica `rank` (replicas solve their own)."""
    return RHS_SEED0 + 100000 * rank + i


def reduce_over_ranks(total_ms: float, solves_per_rank: int, world: int, dev):
    """Whole-job throughput of `world` replicas: the slowest rank's timed
    milliseconds (an all-reduce MAX; the only collective, off the data path)
    and every rank's solves over that time.  Returns (max_ms, solves/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, solves_per_rank * world / (total_ms * 1e-3)


def load_mcrit():
    path = os.path.join(ROOT, "tests", "golden", "mcrit.json")
    table = json.load(open(path))
    return table[f"L{L}_b{BETA:g}_s{FIELD_SEED}"]["m_crit"]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


# ----------------------------------------------------------------------------- reference arm (oracle)

def oracle_hierarchy(theta, m0):
    from oracle import amg
    from oracle import wilson as W
    from paper_2608_03515_b300 import fixtures as fx
    D = W.dirac_matrix(fx.links_from_angles(theta), m0)
    t0 = time.perf_counter()
    levels = amg.build_hierarchy(D, L, L, AGGS)
    return D, levels, time.perf_counter() - t0


def oracle_solve(D, levels, psi_flat):
    from oracle import amg, krylov
    t0 = time.perf_counter()
    res = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), psi_flat, RESTART, TOL, 3000)
    return time.perf_counter() - t0, res


def run_reference(args):
    """The oracle on this arm's workload: the three masses' hierarchies, and
    per timed step one solve, step i on mass i mod 3 with its own right-hand
    side; the solves/s of the 1:1:1 mix (the work of one GPU step per three
    solves) is 3 / sum over masses of the mean solve time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import wilson as W
    from paper_2608_03515_b300 import fixtures as fx
    theta = fx.metropolis_u1(L, L, BETA, SWEEPS, FIELD_SEED)
    mcrit = load_mcrit()
    hiers, setup_s = [], 0.0
    for d in MASS_OFFSETS:
        D, levels, s_ = oracle_hierarchy(theta, mcrit + d)
        hiers.append((D, levels))
        setup_s += s_
    nm = len(MASS_OFFSETS)
    timed_n = max(args.steps, nm)
    for i in range(args.warmup):           # warm-up: the cheapest mass
        oracle_solve(*hiers[0], W.to_flat(fx.gaussian_rhs(1, L, L, RHS_SEED0 + i)[0]))
    per_mass = [[] for _ in range(nm)]
    iters = []
    for i in range(timed_n):
        k = i % nm
        psi = W.to_flat(fx.gaussian_rhs(1, L, L, RHS_SEED0 + args.warmup + i)[0])
        dt, res = oracle_solve(*hiers[k], psi)
        per_mass[k].append(dt)
        iters.append(res.iterations)
    step_s = sum(float(np.mean(t)) for t in per_mass)     # one solve of every mass
    value = nm / step_s
    sample = (f"oracle (FP64 NumPy/SciPy, sparse kernels single-threaded) solves of all {nm} masses, "
              f"{timed_n} timed solves (solve i on mass i mod {nm}) after {args.warmup} warm-up solves; "
              f"value = {nm} / sum of the per-mass mean solve times; setup {setup_s:.1f} s excluded")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(args.gpus),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "iterations": iters,
        "mean_solve_s_per_mass": [round(float(np.mean(t)), 3) for t in per_mass],
    }))


# ----------------------------------------------------------------------------- kernel probe

def run_probe(args):
    """A small, self-contained case of one kernel family, e.g. for an ncu capture:
    random-phase links on an L x L lattice, tiles 4 then 2 (4, 4, 2 from 1024 up)."""
    import torch
    from paper_2608_03515_b300 import build as _b
    _b.build()
    from paper_2608_03515_b300 import amamg as A
    dev = torch.device("cuda:0")
    Lp = args.lattice
    rng = np.random.Generator(np.random.PCG64(5))
    U = torch.from_numpy(np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Lp, Lp)))).to(dev)
    aggs = [int(a) for a in args.tiles.split(",")] if args.tiles else ([4, 4, 2] if Lp >= 1024 else [4, 2])
    prec = A.SOLVE_MIXED if args.prec == "f32" else A.SOLVE_FP64
    h = A.setup(U, 0.1, A.make_params(aggs, precision=prec))
    dt = torch.complex64 if args.prec == "f32" else torch.complex128
    fine = args.probe in ("apply_D", "vcycle", "solve")
    x = torch.randn(args.rhs, 2, Lp, Lp, dtype=dt, device=dev) if fine else None
    y = torch.empty_like(x) if fine else None
    nt1, nx1, _ = h.level_info(1)
    r1 = torch.randn(args.rhs, 2, nt1, nx1, dtype=dt, device=dev)
    e1 = torch.zeros_like(r1)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for rep in range(args.reps + 1):
        if rep == 1:
            ev[0].record(stream)
        if args.probe == "apply_D":
            A.apply_D(h, x, y)
        elif args.probe == "vcycle":
            A.vcycle(h, x, y)
        elif args.probe == "smooth1":
            A.smooth(h, 1, r1, e1, 2)
        elif args.probe == "coarse_apply":
            A.apply_coarse(h, 1, r1, e1)
        elif args.probe in ("coarsest", "coarsest_f32"):
            nt, nx, _ = h.level_info(len(aggs))
            cdt = torch.complex64 if args.probe == "coarsest_f32" else torch.complex128
            xc = torch.randn(args.rhs, 2, nt, nx, dtype=cdt, device=dev)
            A.coarsest_apply(h, xc, torch.empty_like(xc))
        else:
            A.solve(h, x.to(torch.complex128), torch.empty(x.shape, dtype=torch.complex128, device=dev))
    ev[1].record(stream)
    torch.cuda.synchronize()
    print(json.dumps({"probe": args.probe, "lattice": Lp, "rhs": args.rhs, "prec": args.prec,
                      "ms_per_rep": ev[0].elapsed_time(ev[1]) / max(args.reps, 1)}))


# ----------------------------------------------------------------------------- wirebasket-size spread

# (tile sides, edge ownership, normalisation): the wirebasket size with the
# method's readings, then the two other readings at the benchmark's tile sides
SPREAD = ([[4, 2], "tile", "none"], [[2, 2, 2], "tile", "none"], [[4, 4], "tile", "none"],
          [[2, 4], "tile", "none"], [[4, 2], "first_lex", "none"], [[4, 2], "tile", "rowsum"],
          [[4, 2], "first_lex", "rowsum"])


def run_spread(dev, U, masses, psi):
    """The benchmark field and masses solved (FP64) with several hierarchies:
    tile sides (the paper's claim that iteration counts depend little on the
    wirebasket size, Sec. 5), edge ownership (Sec. 4.1) and the normalisation
    of Eq. (16); iterations, solve and setup time per hierarchy."""
    import torch
    from paper_2608_03515_b300 import amamg as A
    out = []
    x = torch.empty_like(psi)
    for aggs, own, norm in SPREAD:
        row = {"tiles": aggs, "ownership": own, "normalization": norm, "iterations": [], "solve_ms": [],
               "setup_ms": []}
        for m0 in masses:
            h = A.setup(U, m0, A.make_params(aggs, precision=A.SOLVE_FP64, restart=RESTART, tol=TOL,
                                             ownership=own, normalization=norm))
            row["setup_ms"].append(round(1e3 * A.setup_seconds(h), 1))
            A.solve(h, psi, x)                                   # warm-up (graphs)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(torch.cuda.current_stream())
            info = A.solve(h, psi, x)
            ev[1].record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            row["iterations"].append(info[0].iterations)
            row["solve_ms"].append(round(ev[0].elapsed_time(ev[1]), 2))
            row.setdefault("converged", []).append(bool(info[0].status == A.OK and info[0].true_relres <= TOL))
            A.destroy(h)
        out.append(row)
    return out


# ----------------------------------------------------------------------------- serving stream

SERVING_SIZES = (64, 128, 256, 512, 1024)


# 512^2 serving fields without a tabulated critical mass take the 256^2 field of
# the same coupling and seed as reference, moved up by this margin: the largest
# difference between tabulated critical masses of one coupling across 64^2,
# 128^2 and 256^2 is 0.0435 (beta = 2)
SERVING_REF_SIZES = (512,)
SERVING_REF_MARGIN = 0.045


def serving_fields_available():
    """(L, k) -> (beta, mass floor) for the serving fields (beta_k = 2 + 10 k / 7,
    seed 10 + k): the tabulated critical mass, or for the sizes in
    SERVING_REF_SIZES the 256^2 field's plus SERVING_REF_MARGIN."""
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "mcrit.json")))
    out = {}
    for L in SERVING_SIZES:
        for k in range(8):
            beta = round(2.0 + 10.0 * k / 7.0, 12)
            key = f"L{L}_b{beta:g}_s{10 + k}"
            ref = f"L256_b{beta:g}_s{10 + k}"
            if key in table:
                out[(L, k)] = (beta, table[key]["m_crit"])
            elif L in SERVING_REF_SIZES and ref in table:
                out[(L, k)] = (beta, table[ref]["m_crit"] + SERVING_REF_MARGIN)
    return out


def field_angles(Lf, beta, seed):
    """Quenched field of the fixtures (run in a worker process of the field pool)."""
    from paper_2608_03515_b300 import fixtures as fx
    return fx.metropolis_u1(Lf, Lf, beta, SWEEPS, seed)


SERVING_SWEEP_REQUESTS = 300


def run_serving(n_requests, rate, dev, mem_budget, thetas):
    """The serving stream: n_requests Poisson arrivals over the resident fields
    whose critical mass is tabulated (thetas[(L, k)]: futures of their angles)."""
    import torch
    from paper_2608_03515_b300 import fixtures as fx
    from paper_2608_03515_b300 import serving
    avail = serving_fields_available()
    sizes = sorted({L for (L, _) in avail})
    fields, mcrit = {}, {}
    for (L, k), (beta, mc) in avail.items():
        U = torch.from_numpy(fx.links_from_angles(thetas[(L, k)].result())).to(dev)
        fields[(L, k)] = (U, mc + 0.005)            # hierarchy at the lowest serving mass
        mcrit[(L, k)] = mc
    saturated = None
    if rate <= 0:
        # calibration: a saturated burst (all requests at t = 0) measures the service rate
        calib = serving.poisson_requests(min(40, n_requests), 1e9, list(avail), mcrit, seed=99)
        srv = serving.Server(fields, mem_budget)
        c = serving.serve(srv, calib)
        saturated = c["requests_per_s"]
        rate = 0.8 * saturated
    srv = serving.Server(fields, mem_budget)
    reqs = serving.poisson_requests(n_requests, rate, list(avail), mcrit, seed=100)
    out = serving.serve(srv, reqs)
    out.update({"rate_req_per_s": rate, "sizes": sizes, "fields": len(fields),
                "setup_s_total": sum(g.setup_s for g in srv.groups.values()),
                "config": "Poisson arrivals at 0.8 x the calibrated saturated request rate; each request draws "
                          "(L, field) uniformly from the resident fields, m0 = m_crit + U[0.005, 0.1] (512^2: "
                          f"m_crit of the 256^2 field of the same coupling + {SERVING_REF_MARGIN} in place of "
                          "m_crit), R ~ U{1..16}; mixed precision to 1e-10",
                "sizes_missing": [Lm for Lm in SERVING_SIZES if Lm not in sizes]})
    if saturated is not None:
        # load sweep: shorter streams at 0.5 x and 1.0 x the saturated rate, same
        # resident hierarchies (the 0.8 x stream above is the headline)
        sweep = {}
        for frac in (0.5, 1.0):
            n_s = min(SERVING_SWEEP_REQUESTS, n_requests)
            rq = serving.poisson_requests(n_s, frac * saturated, list(avail), mcrit, seed=int(100 + 10 * frac))
            o = serving.serve(srv, rq)
            sweep[f"{frac:g}x"] = {k: o[k] for k in ("requests", "solves_per_s", "requests_per_s", "latency_p50_ms",
                                                     "latency_p99_ms", "not_converged")}
            sweep[f"{frac:g}x"]["rate_req_per_s"] = frac * saturated
        out["load_sweep"] = sweep
        out["saturated_req_per_s"] = saturated
    return out


# ----------------------------------------------------------------------------- many right-hand sides

C4_L, C4_BETA, C4_SEED, C4_DM, C4_AGGS, C4_R, C4_RHS_SEED = 1024, 12.0, 5, 0.01, [4, 4], 64, 6
# the 1024^2 field's own critical mass is not tabulated (the oracle's Arnoldi
# route does not finish on the host in hours); the mass is set from the 256^2
# beta = 12 field's, as in tests/golden/make_c4_oracle.py
C4_MASS_REF = "L256_b12_s17"


def c4_mcrit():
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "mcrit.json")))
    e = table.get(C4_MASS_REF)
    return None if e is None else e["m_crit"]


def time_coarse_apply(A, h, xc, yc, reps=20):
    """CUDA-event time of amamg_apply_coarse on level 1 (3 warm-up calls), with
    the library's algorithmic bytes and FLOPs of the call (profile records)."""
    import torch
    for _ in range(3):
        A.apply_coarse(h, 1, xc, yc)
    A.profile_reset(h)
    A.profile_enable(h, True)
    A.apply_coarse(h, 1, xc, yc)
    A.profile_enable(h, False)
    name, _, _, nbytes, flops = [c for c in A.profile_get(h) if c[0].startswith("coarse_apply")][-1]
    A.profile_reset(h)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        A.apply_coarse(h, 1, xc, yc)
    ev[1].record(stream)
    torch.cuda.synchronize()
    us = 1e3 * ev[0].elapsed_time(ev[1]) / reps
    return {"kernel": name, "us": round(us, 1), "algorithmic_GB/s": round(nbytes / us / 1e3, 1),
            "hbm_frac": round(nbytes / us / 1e3 / measured_peaks()[0], 3),
            "useful_TFLOP/s": round(flops / us / 1e6, 2)}


def run_c4(dev, theta_future):
    """64 right-hand sides on the 1024^2 beta = 12 field at m0 = (critical mass
    of the 256^2 beta = 12 field) + 0.01, 3 levels (tiles 4, 4; coarsest
    64^2 = 8192 unknowns, FP64 inverse, tensor-core apply), mixed
    precision, FGMRES(30) to 1e-10: one warm-up and one timed solve of all 64;
    beside it the plain FP64 form on the first right-hand side alone; and the
    oracle's iteration counts and sampled solution entries for the first four
    (tests/golden/c4_oracle.json, when present)."""
    import torch
    from paper_2608_03515_b300 import amamg as A
    from paper_2608_03515_b300 import fixtures as fx
    mc = c4_mcrit()
    if mc is None:
        return {"skipped": f"reference critical mass {C4_MASS_REF} not tabulated"}
    m0 = mc + C4_DM
    U = torch.from_numpy(fx.links_from_angles(theta_future.result())).to(dev)
    psi = torch.from_numpy(fx.gaussian_rhs(C4_R, C4_L, C4_L, C4_RHS_SEED)).to(dev)
    x = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    out = {"workload": f"{C4_L}x{C4_L} quenched U(1) beta={C4_BETA:g} seed {C4_SEED}, m0 = m_crit(256^2 beta=12) "
                       f"+ {C4_DM}, "
                       f"tiles {C4_AGGS} (coarsest 64^2, FP64 inverse), FGMRES(30) to 1e-10, {C4_R} RHS per call",
           "m0": m0}
    # FP64 Gram-Schmidt in its modified form (one fused stage per basis vector,
    # half the FP64 work of the classical two-pass form; at 64 right-hand sides
    # the stages are bandwidth-sized: 3.00 against 2.27 solves/s)
    h = A.setup(U, m0, A.make_params(C4_AGGS, precision=A.SOLVE_MIXED, restart=RESTART, tol=TOL, autotune=True,
                                     gs_method="mgs"))
    out["setup_ms"] = round(1e3 * A.setup_seconds(h), 1)
    out["smoother_fixed_rule"] = A.query_smoother(h, 1, A.F32, C4_R)
    A.solve(h, psi, x)                                       # warm-up (captures the 64-wide graphs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    info = A.solve(h, psi, x)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    its = [i.iterations for i in info]
    out["mixed_batched"] = {"gram_schmidt": "FP64, modified", "solves_per_s": round(C4_R / (ms * 1e-3), 3),
                            "ms": round(ms, 1),
                            "iterations": {"min": min(its), "max": max(its), "mean": round(float(np.mean(its)), 1)},
                            "true_relres_max": max(i.true_relres for i in info),
                            "all_converged": all(i.status == A.OK for i in info)}
    out["smoother_autotuned"] = A.query_smoother(h, 1, A.F32, C4_R)
    xh = x[:4].cpu().numpy()
    # the level-1 operator (256^2 coarse sites, 21 offsets) applied to the 64
    # right-hand sides: tensor cores (FP16 super-block GEMMs) here, the CUDA-core
    # FP32 kernel on the FP64 handle below (same links, mass, tiles: same operator)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    n1 = C4_L // C4_AGGS[0]
    xc = torch.randn(C4_R, 2, n1, n1, dtype=torch.complex64, device=dev, generator=g)
    yc_tc = torch.empty_like(xc)
    ca_tc = time_coarse_apply(A, h, xc, yc_tc)
    A.destroy(h)
    # the same batch with the opt-in double-float Gram-Schmidt (FP64 Gram-Schmidt
    # bounds the step above)
    hd = A.setup(U, m0, A.make_params(C4_AGGS, precision=A.SOLVE_MIXED, restart=RESTART, tol=TOL, autotune=True,
                                      gs="df64"))
    A.solve(hd, psi, x)
    ev[0].record(stream)
    info_d = A.solve(hd, psi, x)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms_d = ev[0].elapsed_time(ev[1])
    its_d = [i.iterations for i in info_d]
    out["mixed_batched_gs_df64"] = {"gram_schmidt": "double-float, classical with DGKS second pass",
                                    "solves_per_s": round(C4_R / (ms_d * 1e-3), 3), "ms": round(ms_d, 1),
                                    "iterations": {"min": min(its_d), "max": max(its_d),
                                                   "mean": round(float(np.mean(its_d)), 1)},
                                    "true_relres_max": max(i.true_relres for i in info_d),
                                    "all_converged": all(i.status == A.OK for i in info_d)}
    A.destroy(hd)
    del x
    # the plain FP64 form, one right-hand side per call
    h64 = A.setup(U, m0, A.make_params(C4_AGGS, precision=A.SOLVE_FP64, restart=RESTART, tol=TOL))
    yc_cc = torch.empty_like(xc)
    prev = os.environ.get("AMAMG_COARSE_TC")
    os.environ["AMAMG_COARSE_TC"] = "0"                      # read at a level's first apply
    ca_cc = time_coarse_apply(A, h64, xc, yc_cc)
    if prev is None:
        del os.environ["AMAMG_COARSE_TC"]
    else:
        os.environ["AMAMG_COARSE_TC"] = prev
    d = (yc_tc - yc_cc).abs().max().item() / yc_cc.abs().max().item()
    out["coarse_apply_level1"] = {
        "workload": f"level 1 of the {C4_L}^2 hierarchy ({n1}x{n1} coarse sites, 21 offsets), {C4_R} RHS, "
                    "FP32 vectors, Gaussian inputs",
        "tensor_core": ca_tc, "cuda_core": ca_cc,
        "speedup": round(ca_cc["us"] / ca_tc["us"], 2),
        "max_rel_diff_tc_vs_cuda_core": d}
    del xc, yc_tc, yc_cc
    x1 = torch.empty_like(psi[:1])
    A.solve(h64, psi[:1], x1)
    ev[0].record(stream)
    i64 = A.solve(h64, psi[:1], x1)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms64 = ev[0].elapsed_time(ev[1])
    out["fp64_single"] = {"solves_per_s": round(1.0 / (ms64 * 1e-3), 3), "ms": round(ms64, 1),
                          "iterations": i64[0].iterations, "true_relres": i64[0].true_relres}
    out["speedup_mixed_batched_vs_fp64_single"] = round(out["mixed_batched"]["solves_per_s"] /
                                                        out["fp64_single"]["solves_per_s"], 2)
    A.destroy(h64)
    gold = os.path.join(ROOT, "tests", "golden", "c4_oracle.json")
    if os.path.exists(gold) and abs(json.load(open(gold))["m0"] - m0) <= 1e-15:
        g = json.load(open(gold))
        cmp = []
        for row in g["solves"]:
            r = row["rhs"]
            xs = np.array([[complex(*v) for v in site] for site in row["x_at_sites"]])
            xg = np.array([[xh[r][a, t, xx] for a in range(2)] for (t, xx) in g["sites"]])
            cmp.append({"rhs": r, "iterations": its[r], "oracle_iterations": row["iterations"],
                        "sampled_rel_err": float(np.max(np.abs(xg - xs)) / row["x_norm"])})
        out["vs_oracle"] = cmp
    return out


# ----------------------------------------------------------------------------- our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--probe", default=None,
                    choices=["apply_D", "vcycle", "smooth1", "coarse_apply", "solve", "coarsest", "coarsest_f32"],
                    help="time one kernel family on a small random-phase case (for profiler captures)")
    ap.add_argument("--lattice", type=int, default=512)
    ap.add_argument("--tiles", default="", help="probe: tile sides, e.g. 4,4")
    ap.add_argument("--rhs", type=int, default=1)
    ap.add_argument("--prec", default="f64", choices=["f64", "f32"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--serving", type=int, default=2000,
                    help="serving stream of this many requests (continuous batching, mixed precision; 0: skip)")
    ap.add_argument("--no-c4", action="store_true",
                    help="skip the 1024^2, 64-right-hand-side mixed-precision leg")
    ap.add_argument("--no-spread", action="store_true",
                    help="skip the parameter spread (tile sides, edge ownership, normalisation)")
    ap.add_argument("--serving-rate", type=float, default=0.0,
                    help="Poisson arrival rate in requests/s (0: 0.8 x the calibrated saturated rate)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.probe:
        run_probe(args)
        return

    # host-side fixtures of the later legs, generated by a spawned process pool
    # (started before the first CUDA call) while the GPU runs the earlier ones
    import concurrent.futures
    import multiprocessing
    pool = concurrent.futures.ProcessPoolExecutor(max_workers=max(1, min(8, cpu_cores() - 2)),
                                                  mp_context=multiprocessing.get_context("spawn"))
    c4_theta = None
    if not args.no_c4 and c4_mcrit() is not None:
        c4_theta = pool.submit(field_angles, C4_L, C4_BETA, C4_SEED)
    serving_thetas = {}
    if args.serving > 0:
        for (Ls, k), (beta, _) in serving_fields_available().items():
            serving_thetas[(Ls, k)] = pool.submit(field_angles, Ls, beta, 10 + k)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2608_03515_b300 import build as _b
    _b.build()
    from paper_2608_03515_b300 import amamg as A
    from paper_2608_03515_b300 import fixtures as fx

    theta = fx.metropolis_u1(L, L, BETA, SWEEPS, FIELD_SEED)
    U = torch.from_numpy(fx.links_from_angles(theta)).to(dev)
    mcrit = load_mcrit()
    masses = [mcrit + d for d in MASS_OFFSETS]
    nsteps = args.warmup + args.steps
    # right-hand sides resident in HBM before the timed region (replicas draw their own)
    psis = [torch.from_numpy(fx.gaussian_rhs(1, L, L, replica_rhs_seed(rank, i))).to(dev) for i in range(nsteps)]
    x = torch.empty_like(psis[0])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def build_hiers(prec):
        hs, setup_ms = [], []
        for m0 in masses:
            h = A.setup(U, m0, A.make_params(AGGS, precision=prec, restart=RESTART, tol=TOL))
            hs.append(h)
            setup_ms.append(1e3 * A.setup_seconds(h))
        return hs, setup_ms

    def run(hs, nst=None, skip=0):
        """Runs steps; returns per-step device ms (events) and per-solve ms."""
        stream = torch.cuda.current_stream()
        step_ms, solve_ms, iters, relres = [], [], [], []
        for i in range(nst if nst is not None else nsteps):
            flush.zero_()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(hs) + 1)]
            evs[0].record(stream)
            for k, h in enumerate(hs):
                info = A.solve(h, psis[i], x)
                evs[k + 1].record(stream)
                iters.append(info[0].iterations)
                relres.append(info[0].true_relres)
                assert info[0].status == A.OK and info[0].true_relres <= TOL, info
            torch.cuda.synchronize()
            if i >= skip:
                step_ms.append(evs[0].elapsed_time(evs[-1]))
                solve_ms += [evs[k].elapsed_time(evs[k + 1]) for k in range(len(hs))]
        return step_ms, solve_ms, iters, relres

    hs64, setup64 = build_hiers(A.SOLVE_FP64)
    hs32, setup32 = build_hiers(A.SOLVE_MIXED)

    # warm-up, then the timed FP64 region
    run(hs64, nst=args.warmup)
    launches0 = sum(A.launch_count(h) for h in hs64)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    torch.cuda.profiler.start()          # profiler window (ncu --profile-from-start off) = timed region
    t_wall = time.perf_counter()
    # timed steps use the right-hand sides after the warm-up ones
    psis_w = psis
    step_ms, solve_ms, iters64, relres64 = [], [], [], []
    stream = torch.cuda.current_stream()
    for i in range(args.warmup, nsteps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in hs64]
        e0.record(stream)
        prev = e0
        for k, h in enumerate(hs64):
            info = A.solve(h, psis_w[i], x)
            evs[k].record(stream)
            iters64.append(info[0].iterations)
            relres64.append(info[0].true_relres)
            if not (info[0].status == A.OK and info[0].true_relres <= TOL):
                raise RuntimeError(f"solve did not converge: {info}")
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(evs[-1]))
        solve_ms += [(e0 if k == 0 else evs[k - 1]).elapsed_time(evs[k]) for k in range(len(hs64))]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall_s = time.perf_counter() - t_wall
    torch.cuda.profiler.stop()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = sum(A.launch_count(h) for h in hs64) - launches0
    total_ms, value = reduce_over_ranks(float(np.sum(step_ms)), args.steps * len(masses), world, dev)

    # mixed precision on the same inputs
    run(hs32, nst=args.warmup)
    st32, sv32, it32, rr32 = run(hs32, nst=nsteps, skip=args.warmup)
    for r in rr32:
        assert r <= TOL
    mixed_value = len(sv32) / (np.sum(st32) * 1e-3) * world

    # the first timed right-hand side on the m_crit + 0.1 hierarchy, FP64 and
    # mixed, kept for the comparison with the oracle's solution
    A.solve(hs64[0], psis[args.warmup], x)
    x_check64 = x.cpu().numpy()[0].copy()
    A.solve(hs32[0], psis[args.warmup], x)
    x_check32 = x.cpu().numpy()[0].copy()
    errs_vs_oracle = {}

    # multi-RHS batches: R right-hand sides per solve call (mixed precision), all
    # three masses; solves/s counts right-hand sides
    batched = {}
    for Rb in (4, 16):
        psib = [torch.from_numpy(fx.gaussian_rhs(Rb, L, L, RHS_SEED0 + 50000 + 100 * Rb + i)).to(dev)
                for i in range(2)]
        xb = torch.empty_like(psib[0])
        for h in hs32:
            A.solve(h, psib[0], xb)                         # warm-up (captures the R-wide graphs)
        flush.zero_()
        eb = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        eb[0].record(stream)
        its = []
        for h in hs32:
            info = A.solve(h, psib[1], xb)
            its.append(max(i.iterations for i in info))
            assert all(i.status == A.OK and i.true_relres <= TOL for i in info)
        eb[1].record(stream)
        torch.cuda.synchronize()
        ms = eb[0].elapsed_time(eb[1])
        batched[f"R{Rb}"] = {"solves_per_s": round(Rb * len(hs32) / (ms * 1e-3), 3), "ms": round(ms, 2),
                             "max_iterations": its}
        if Rb == 16:
            # the same 16-wide calls with the modified Gram-Schmidt (FP64)
            hs_m = [A.setup(U, m0, A.make_params(AGGS, precision=A.SOLVE_MIXED, restart=RESTART, tol=TOL,
                                                 gs_method="mgs")) for m0 in masses]
            for h in hs_m:
                A.solve(h, psib[0], xb)
            flush.zero_()
            eb[0].record(stream)
            its = []
            for h in hs_m:
                info = A.solve(h, psib[1], xb)
                its.append(max(i.iterations for i in info))
                assert all(i.status == A.OK and i.true_relres <= TOL for i in info)
            eb[1].record(stream)
            torch.cuda.synchronize()
            ms = eb[0].elapsed_time(eb[1])
            batched["R16_mgs"] = {"solves_per_s": round(Rb * len(hs_m) / (ms * 1e-3), 3), "ms": round(ms, 2),
                                  "max_iterations": its}
            for h in hs_m:
                A.destroy(h)
        del psib, xb

    # the opt-in double-float Gram-Schmidt (mixed form): one right-hand side per
    # call over the three masses, then 16 per call, same inputs as above
    hs_df = [A.setup(U, m0, A.make_params(AGGS, precision=A.SOLVE_MIXED, restart=RESTART, tol=TOL, gs="df64"))
             for m0 in masses]
    run(hs_df, nst=args.warmup)
    st_df, sv_df, it_df, rr_df = run(hs_df, nst=nsteps, skip=args.warmup)
    gs_df64 = {"solves_per_s": round(len(sv_df) / (np.sum(st_df) * 1e-3), 3), "iterations": it_df[-len(masses):],
               "true_relres_max": max(rr_df)}
    psib = [torch.from_numpy(fx.gaussian_rhs(16, L, L, RHS_SEED0 + 50000 + 1600 + i)).to(dev) for i in range(2)]
    xb = torch.empty_like(psib[0])
    for h in hs_df:
        A.solve(h, psib[0], xb)
    flush.zero_()
    eb = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    eb[0].record(stream)
    for h in hs_df:
        info = A.solve(h, psib[1], xb)
        assert all(i.status == A.OK and i.true_relres <= TOL for i in info)
    eb[1].record(stream)
    torch.cuda.synchronize()
    gs_df64["R16_solves_per_s"] = round(16 * len(hs_df) / (eb[0].elapsed_time(eb[1]) * 1e-3), 3)
    for h in hs_df:
        A.destroy(h)
    del psib, xb

    # the coarse-smoother autotuner (amamg_params.autotune): the same solves with
    # the kernel and shape of the level-1 Gauss-Seidel timed and picked at the
    # first solve (warm-up), FP64 and mixed
    autotuned = {}
    for name, prec, vp in (("fp64", A.SOLVE_FP64, A.F64), ("mixed", A.SOLVE_MIXED, A.F32)):
        hs_at = [A.setup(U, m0, A.make_params(AGGS, precision=prec, restart=RESTART, tol=TOL, autotune=True))
                 for m0 in masses]
        fixed = A.query_smoother(hs_at[0], 1, vp, 1)
        run(hs_at, nst=1)
        st_at, _, it_at, _ = run(hs_at, nst=1 + args.steps, skip=1)
        autotuned[name] = {"solves_per_s": round(len(masses) * args.steps / (np.sum(st_at) * 1e-3), 3),
                           "iterations": it_at[-len(masses):], "level1_fixed_rule": fixed,
                           "level1_autotuned": [A.query_smoother(h, 1, vp, 1) for h in hs_at]}
        for h in hs_at:
            A.destroy(h)

    # the opt-in spin-split hierarchy (spin-diagonal interpolation weights; a
    # comparison beside the method as read): one warm-up and one timed step
    hs_ss = []
    for m0 in masses:
        hs_ss.append(A.setup(U, m0, A.make_params(AGGS, precision=A.SOLVE_FP64, restart=RESTART, tol=TOL,
                                                 spin_split=True)))
    run(hs_ss, nst=1)
    st_ss, _, it_ss, _ = run(hs_ss, nst=2, skip=1)
    spin_split = {"fp64_solves_per_s": round(len(masses) / (st_ss[0] * 1e-3), 3),
                  "iterations": it_ss[-len(masses):]}
    for h in hs_ss:
        A.destroy(h)

    # the paper's coarsest setting (GMRES(30) to 0.1 instead of the exact
    # solve), FP64 and mixed: one warm-up and one timed step each
    coarsest_gmres = {}
    for name, prec in (("fp64", A.SOLVE_FP64), ("mixed", A.SOLVE_MIXED)):
        hs_g = [A.setup(U, m0, A.make_params(AGGS, precision=prec, restart=RESTART, tol=TOL, coarsest="gmres"))
                for m0 in masses]
        run(hs_g, nst=1)
        st_g, sv_g, it_g, rr_g = run(hs_g, nst=2, skip=1)
        coarsest_gmres[name] = {"solves_per_s": round(len(masses) / (st_g[0] * 1e-3), 3),
                                "iterations": it_g[-len(masses):], "solve_ms": [round(v, 2) for v in sv_g],
                                "true_relres_max": max(rr_g[-len(masses):])}
        for h in hs_g:
            A.destroy(h)

    # the paper's unpreconditioned comparison solver: CG on the normal
    # equations (D^H = sigma_3 D sigma_3), FP64, same right-hand side per mass
    cgnr = {"iterations": [], "solve_ms": [], "true_relres": []}
    for h in hs64:
        A.cgnr(h, psis[0], x, max_iter=200000, tol=TOL)           # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        info = A.cgnr(h, psis[args.warmup], x, max_iter=200000, tol=TOL)
        ev[1].record(stream)
        torch.cuda.synchronize()
        cgnr["iterations"].append(info[0].iterations)
        cgnr["solve_ms"].append(round(ev[0].elapsed_time(ev[1]), 2))
        cgnr["true_relres"].append(info[0].true_relres)
    cgnr["amg_iterations"] = iters64[-len(masses):]
    amg_ms = [float(np.mean(solve_ms[k::len(masses)])) for k in range(len(masses))]   # per mass, timed steps
    cgnr["time_ratio_vs_amg_fp64"] = [round(c / a, 2) for c, a in zip(cgnr["solve_ms"], amg_ms)]

    # end to end through the public API with host buffers
    psi_h = [p.cpu().pin_memory() for p in psis]
    x_h = torch.empty(psis[0].shape, dtype=torch.complex128).pin_memory()
    psi_d = torch.empty_like(psis[0])
    e2e_ms = []
    for i in range(nsteps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h in hs64:
            psi_d.copy_(psi_h[i], non_blocking=True)
            A.solve(h, psi_d, x)
            x_h.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = args.steps * len(masses) * world / (np.sum(e2e_ms) * 1e-3)
    nbytes = psis[0].numel() * 16

    # per-kernel profile: a replay of the timed steps with event-bracketed launches
    peak, peak_kind = measured_peaks()

    def profile(hs):
        for h in hs:
            A.profile_reset(h)
            A.profile_enable(h, True)
        run(hs, nst=nsteps, skip=args.warmup)
        cats = {}
        for h in hs:
            A.profile_enable(h, False)
            for name, n, ms, by, fl in A.profile_get(h):
                c = cats.setdefault(name, [0, 0.0, 0.0, 0.0])
                c[0] += n
                c[1] += ms
                c[2] += by
                c[3] += fl
        tot = sum(c[1] for c in cats.values())
        share = {k: round(v[1] / tot, 4) for k, v in sorted(cats.items(), key=lambda kv: -kv[1][1])}
        # the analytic operation count of a solve (the per-kernel FLOP formulas
        # x launches, averaged over the replay's solves): the paper's GFLOP metric
        flop_count[len(flop_count)] = {"gflop_per_solve": round(sum(c[3] for c in cats.values()) / 1e9 /
                                                                (nsteps * len(hs)), 3),
                                       "solves": nsteps * len(hs)}
        dname, (dn, dms, dby, dfl) = max(cats.items(), key=lambda kv: kv[1][1])
        gbs = dby / (dms * 1e-3) / 1e9
        gflops = dfl / (dms * 1e-3) / 1e9
        fp64 = dname.endswith("f64") or dname.startswith("gs")
        roof = {"bound": "hbm", "kernel": dname, "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs / peak, 4), "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                "launches": dn, "avg_launch_us": round(1e3 * dms / dn, 3), "bytes_per_launch": round(dby / dn),
                "flops_per_launch": round(dfl / dn), "pass": "profiled replay of the timed steps"}
        if fp64 and gflops / FP64_PEAK_GFLOPS > gbs / peak:
            roof.update({"bound": "alu", "achieved": round(gflops, 1), "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": round(gflops / FP64_PEAK_GFLOPS, 4),
                         "peak_source": "nominal B300 FP64 rate (no measured FP64 figure)",
                         "hbm_GB/s": round(gbs, 1), "hbm_frac": round(gbs / peak, 4)})
        if dname == "coarse_smooth_f64" and COARSE_SMOOTH_F64_DRAM_BYTES is not None:
            roof["traffic"] = COARSE_SMOOTH_F64_DRAM_BYTES
            roof["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch (64x64 owner sweep)"
        return roof, share

    flop_count = {}
    roofline, kernel_share = profile(hs64)
    roofline_mixed, kernel_share_mixed = profile(hs32)
    flop_count = {"fp64": flop_count[0], "mixed": flop_count[1],
                  "note": "mean over the three masses' solves; per-kernel formulas in the library's profile"}

    # stencil bandwidth on working sets larger than L2 (1024^2, random-phase links)
    d_apply = {}
    Nd = 1024
    rng = np.random.Generator(np.random.PCG64(77))
    Ud = torch.from_numpy(np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nd, Nd)))).to(dev)
    hd = A.setup(Ud, 0.1, A.make_params([4, 4, 2]))
    for prec, R, dt in (("f64", 4, torch.complex128), ("f32", 8, torch.complex64)):
        xin = torch.randn(R, 2, Nd, Nd, dtype=dt, device=dev)
        yout = torch.empty_like(xin)
        for _ in range(3):
            A.apply_D(hd, xin, yout)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = 20
        ev[0].record(stream)
        for _ in range(reps):
            A.apply_D(hd, xin, yout)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / reps
        cb = 16 if prec == "f64" else 8
        by = Nd * Nd * (R * 2 * 2 * cb + 2 * cb)
        gbs = by / (ms * 1e-3) / 1e9
        d_apply[prec] = {"lattice": f"{Nd}x{Nd}", "rhs": R, "ms": round(ms, 4), "GB/s": round(gbs, 1),
                         "frac_of_hbm": round(gbs / peak, 3), "bytes_per_launch": by}
        if prec == "f64":
            # 56 FLOPs per site and right-hand side (the stencil's complex
            # multiply-adds): on B300 the FP64 form is bound by the FP64 pipe
            gfl = Nd * Nd * R * 56.0 / (ms * 1e-3) / 1e9
            d_apply[prec].update({"bound": "alu (FP64 pipe)", "GFLOP/s": round(gfl, 1),
                                  "frac_of_fp64_peak": round(gfl / FP64_PEAK_GFLOPS, 3),
                                  "fp64_peak": f"{FP64_PEAK_GFLOPS:g} GFLOP/s nominal"})
        else:
            d_apply[prec]["bound"] = "hbm"
        del xin, yout
    del hd

    spread_out = None if args.no_spread else run_spread(dev, U, masses, psis[0])

    c4_out = run_c4(dev, c4_theta) if not args.no_c4 else None

    serving_out = None
    if args.serving > 0:
        free, total = torch.cuda.mem_get_info()
        serving_out = run_serving(args.serving, args.serving_rate, dev, int(0.7 * free), serving_thetas)

    out = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            from oracle import wilson as W
            D0, lv0, setup_s = oracle_hierarchy(theta, masses[0])
            ot, ores = oracle_solve(D0, lv0, W.to_flat(psis[args.warmup].cpu().numpy()[0]))
            cpu = {"value": 1.0 / ot, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"1 oracle solve (m_crit+0.1 mass, {ores.iterations} iterations, FP64 NumPy/SciPy, "
                             f"sparse kernels single-threaded); oracle setup {setup_s:.1f} s excluded"}
            # error of the GPU solutions of that right-hand side against the oracle's
            xo = ores.x
            for key, xg in (("fp64", x_check64), ("mixed", x_check32)):
                xf = W.to_flat(xg)
                errs_vs_oracle[key] = float(np.linalg.norm(xf - xo) / np.linalg.norm(xo))
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(world),
            "e2e": {"value": round(e2e_value, 3), "unit": "solves/s", "h2d_bytes_per_step": nbytes * len(masses),
                    "d2h_bytes_per_step": nbytes * len(masses)},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "kernel_share": kernel_share,
            "roofline_mixed": roofline_mixed,
            "kernel_share_mixed": kernel_share_mixed,
            "flop_count": flop_count,
            "cpu_baseline": cpu,
            "clocks": clk,
            "error_vs_oracle": ({"x": "||x_gpu - x_oracle|| / ||x_oracle||, m_crit+0.1 mass, first timed RHS",
                                 **errs_vs_oracle} if errs_vs_oracle else None),
            "mixed": {"value": round(mixed_value, 3), "unit": "solves/s", "speedup_vs_fp64": round(mixed_value / value, 3),
                      "error_vs_oracle": errs_vs_oracle.get("mixed"),
                      "iterations": it32[-len(masses):], "true_relres_max": max(rr32),
                      "latency_ms": {"p50": round(float(np.percentile(sv32, 50)), 3),
                                     "p99": round(float(np.percentile(sv32, 99)), 3)},
                      "setup_ms": [round(s, 2) for s in setup32]},
            "mixed_gs_df64": gs_df64,
            "autotuned": autotuned,
            "latency_ms": {"p50": round(float(np.percentile(solve_ms, 50)), 3),
                           "p99": round(float(np.percentile(solve_ms, 99)), 3)},
            "batched_mixed": batched,
            "spin_split": spin_split,
            "coarsest_gmres": coarsest_gmres,
            "cgnr": cgnr,
            "iterations": iters64[-len(masses):],
            "true_relres_max": max(relres64),
            "setup_ms": [round(s, 2) for s in setup64],
            "d_apply": d_apply,
            "wall_s_timed_region": round(wall_s, 3),
        }
        if c4_out is not None:
            out["c4"] = c4_out
        if serving_out is not None:
            out["serving"] = serving_out
        if spread_out is not None:
            out["spread"] = spread_out
        print(json.dumps(out))
    pool.shutdown(wait=False, cancel_futures=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
