#!/usr/bin/env python3
"""Benchmark: seconds per HMC trajectory of the Schwarz-preconditioned
two-flavour Wilson HMC (one-dimensional x0-slab decomposition) on a
16^3 x 32 lattice, mixed-precision batched form, beside the plain
double-precision GPU form, the Dslash bandwidth against the HBM roofline
and the FP64 CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  A step is one full trajectory (heatbath,
molecular dynamics with the W1 and boundary (Schur) pseudo-fermion forces
and the gauge force on three time scales, Metropolis, x0 shift) on seeded
synthetic links; inputs are resident in HBM and L2 is flushed between
timed trajectories.  With N > 1 every rank runs an independent replica on
its own GPU (the path is not sharded here), the time is the maximum over
ranks and value = that time / all trajectories of the job.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# ---------------------------------------------------------------------------
# the workload (16^3 x 32, kappa = 0.1575, beta = 5.6, l0 = 4: 8 slabs)
# ---------------------------------------------------------------------------
WL = dict(L=(32, 16, 16, 16), l0=4, kappa=0.1575, beta=5.6, eps=0.6, seed=2009, tau=1.0,
          nlevels=3, scheme=(1, 1, 1), nsteps=(2, 4, 8), lam=0.1931833275037836,
          level_gauge=0, level_w1=1, level_schur=2, tol=1e-10, max_iter=20000, therm=40)
WORKLOAD_NAME = ("Schwarz-HMC trajectory 16^3x32, l0=4 (8 x0-slabs, red/black), kappa=0.1575, "
                 "beta=5.6, tau=1, Omelyan (lambda=0.1932) on 3 time scales: gauge / W1 / boundary "
                 "Schur force, n=(2,4,8); links exp(i 0.6 H) thermalised by 40 pure-gauge HMC "
                 "trajectories at beta=5.6")
DSLASH_L = (64, 32, 32, 32)
# the one metric both arms print (the precision is in dtype / config)
METRIC = "s/HMC trajectory (16^3x32 Schwarz HMC)"


def thermalise(lat, U, beta, ntraj, seed):
    """seeded pure-gauge HMC at beta from a rough random start (the paper's
    inputs are thermalised beta = 5.6 fields): 20 trajectories without the
    accept/reject step, the rest with it"""
    from paper_0710_0066_gb300 import lqcd

    prm = lqcd.hmc_params(beta, 0.0, 1.0, 1, (lqcd.SW,), (10,), 0, -1, -1, lam=0.1931833275037836,
                          roll=0, metropolis=0, precision=lqcd.PREC_F64, tol=1e-10)
    res = None
    for t in range(ntraj):
        prm.metropolis = 1 if t >= min(20, ntraj // 2) else 0
        U, res = lat.hmc_trajectory(U, prm, seed, 1000000 + t)
    return U, res


def thermalise_dynamical(lat, U, prm, ntraj, seed):
    """input preparation, continued: full trajectories with the fermion
    action (the timed schedule at a looser solver tolerance) from the
    pure-gauge start, so that the plaquette and the solver work are
    stationary over the timed trajectories; returns the field and the
    plaquettes seen"""
    tol, graph = prm.tol, prm.use_graph
    prm.tol, prm.use_graph = 1e-8, 0
    plaq = []
    try:
        for t in range(ntraj):
            U, res = lat.hmc_trajectory(U, prm, seed, 2000000 + t)
            plaq.append(res.plaq)
    finally:
        prm.tol, prm.use_graph = tol, graph
    return U, plaq


PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")

# DRAM bytes per k_solve launch from the ncu capture summarised in
# profiles/k_solve_16x16x16x32_f32.md, valid only for the solver source
# that was captured (bench.py reports null once the source differs)
SOLVER_SOURCES = ("lqcd_solver.cu", "lqcd_common.cuh", "lqcd_df.cuh")  # the sources k_solve is built from
SOLVER_TRAFFIC = dict(src_sha256="aef4788cc714dda78760d271604c272fd83e3842839fc76a07edbe1288dfd3b3",
                      block_series=(303.767e6 + 154.127e6), block=(307.420e6 + 312.868e6),
                      glob=(392.167e6 + 425.938e6))


def solver_traffic():
    import hashlib

    h = hashlib.sha256()
    try:
        for name in SOLVER_SOURCES:
            with open(os.path.join(ROOT, "paper_0710_0066_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
    except OSError:
        return None, None
    sha = h.hexdigest()
    if sha != SOLVER_TRAFFIC["src_sha256"]:
        return None, None
    return SOLVER_TRAFFIC["block_series"], {"batched_slab_solve_series": SOLVER_TRAFFIC["block_series"],
                                            "batched_slab_solve_bicgstab": SOLVER_TRAFFIC["block"],
                                            "global_solve_bicgstab": SOLVER_TRAFFIC["glob"],
                                            "source": "profiles/k_solve_16x16x16x32_f32.md"}


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle timing (host cores)
# ---------------------------------------------------------------------------
def oracle_problem(L, l0, eps, seed):
    """the oracle lattice, links and a source of the workload (built once)"""
    from oracle import oracle as O
    from paper_0710_0066_gb300 import synthetic as syn

    lat = O.Lattice(L, l0, -1)
    U = syn.random_links(L, eps, seed)
    x = syn.gaussian_spinor(lat.V, seed + 1)
    return lat, U, x


def oracle_M_seconds(budget_s, L, l0, eps, seed, problem=None):
    """seconds per application of the oracle's full-lattice Wilson matrix"""
    import numpy as np

    lat, U, x = problem if problem is not None else oracle_problem(L, l0, eps, seed)
    lat.M(U, 0.1575, x)
    n, t0 = 0, time.perf_counter()
    while True:
        x = lat.M(U, 0.1575, x)
        x /= np.linalg.norm(x)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return (time.perf_counter() - t0) / n, n


def oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


# Wilson-matrix applications in one trajectory of this workload, the count
# both oracle figures (the reference arm and cpu_baseline) scale the
# oracle's measured time per application by: the library counts the
# half-lattice hopping site updates of every inner iteration (hop_sites; a
# full application is V of them), and this is that count for the 16^3x32
# trajectory with every solve started from zero (the method's own work:
# geometric series for W1, BiCGstab elsewhere).  The oracle's own solver,
# CG on the normal equations, needs several times more applications (about
# 500 for one slab solve of a thermalised 16x4^3 field to 1e-10), so the
# figure is a lower bound on the oracle's time.
M_APPS_PER_TRAJ = 25187.0


def job_time(rank_ms, steps, dist=None, device="cpu"):
    """whole-job timing of N replicas: the slowest rank's time of its timed
    steps (max over ranks) and the job's seconds per trajectory, that time
    divided by every trajectory of the job (weak scaling: each rank runs
    `steps` trajectories of its own replica)"""
    import torch

    world = dist.get_world_size() if dist is not None else 1
    total_ms = float(rank_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, total_ms / 1e3 / (steps * world)


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    L, l0 = WL["L"], WL["l0"]
    times, wall, napp = [], [], 0
    problem = oracle_problem(L, l0, WL["eps"], WL["seed"])
    for k in range(args.warmup + args.steps):
        w0 = time.perf_counter()
        t_M, n = oracle_M_seconds(args.ref_sample_seconds, L, l0, WL["eps"], WL["seed"], problem)
        if k >= args.warmup:
            times.append(t_M * M_APPS_PER_TRAJ)
            wall.append(time.perf_counter() - w0)
            napp += n
    v = statistics.mean(times)
    sample = ("per step %.1f s of wall time: applications of the oracle's FP64 Wilson matrix at 16^3x32 "
              "(%.1f ms each), the seconds per application scaled by %d applications per trajectory (the "
              "method's count with every solve from zero; the oracle's CGNR needs more, so this is a lower "
              "bound)" % (statistics.mean(wall), 1e3 * statistics.mean(times) / M_APPS_PER_TRAJ,
                          M_APPS_PER_TRAJ))
    line = {
        "impl": "reference", "metric": METRIC, "value": v,
        "unit": "s/trajectory", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(wall), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD_NAME},
        "extrapolated": {"model": "oracle seconds per Wilson-matrix application x %d applications per trajectory"
                                  % M_APPS_PER_TRAJ,
                         "measured_wall_s_per_step": statistics.mean(wall),
                         "applications_timed": napp},
        "cpu_baseline": {"value": v, "unit": "s/trajectory", "cores": oracle_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "s/trajectory", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_0710_0066_gb300 import lqcd, synthetic as syn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    L, l0 = WL["L"], WL["l0"]
    lat = lqcd.Lattice(L, l0, -1)
    U0 = syn.random_links_torch(L, WL["eps"], WL["seed"] + rank, "cuda").contiguous()
    U0, rth = thermalise(lat, U0, WL["beta"], WL["therm"], WL["seed"] + rank)
    # launch schedules measured on this lattice and field (outside the timed region)
    lat.set_gauge(U0)
    lqcd.lqcd_autotune(lat.h, 3, WL["kappa"])
    tune = lqcd.lqcd_tune_read(lat.h)
    if args.global_solver != "bicgstab":
        lqcd.lqcd_set_global_solver(lat.h, lqcd.SOLVER_SAP if args.global_solver == "sap"
                                    else lqcd.SOLVER_SAP_BLOCKS, args.sap_terms)

    def params(prec):
        return lqcd.hmc_params(WL["beta"], WL["kappa"], WL["tau"], WL["nlevels"], WL["scheme"], WL["nsteps"],
                               WL["level_gauge"], WL["level_w1"], WL["level_schur"], lam=WL["lam"], roll=1,
                               metropolis=1, precision=prec, tol=WL["tol"], max_iter=WL["max_iter"],
                               use_graph=0 if args.no_graph else 1, chrono=0 if args.no_chrono else args.chrono,
                               block_solver=lqcd.SOLVER_SERIES if args.block_solver == "series"
                               else lqcd.SOLVER_BICGSTAB)

    prec = {"f16": lqcd.PREC_F16, "bf16": lqcd.PREC_BF16, "f32": lqcd.PREC_F32, "f64": lqcd.PREC_F64}[args.precision]
    prm = params(prec)
    block_solver = args.block_solver

    def run_or_fall_back(fn):
        # the geometric series needs its spectral radius below one; if a slab
        # of this field does not satisfy that, the W1 solves fall back to
        # BiCGstab for the whole measurement (reported)
        nonlocal prm, block_solver
        try:
            return fn()
        except lqcd.LqcdError as e:
            if e.status != lqcd.ERR_NOCONVERGE or args.block_solver != "series":
                raise
            block_solver = "bicgstab (the series did not converge on this field)"
            args.block_solver = "bicgstab"
            prm = params(prec)
            return fn()

    U0, plaq_dyn = run_or_fall_back(lambda: thermalise_dynamical(lat, U0, prm, args.therm_fermion,
                                                                 WL["seed"] + rank))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    U = U0.clone()
    traj = 0
    for _ in range(args.warmup):
        U, res = run_or_fall_back(lambda: lat.hmc_trajectory(U, prm, WL["seed"], traj))
        traj += 1
    torch.cuda.synchronize()

    # ---- timed region: K trajectories, L2 flushed between them
    lqcd.lqcd_profile_reset(lat.h)
    lqcd.lqcd_profile_enable(lat.h, 1 << lqcd.KERNEL_SOLVER)
    l0_launch = lqcd.lqcd_launch_count(lat.h)
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    step_ms, results, U_in = [], [], []
    for k in range(args.steps):
        flush.zero_()
        barrier()
        U_in.append((U.clone(), traj))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        U, res = lat.hmc_trajectory(U, prm, WL["seed"], traj)
        b.record(stream)
        barrier()
        step_ms.append(a.elapsed_time(b))
        results.append(res)
        traj += 1
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = lqcd.lqcd_launch_count(lat.h) - l0_launch
    n_sol, ms_sol, by_sol = lqcd.lqcd_profile_read(lat.h, lqcd.KERNEL_SOLVER)
    sol_ms = lqcd.lqcd_profile_times(lat.h, lqcd.KERNEL_SOLVER)[:max(1, n_sol // max(1, args.steps))]
    lqcd.lqcd_profile_enable(lat.h, 0)
    total_ms, value = job_time(sum(step_ms), args.steps, dist, "cuda")

    # ---- plain double-precision GPU form on the inputs of the first timed
    # trajectories (one untimed trajectory first records its MD graph)
    fp64 = None
    if not args.no_fp64 and prec != lqcd.PREC_F64:
        prm64 = params(lqcd.PREC_F64)
        lat.hmc_trajectory(U_in[0][0], prm64, WL["seed"], U_in[0][1])
        t64, d64 = [], []
        nf = min(args.fp64_steps, len(U_in))
        for k in range(nf):
            Uk, tk = U_in[k]
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, r64 = lat.hmc_trajectory(Uk, prm64, WL["seed"], tk)
            b.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(b) / 1e3)
            d64.append(abs(r64.dH - results[k].dH))
        mixed = statistics.mean(step_ms[:nf]) / 1e3
        fp64 = {"s_per_traj": statistics.mean(t64), "trajectories": nf,
                "mixed_s_per_traj_same_inputs": mixed, "speedup_mixed_vs_fp64": statistics.mean(t64) / mixed,
                "max_abs_dH_diff": max(d64)}

    # ---- end to end through the C-ABI with host buffers
    Uh = torch.empty_like(U, device="cpu").pin_memory()
    Uh.copy_(U)
    Ud = torch.empty_like(U)
    e2e_ms = []
    for k in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ud.copy_(Uh, non_blocking=True)
        res = lqcd.lqcd_hmc_trajectory(lat.h, Ud, prm, WL["seed"], traj)
        Uh.copy_(Ud, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        traj += 1
    e2e_value = statistics.mean(e2e_ms[1:]) / 1e3
    ubytes = U.numel() * 16

    # ---- Dslash (even-odd hopping sweep) bandwidth at 32^3 x 64 (> L2)
    peak, peak_kind = hbm_peak()
    dslash = {}
    if not args.no_dslash:
        latd = lqcd.Lattice(DSLASH_L, 8, -1)
        Ud_ = syn.random_links_torch(DSLASH_L, WL["eps"], WL["seed"] + 7, "cuda").contiguous()
        latd.set_gauge(Ud_)
        del Ud_
        lqcd.lqcd_autotune(latd.h, 1, 0.0)
        x = torch.randn((latd.Vh, 4, 3), dtype=torch.complex128, device="cuda")
        for name, pr in (("f32", lqcd.PREC_F32), ("f16", lqcd.PREC_F16), ("bf16", lqcd.PREC_BF16),
                         ("f64", lqcd.PREC_F64)):
            # the k_hop launch alone, timed by the library's CUDA events
            # around each of 100 launches queued back to back (the layout
            # conversions of each call run between them); one launch moves
            # 0.3 GB (f16) to 1.6 GB (f64), far more than the 129 MB L2, so
            # every launch streams from HBM; median reported
            for _ in range(5):
                latd.dslash_eo(x, 0, 0.0, 0, lqcd.OP_HOP, pr)
            lqcd.lqcd_profile_reset(latd.h)
            lqcd.lqcd_profile_enable(latd.h, 1 << lqcd.KERNEL_HOP)
            for _ in range(100):
                latd.dslash_eo(x, 0, 0.0, 0, lqcd.OP_HOP, pr)
            n, ms, by = lqcd.lqcd_profile_read(latd.h, lqcd.KERNEL_HOP)
            per = lqcd.lqcd_profile_times(latd.h, lqcd.KERNEL_HOP)
            lqcd.lqcd_profile_enable(latd.h, 0)
            med = statistics.median(per)
            dslash[name] = {"gbs": round(by / n / med / 1e6, 1), "frac": round(by / n / med / 1e6 / peak, 4),
                            "ms_median": round(med, 4), "bytes_per_launch": by / n}
        latd.close()

    # ---- force-profile diagnostic (Sec. 3, Fig. 1) on the thermalised field
    # (--force-profile): mean |F| on space-like links per time slice
    profile = None
    if args.force_profile:
        profile = {}
        lat.set_gauge(U)
        g = torch.Generator(device="cuda")
        g.manual_seed(WL["seed"] + 11)
        eta1 = torch.randn((lat.V, 4, 3), dtype=torch.complex128, device="cuda", generator=g) * math.sqrt(0.5)
        phi1 = lat.block_dslash(eta1, WL["kappa"])
        eta2 = torch.randn(lat.boundary().shape, dtype=torch.complex128, device="cuda", generator=g) * math.sqrt(0.5)
        phi2 = lat.schur(eta2.contiguous(), WL["kappa"], lqcd.SCHUR_R, lqcd.PREC_F32, tol=WL["tol"])
        _, Fw = lat.pf_force(phi1, WL["kappa"], lqcd.TERM_W1, lqcd.PREC_F32, tol=WL["tol"])
        _, Fs = lat.pf_force(phi2, WL["kappa"], lqcd.TERM_SCHUR, lqcd.PREC_F32, tol=WL["tol"])
        _, _, Fg = lat.gauge_force(WL["beta"])
        for name, F in (("gauge", Fg), ("w1", Fw), ("schur", Fs)):
            profile[name] = [round(v, 5) for v in lat.force_profile(F)[0].tolist()]

    # ---- oracle on the host cores (bounded sample), scaled by the same
    # application count as the reference arm
    m_apps = statistics.mean(r.hop_sites for r in results) / lat.V
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        t_M, n = oracle_M_seconds(args.cpu_seconds, L, l0, WL["eps"], WL["seed"])
        cpu = {"value": t_M * M_APPS_PER_TRAJ, "unit": "s/trajectory", "cores": oracle_threads(), "kind": "oracle",
               "sample": "%d applications of the oracle's FP64 Wilson matrix at 16^3x32 (%.1f ms each) x %d "
                         "applications per trajectory (solves from zero; a lower bound for the oracle's CGNR)"
                         % (n, 1e3 * t_M, M_APPS_PER_TRAJ)}

    achieved = by_sol / ms_sol / 1e6 if ms_sol > 0 else None
    traffic, traffic_detail = solver_traffic() if prec == lqcd.PREC_F32 else (None, None)
    sm = step_ms
    half = max(1, len(sm) // 2)
    line = {
        "metric": METRIC,
        "value": value, "unit": "s/trajectory", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "f64" else ("f32+f64" if args.precision == "f32"
                                                                  else args.precision + "-storage+f32+f64"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "lattice": "x".join(map(str, L)), "l0": l0,
                   "inner_precision": args.precision, "l2": "flushed between timed trajectories",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "md_as_cuda_graph": not args.no_graph, "w1_block_solver": block_solver,
                   "chronological_guesses": 0 if args.no_chrono else args.chrono,
                   "global_solver": ("Schwarz-preconditioned BiCGstab, %d series terms per slab solve"
                                     % args.sap_terms) if args.global_solver == "sap"
                                    else ("Schwarz-preconditioned BiCGstab over 4^4 blocks in shared memory, "
                                          "%d series terms per block solve" % args.sap_terms)
                                    if args.global_solver == "sap-blocks" else "even-odd BiCGstab",
                   "dynamical_thermalisation": args.therm_fermion},
        "roofline": {"bound": "hbm", "kernel": "persistent batched solver (k_solve)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_kind": peak_kind, "launches": n_sol,
                     "kernel_share_of_step": ms_sol / total_ms if total_ms else None,
                     "dslash_64x32x32x32": dslash},
        "fp64_form": fp64,
        "trajectory": {"step_ms_first_half_mean": statistics.mean(sm[:half]),
                       "step_ms_second_half_mean": statistics.mean(sm[half:]) if len(sm) > 1 else sm[0],
                       "step_ms_min": min(sm), "step_ms_max": max(sm),
                       "solver_iters_first": results[0].solver_iters, "solver_iters_last": results[-1].solver_iters,
                       "plaq_first": results[0].plaq, "plaq_last": results[-1].plaq,
                       "acceptance": sum(r.accepted for r in results) / len(results),
                       "dH_rms": math.sqrt(statistics.mean(r.dH ** 2 for r in results)),
                       "n_solves": results[-1].n_solves, "n_force": results[-1].n_force},
        "m_apps_per_traj": m_apps,
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "s/trajectory", "h2d_bytes_per_step": ubytes,
                "d2h_bytes_per_step": ubytes},
    }
    if profile is not None:
        line["force_profile_spatial"] = profile
    if args.detail and rank == 0:
        with open(args.detail, "w") as f:
            json.dump({"step_ms": step_ms, "solver_iters": [r.solver_iters for r in results],
                       "plaq": [r.plaq for r in results], "dH": [r.dH for r in results],
                       "accepted": [r.accepted for r in results], "plaq_dynamical_thermalisation": plaq_dyn,
                       "pure_gauge_plaq": rth.plaq if rth else None, "autotune": tune,
                       "solver_traffic": traffic_detail, "fp64": fp64, "e2e_ms": e2e_ms,
                       "solver_launch_ms_one_trajectory": sol_ms}, f)
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()


# the iterated decomposition at 32^3 x 64: slabs l0 = 8 split into sub-slabs
# of thickness 4, action S_G + |R^-1 phi2|^2 + |R2^-1 phi4|^2 + |W2^-1 phi3|^2
# on four time scales (gauge / W2 / R2 / R), Omelyan on every level
WL_ITER = dict(L=(64, 32, 32, 32), l0=8, l0s=4, kappa=0.158, beta=5.6, eps=0.6, seed=2010, tau=1.0,
               nlevels=4, scheme=(1, 1, 1, 1), nsteps=(2, 2, 2, 6), lam=0.1931833275037836,
               level_gauge=0, level_w2=1, level_schur2=2, level_schur=3, tol=1e-10, max_iter=20000, therm=40,
               name="iterated", metric="s/HMC trajectory (32^3x64, iterated slab decomposition)",
               levels="gauge/W2/R2/R")
# the paper's production form at 32 x 16^3 (Sec. 1-3, Table 1 row L0 = 32,
# L = 16, kappa = 0.1575): l0 = L0/2, l0s = L0/4, the four-part action
# S4 (R) + S3 (R2) + S2 + S1 with W3,eo = W2,eo + rho, rho = 0.20, five levels
# n = (n0..n4) = (4, 2, 3, 1, 4), SW on levels 0, 1 and LF on 2, 3, 4,
# lambda = 1/6, step-size scheme B
WL_PROD = dict(L=(32, 16, 16, 16), l0=16, l0s=8, kappa=0.1575, beta=5.6, eps=0.6, seed=2011, tau=1.0,
               nlevels=5, scheme=(1, 1, 0, 0, 0), nsteps=(4, 2, 3, 1, 4), lam=1.0 / 6.0,
               level_gauge=0, level_w2=-1, level_schur2=3, level_schur=4, rho=0.20, level_s2=2, level_s1=1,
               step_scheme=2, tol=1e-10, max_iter=20000, therm=40, name="production",
               metric="s/HMC trajectory (32x16^3, four-part action, Table 1 schedule)",
               levels="gauge/S1/S2/S3(R2)/S4(R)")


# Table 1's last row (Sec. 3): 32 x 24^3, kappa = 0.15825, scheme C,
# rho = 0.15, (n4, n3, n2, n1, n0) = (5, 3, 2, 2, 4): the configuration of
# the paper's timing remark (about 2.5 h per trajectory on 8 CPUs), here on
# a seeded quenched-thermalised field instead of the paper's ensemble
WL_TABLE1 = dict(L=(32, 24, 24, 24), l0=16, l0s=8, kappa=0.15825, beta=5.6, eps=0.6, seed=2012, tau=1.0,
                 nlevels=5, scheme=(1, 1, 0, 0, 0), nsteps=(4, 2, 2, 3, 5), lam=1.0 / 6.0,
                 level_gauge=0, level_w2=-1, level_schur2=3, level_schur=4, rho=0.15, level_s2=2, level_s1=1,
                 step_scheme=3, tol=1e-10, max_iter=40000, therm=40, name="table1",
                 metric="s/HMC trajectory (32x24^3, kappa=0.15825, Table 1 schedule)",
                 levels="gauge/S1/S2/S3(R2)/S4(R)",
                 paper_context="about 2.5 h per trajectory on 8 CPUs (AMD Opteron 2.2 GHz, Cray XD1), "
                               "the paper's thermalised ensemble (Sec. 3)")


def run_iterated(args, W=WL_ITER):
    """--case iterated / production: K trajectories of a four-part action in
    the mixed-precision form, the first input again in the plain double
    form; one JSON line"""
    import torch

    from paper_0710_0066_gb300 import lqcd, synthetic as syn

    torch.cuda.set_device(0)
    L = W["L"]
    lat = lqcd.Lattice(L, W["l0"], -1, l0s=W["l0s"])
    U0 = syn.random_links_torch(L, W["eps"], W["seed"], "cuda").contiguous()
    U0, rth = thermalise(lat, U0, W["beta"], W["therm"], W["seed"])
    lat.set_gauge(U0)
    lqcd.lqcd_autotune(lat.h, 3, W["kappa"])
    tune = lqcd.lqcd_tune_read(lat.h)

    def params(prec):
        return lqcd.hmc_params(W["beta"], W["kappa"], W["tau"], W["nlevels"], W["scheme"], W["nsteps"],
                               W["level_gauge"], -1, W["level_schur"], lam=W["lam"], roll=1, metropolis=1,
                               precision=prec, tol=W["tol"], max_iter=W["max_iter"], level_w2=W["level_w2"],
                               level_schur2=W["level_schur2"], rho=W.get("rho", 0.0),
                               level_s2=W.get("level_s2", -1), level_s1=W.get("level_s1", -1),
                               step_scheme=W.get("step_scheme", 0),
                               eo_solver=lqcd.SOLVER_SERIES if args.eo_solver == "series" else lqcd.SOLVER_BICGSTAB,
                               use_graph=0 if args.no_graph else 1, chrono=0 if args.no_chrono else 1)

    prec = {"f16": lqcd.PREC_F16, "bf16": lqcd.PREC_BF16, "f32": lqcd.PREC_F32, "f64": lqcd.PREC_F64}[args.precision]
    prm = params(prec)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    U = U0.clone()
    traj = 0
    for _ in range(args.warmup):
        U, res = lat.hmc_trajectory(U, prm, W["seed"], traj)
        traj += 1
    lqcd.lqcd_profile_reset(lat.h)
    lqcd.lqcd_profile_enable(lat.h, 1 << lqcd.KERNEL_SOLVER)
    clocks = Clocks(0)
    clocks.start()
    step_ms, results, U_in = [], [], []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        U_in.append((U.clone(), traj))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        U, res = lat.hmc_trajectory(U, prm, W["seed"], traj)
        b.record(stream)
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
        results.append(res)
        traj += 1
    clk = clocks.stop()
    n_sol, ms_sol, by_sol = lqcd.lqcd_profile_read(lat.h, lqcd.KERNEL_SOLVER)
    lqcd.lqcd_profile_enable(lat.h, 0)
    fp64 = None
    if not args.no_fp64 and prec != lqcd.PREC_F64:
        Uk, tk = U_in[0]
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, r64 = lat.hmc_trajectory(Uk, params(lqcd.PREC_F64), W["seed"], tk)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        fp64 = {"s_per_traj": t64, "dH": r64.dH, "dH_mixed": results[0].dH,
                "abs_dH_diff": abs(r64.dH - results[0].dH), "speedup_mixed_vs_fp64": t64 / (step_ms[0] / 1e3),
                "accepted": r64.accepted}
    # force profile of every term (Sec. 3, Fig. 1 analogue) on the field of
    # the last trajectory, pseudo-fermions drawn as the heatbath draws them
    profile = {}
    if W.get("level_s1", -1) >= 0 and not args.no_dslash:
        lat.set_gauge(U)
        g = torch.Generator(device="cuda")
        g.manual_seed(W["seed"] + 11)

        def gauss(shape):
            return (torch.randn(shape, dtype=torch.complex128, device="cuda", generator=g)
                    * math.sqrt(0.5)).contiguous()

        k, rho = W["kappa"], W["rho"]
        tol = W["tol"]
        phi4 = lat.schur(gauss(lat.boundary().shape), k, lqcd.SCHUR_R, lqcd.PREC_F32, tol=tol)
        phi3 = lat.schur(gauss(lat.boundary2().shape), k, lqcd.SCHUR2_R, lqcd.PREC_F32, tol=tol)
        e2, _ = lat.solve_w3eo(gauss((lat.Vh, 4, 3)), k, rho, 0, lqcd.PREC_F32, tol=tol)
        phi2 = lat.w3eo(e2, k, 0.0)
        phi1 = lat.w3eo(gauss((lat.Vh, 4, 3)), k, rho)
        terms = {"S4": lat.pf_force(phi4, k, lqcd.TERM_SCHUR, lqcd.PREC_F32, tol)[1],
                 "S3": lat.pf_force(phi3, k, lqcd.TERM_SCHUR2, lqcd.PREC_F32, tol)[1],
                 "S2": lat.pf_force_eo(phi2, k, rho, lqcd.TERM_S2, lqcd.PREC_F32, tol)[1],
                 "S1": lat.pf_force_eo(phi1, k, rho, lqcd.TERM_S1, lqcd.PREC_F32, tol)[1],
                 "S0": lat.gauge_force(W["beta"])[2]}
        for name, F in terms.items():
            profile[name] = [round(v, 5) for v in lat.force_profile(F)[0].tolist()]
    peak, peak_kind = hbm_peak()
    achieved = by_sol / ms_sol / 1e6 if ms_sol > 0 else None
    line = {
        "case": W["name"], "metric": W["metric"],
        "value": sum(step_ms) / 1e3 / args.steps, "unit": "s/trajectory", "steps": args.steps,
        "warmup": args.warmup, "precision": args.precision,
        "config": {"lattice": "x".join(map(str, L)), "l0": W["l0"], "l0s": W["l0s"], "kappa": W["kappa"],
                   "beta": W["beta"], "nsteps": W["nsteps"], "levels": W["levels"], "rho": W.get("rho"),
                   "step_scheme": W.get("step_scheme", 0), "scheme": W["scheme"], "eo_solver": args.eo_solver,
                   "chronological_guesses": 0 if args.no_chrono else args.chrono,
                   "thermalisation": "%d pure-gauge trajectories from exp(i %.1f H)" % (W["therm"], W["eps"]),
                   "autotune": tune,
                   "l2": "flushed between timed trajectories"},
        "solver": {"achieved_gbs": achieved, "peak": peak, "peak_kind": peak_kind,
                   "frac": (achieved / peak) if achieved else None, "launches": n_sol,
                   "share_of_step": ms_sol / sum(step_ms)},
        "trajectory": {"dH": [r.dH for r in results], "accepted": [r.accepted for r in results],
                       "plaq": results[-1].plaq, "solver_iters": [r.solver_iters for r in results],
                       "n_solves": results[-1].n_solves, "n_force": results[-1].n_force, "step_ms": step_ms},
        "acceptance": sum(r.accepted for r in results) / len(results),
        "fp64_form": fp64, "thermalisation_plaq": rth.plaq if rth else None, "clocks": clk,
        "paper_context": W.get("paper_context"),
        "force_profile_spatial": profile,
    }
    print(json.dumps(line), flush=True)
    lat.close()


def run_case(args):
    """small single-kernel cases for profiler captures (a few GB on the device)"""
    import torch

    from paper_0710_0066_gb300 import lqcd, synthetic as syn

    torch.cuda.set_device(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(WL["seed"])
    prec = {"f16": lqcd.PREC_F16, "bf16": lqcd.PREC_BF16, "f32": lqcd.PREC_F32, "f64": lqcd.PREC_F64}[args.precision]
    if args.case == "iterated":
        return run_iterated(args, WL_ITER)
    if args.case == "production":
        return run_iterated(args, WL_PROD)
    if args.case == "table1":
        return run_iterated(args, WL_TABLE1)
    if args.case == "solver":
        # the batched slab solve (8 slabs) and the global solve of the
        # workload, on the field the timed trajectories start from (pure-
        # gauge, then dynamical thermalisation)
        L, l0 = WL["L"], WL["l0"]
        lat = lqcd.Lattice(L, l0, -1)
        U = syn.random_links_torch(L, WL["eps"], WL["seed"], "cuda").contiguous()
        U, _ = thermalise(lat, U, WL["beta"], WL["therm"], WL["seed"])
        if args.therm_fermion:
            prm = lqcd.hmc_params(WL["beta"], WL["kappa"], WL["tau"], WL["nlevels"], WL["scheme"], WL["nsteps"],
                                  WL["level_gauge"], WL["level_w1"], WL["level_schur"], lam=WL["lam"], roll=1,
                                  metropolis=1, precision=lqcd.PREC_F32, tol=WL["tol"], max_iter=WL["max_iter"],
                                  chrono=1, block_solver=lqcd.SOLVER_SERIES)
            U, _ = thermalise_dynamical(lat, U, prm, args.therm_fermion, WL["seed"])
        lat.set_gauge(U)
        b = torch.randn((lat.V, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
        lqcd.lqcd_profile_enable(lat.h, 1 << lqcd.KERNEL_SOLVER)
        out = {}
        for name in ("block", "block_series", "global"):
            lqcd.lqcd_profile_reset(lat.h)
            if name == "block":
                x, it, rs = lat.block_solve(b, WL["kappa"], -1, 0, prec, tol=WL["tol"])
                it, rs = it[:lat.nb], max(rs[:lat.nb])
            elif name == "block_series":
                # the same 8 slab systems by the geometric series: W1,eo of the
                # l0 = 4 slabs is the sub-slab operator of an l0 = 8 handle
                lat2 = lqcd.Lattice(L, 2 * l0, -1, l0s=l0)
                lat2.set_gauge(U)
                lqcd.lqcd_profile_enable(lat2.h, 1 << lqcd.KERNEL_SOLVER)
                x, it = lat2.solve_w3eo(b[:lat.Vh].contiguous(), WL["kappa"], 0.0, 0, prec, tol=WL["tol"],
                                        method=lqcd.SOLVER_SERIES)
                n, ms, by = lqcd.lqcd_profile_read(lat2.h, lqcd.KERNEL_SOLVER)
                out[name] = {"iters": it[:lat2.nbs], "ms": ms, "alg_bytes": by, "gbs": by / ms / 1e6}
                lat2.close()
                continue
            else:
                x, it, rs = lat.solve(b, WL["kappa"], 0, prec, tol=WL["tol"])
            n, ms, by = lqcd.lqcd_profile_read(lat.h, lqcd.KERNEL_SOLVER)
            out[name] = {"iters": it, "resid": rs, "ms": ms, "alg_bytes": by, "gbs": by / ms / 1e6}
        # the global solve with the Schwarz preconditioner (Sec. 3, S4
        # solver) for several series lengths of its slab solves; each timed
        # after one untimed solve
        for tag, meth in (("sap", lqcd.SOLVER_SAP), ("sapb", lqcd.SOLVER_SAP_BLOCKS)):
            for nsap in args.sap_sweep:
                lqcd.lqcd_set_global_solver(lat.h, meth, nsap)
                lat.solve(b, WL["kappa"], 0, prec, tol=WL["tol"])
                lqcd.lqcd_profile_reset(lat.h)
                x, it, rs = lat.solve(b, WL["kappa"], 0, prec, tol=WL["tol"])
                n, ms, by = lqcd.lqcd_profile_read(lat.h, lqcd.KERNEL_SOLVER)
                out["global_%s%d" % (tag, nsap)] = {"iters": it, "resid": rs, "ms": ms, "alg_bytes": by,
                                                    "gbs": by / ms / 1e6}
        lqcd.lqcd_set_global_solver(lat.h, lqcd.SOLVER_BICGSTAB, 0)
        print(json.dumps({"case": "solver", "lattice": "x".join(map(str, L)), "precision": args.precision,
                          **out}), flush=True)
        lat.close()
    else:
        # even-odd hopping sweep at 32^3 x 64, the lattice of the bench's
        # Dslash figure (one launch moves 0.3-1.6 GB, far more than L2)
        L = DSLASH_L
        lat = lqcd.Lattice(L, 8, -1)
        U = syn.random_links_torch(L, WL["eps"], WL["seed"], "cuda").contiguous()
        lat.set_gauge(U)
        x = torch.randn((lat.Vh, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
        lqcd.lqcd_profile_enable(lat.h, 1 << lqcd.KERNEL_HOP)
        out = {}
        for name, pr in (("f32", lqcd.PREC_F32), ("f16", lqcd.PREC_F16), ("bf16", lqcd.PREC_BF16),
                         ("f64", lqcd.PREC_F64)):
            lat.dslash_eo(x, 0, 0.0, 0, lqcd.OP_HOP, pr)  # warm-up: launch 4k of this precision
            lqcd.lqcd_profile_reset(lat.h)
            for _ in range(3):
                lat.dslash_eo(x, 0, 0.0, 0, lqcd.OP_HOP, pr)
            n, ms, by = lqcd.lqcd_profile_read(lat.h, lqcd.KERNEL_HOP)
            out[name] = {"ms": ms / n, "gbs": by / ms / 1e6, "bytes_per_launch": by / n}
        print(json.dumps({"case": "dslash", "lattice": "x".join(map(str, L)), **out}), flush=True)
        lat.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default=None, choices=["solver", "dslash", "iterated", "production", "table1"],
                    help="run one small kernel case instead of the benchmark (profiler captures)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f16", "bf16", "f32", "f64"],
                    help="storage of the inner Krylov iterations (outer residuals stay double)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--block-solver", default="series", choices=["bicgstab", "series"],
                    help="inner iteration of the W1 slab solves of the trajectory (the paper's "
                         "geometric series by default)")
    ap.add_argument("--eo-solver", default="bicgstab", choices=["bicgstab", "series"],
                    help="inner iteration of the S2 / S1 solves (--case production)")
    ap.add_argument("--therm-fermion", type=int, default=80,
                    help="trajectories with the fermion action after the pure-gauge thermalisation "
                         "(input preparation, untimed)")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="trajectories of the plain double form timed on the first timed inputs")
    ap.add_argument("--ref-sample-seconds", type=float, default=5.0,
                    help="--impl reference: wall seconds of oracle work per step")
    ap.add_argument("--force-profile", action="store_true",
                    help="add the per-time-slice force profile of each term to the line")
    ap.add_argument("--detail", default=None, help="write per-trajectory records to this JSON file")
    ap.add_argument("--global-solver", default="bicgstab", choices=["bicgstab", "sap", "sap-blocks"],
                    help="inner iteration of the whole-lattice solves: even-odd BiCGstab, or BiCGstab "
                         "with the Schwarz preconditioner (Sec. 3, S4 solver) over the x0-slabs or over "
                         "4-D blocks")
    ap.add_argument("--sap-terms", type=int, default=4,
                    help="geometric-series terms of every slab solve of the Schwarz preconditioner")
    ap.add_argument("--sap-sweep", type=int, nargs="*", default=[1, 2, 4, 8],
                    help="--case solver: series lengths of the Schwarz-preconditioned global solves timed")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-dslash", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--chrono", type=int, default=2, choices=[1, 2, 3],
                    help="chronological guesses: 1 linear (two solutions), 2 quadratic (three), 3 quadratic "
                         "with minimal-residual guesses (six solutions) for the whole-lattice solves")
    ap.add_argument("--no-chrono", action="store_true",
                    help="start every force solve from zero instead of the previous solution of its term")
    ap.add_argument("--no-graph", action="store_true",
                    help="run the molecular dynamics eagerly instead of replaying it as a CUDA graph")
    args = ap.parse_args()
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
