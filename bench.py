#!/usr/bin/env python
"""Benchmark: even-odd preconditioned Wilson CG to a 1e-10 FP64 true residual
on a 24^3 x 48 lattice (links exp(0.3 i H), m = 0.01) on one GB300.

One step = one full solve of D_W x = b from resident FP64 inputs with
lqcd_eo_solve: link preparation (FP64 and FP16 / 12-real device layouts),
source preparation b_hat = b_e + H_eo b_o / 2c, CGNR on M_hat^dag M_hat with
FP16-storage / 12-real inner iteration, FP32-arithmetic residual replacements
and reliable updates of b_hat - M_hat x in double-float arithmetic on the FP64
fields, and the odd half. The headline value is the Dslash throughput
sustained inside the step: (hops in the step) x 1320 flop x Vh / step time.
The JSON line also carries the FP64 and other mixed solves (the mixed vs FP64
comparison), the roofline of the dominant kernel (the FP16 / 12-real hop), the
oracle CPU baseline on the host cores and the end-to-end number through host
buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lqcd|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GFLOP/s & HBM-roofline %; mixed vs FP64 CG time to 1e-10 residual"
FLOP_PER_SITE = 1320
BC = (1.0, 1.0, 1.0, -1.0)
WORKLOAD = "wilson_eo_cg_24x24x24x48_m0.01_exp0.3_tol1e-10"
# Solver variants of the headline workload, key -> (inner storage precision, delta, delta_mid).
# Every variant is lqcd_eo_solve (even-odd CGNR: the exit test is the FP64 residual of the
# even-odd system, ||b_hat - M_hat x|| / ||b_hat||). A reliable update recomputes it with two
# FP64 hops, which on GB300 are bound by the FP64 pipe, so the largest drop per update that the
# inner iteration sustains wins: delta = 3e-6 with FP32 storage (2 updates, 64 iterations;
# 1e-5 needs 3 updates under this exit test) and 0.003 with FP16 storage alone (5 updates).
# Variant 3 keeps FP16 storage and puts FP32-arithmetic residual replacements (delta_mid =
# 0.003) between the FP64 updates at delta = 3e-6: 2 updates, 3 replacements, 66 iterations,
# the fastest (16.7 ms against 17.6 ms for FP32 storage, whole even-odd solve).
VARIANTS = {0: (0, 0.1, 0.0), 1: (1, 3e-6, 0.0), 2: (2, 0.003, 0.0), 3: (2, 3e-6, 0.003)}
VARIANT_NAMES = {0: "fp64", 1: "mixed_fp32", 2: "mixed_fp16", 3: "mixed_fp16_three_level"}
HEADLINE = 3
HEADLINE_PREC = VARIANTS[HEADLINE][0]
DELTA = {q: VARIANTS[q][1] for q in (0, 1, 2)}
DELTA_3LVL, DELTA_MID = VARIANTS[3][1], VARIANTS[3][2]
# lqcd_cg_solve (normal-equation exit test: multi-RHS, force, batch) keeps 1e-5 with FP32 storage
DELTA_NORMAL_FP32 = 1e-5
PREC_TAG = {1: "f32", 2: "f16"}
PROFILE_JSON = {q: os.path.join(ROOT, "profiles", f"hop_{PREC_TAG[q]}r12_24x24x24x48.json") for q in (1, 2)}
DSLASH_COMMON = ["dslash_kernels.cuh", "lqcd_common.cuh", "cg_site.cuh", "dslash_launch.cuh", "hop_pair.cuh", "df.cuh",
                 "hop_async.cuh", "lqcd_internal.h"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lqcd", "reference"], default="lqcd")
    ap.add_argument("--dims", type=int, nargs=4, default=[24, 24, 24, 48])
    ap.add_argument("--mass", type=float, default=0.01)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the solver's kernels directly instead of replaying its CUDA graph "
                         "(profilers list kernels inside conditional graph bodies only this way)")
    ap.add_argument("--check-interval", type=int, default=64,
                    help="iterations per graph launch / host check of the solver")
    ap.add_argument("--tune-file", default=None,
                    help="autotuner table: loaded before the run if the file exists (no launch shape is then "
                         "re-timed), written after it otherwise -- so that a profiler run launches the same "
                         "shapes as the plain run that wrote it")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the domain-wall, multi-RHS, batch and force measurements")
    ap.add_argument("--hop-shape", default=None,
                    help="hops mode: run only this shape (f32r12_24x24x24x48, f16r12_24x24x24x48, "
                         "dwf_f32r12_16x4_ls16, f32r12_32x4_12rhs)")
    ap.add_argument("--hop-prec", type=int, choices=[0, 1, 2, 3], default=HEADLINE_PREC,
                    help="the hop timed by --mode hop: 1 FP32, 2 FP16 storage (12-real links); 0 FP64, "
                         "3 FP64 fields in double-float arithmetic (18-real links)")
    ap.add_argument("--mode", choices=["full", "step", "hop", "hops", "dwf", "blockcg"], default="full",
                    help="step: only the timed solves; hop: only the dominant kernel's roofline loop; "
                         "hops: the three hop shapes (profiling)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_inputs(dims):
    from synthetic import config_seed, gauge_field, gaussian_spinor
    U = gauge_field(dims, "exp", config_seed(1, 0), eps=0.3)
    b = gaussian_spinor(dims, config_seed(1, 1), lead=(1,))
    return U, b


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ L2 flush

class L2Flush:
    """Leaves L2 cold and clean before a timed region: writes a 512 MB buffer (4x the
    129 MB L2), then reads a separate 256 MB buffer, so that the dirty lines of the
    write are written back inside the flush and not during the timed kernel (a
    write-only flush leaves up to an L2 of dirty lines whose write-back lands on
    whatever runs next)."""

    def __init__(self, device):
        import torch
        self.w = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=device)
        self.r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=device)

    def __call__(self):
        import torch
        self.w.zero_()
        torch.sum(self.r)


# ------------------------------------------------------------------ oracle timing (CPU baseline)

def host_info():
    """Core count, CPU model and memory of the host the oracle runs on."""
    info = {"nproc": os.cpu_count() or 1}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Model name", "Architecture", "CPU(s)", "L3 cache"):
                info[k.strip()] = v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/meminfo") as fh:
            for ln in fh:
                if ln.startswith("MemAvailable:"):
                    info["mem_available_gb"] = round(int(ln.split()[1]) / 1e6, 1)
    except OSError:
        pass
    return info


def _time_oracle_hops(path, reps):
    from oracle import wilson
    U = np.load(path + ".U.npy", mmap_mode="r")
    psi = np.load(path + ".psi.npy", mmap_mode="r")
    t0 = time.perf_counter()
    for _ in range(reps):
        wilson.hop_eo(U, psi, BC, 0)
    return time.perf_counter() - t0


def _oracle_fields(dims, seed, tmpdir):
    from oracle import wilson
    from synthetic import gauge_field, gaussian_spinor
    base = os.path.join(tmpdir, "x".join(map(str, dims)))
    if not os.path.exists(base + ".psi.npy"):
        np.save(base + ".U.npy", gauge_field(dims, "exp", seed, eps=0.3))
        np.save(base + ".psi.npy", wilson.restrict(gaussian_spinor(dims, seed + 1, lead=(1,))[0], 1))
    return base


def cpu_baseline(budget_s=40.0):
    """The FP64 numpy oracle, as it stands, on the host cores: even-odd hop GFLOP/s
    (1320 flop per output site) on 8^4, 16^4 and 24^3 x 48 with one process and with
    one process per core (a spawn pool: every process times its own hops on
    memory-mapped shared fields; the aggregate is all processes' flops over the wall
    time), and the oracle's unpreconditioned CG on M^dag M of config 1 (8^4, Haar
    links, m = 0.1) to 1e-10, measured. The oracle itself runs on one thread
    (numpy einsum and roll)."""
    import multiprocessing as mp
    import tempfile
    from oracle import cg as ocg
    from oracle import wilson
    from synthetic import config_seed, gauge_field, gaussian_spinor
    info = host_info()
    cores = int(info["nproc"])
    t_start = time.perf_counter()
    out = {"host": info, "hop_gflops": {}}
    tmpdir = tempfile.mkdtemp(prefix="lqcd_oracle_")
    big_ok = info.get("mem_available_gb", 0.0) >= 3.0 * cores  # ~2 GB of temporaries per process at 24^3 x 48
    sizes = [((8, 8, 8, 8), 20), ((16, 16, 16, 16), 3), ((24, 24, 24, 48), 1)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for dims, reps in sizes:
            vh = int(np.prod(dims)) // 2
            base = _oracle_fields(dims, 7, tmpdir)
            one = _time_oracle_hops(base, reps)
            row = {"1_core": round(reps * FLOP_PER_SITE * vh / one / 1e9, 4), "sample_1_core_s": round(one, 2)}
            if dims != (24, 24, 24, 48) or big_ok:
                t0 = time.perf_counter()
                times = pool.map(_time_oracle_hops_star, [(base, reps)] * cores)
                wall = time.perf_counter() - t0
                row[f"{cores}_cores"] = round(cores * reps * FLOP_PER_SITE * vh / wall / 1e9, 4)
                row["sample_all_cores_s"] = round(wall, 2)
                row["per_process_s_max"] = round(max(times), 2)
            out["hop_gflops"]["x".join(map(str, dims))] = row
    # config 1: 8^4 Haar links, m = 0.1, unpreconditioned CG on M^dag M to 1e-10 (measured)
    dims = (8, 8, 8, 8)
    U = gauge_field(dims, "haar", config_seed(0, 0))
    b = gaussian_spinor(dims, config_seed(0, 1), lead=(1,))
    t0 = time.perf_counter()
    _, inf = ocg.cg(lambda v: wilson.dirac_dag_dirac(U, v, 0.1, BC), b, 1e-10, 5000)
    dt = time.perf_counter() - t0
    out["cg_8x4_m0.1_unpreconditioned"] = {"seconds": round(dt, 2), "iterations": inf.iterations,
                                          "seconds_per_iteration": round(dt / max(inf.iterations, 1), 4),
                                          "true_rel_residual": inf.true_rel_residual, "cores": 1}
    out["elapsed_s"] = round(time.perf_counter() - t_start, 1)
    return out


def _time_oracle_hops_star(args):
    return _time_oracle_hops(*args)


# ------------------------------------------------------------------ lqcd arm

def dslash_sources_hash(prec):
    """Hash of the sources that make the hop kernel of one storage precision."""
    h = hashlib.sha256()
    for f in DSLASH_COMMON + [f"dslash_{PREC_TAG[prec]}.cu", f"dslash_{PREC_TAG[prec]}_dag.cu"]:
        with open(os.path.join(ROOT, "paper_1512_03487_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def workload_config(dims, mass, world):
    """The workload both arms name (the GPU arm and the oracle reference arm)."""
    return {"workload": WORKLOAD, "lattice": list(dims), "mass": mass, "bc": list(BC),
            "solver": "lqcd_eo_solve: even-odd CGNR (CG on M_hat^dag M_hat x = M_hat^dag b_hat), "
                      "FP16-storage / 12-real inner iteration, FP32-arithmetic residual replacements at "
                      f"delta_mid {DELTA_MID}, reliable updates of b_hat - M_hat x in double-float arithmetic on the "
                      f"FP64 fields at delta {DELTA_3LVL}",
            "tol": 1e-10, "tol_applies_to": "true residual of the full system, ||b - D x|| / ||b||: the exit test "
                                            "is ||b_hat - M_hat x_e|| <= tol ||b|| on the reliable update's "
                                            "b_hat - M_hat x_e (the full residual's even rows; its odd rows "
                                            "vanish once x_o is reconstructed), recomputed with the FP64 "
                                            "operator after the step",
            "l2": "flushed before every timed step (512 MB write, then 256 MB read)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_lqcd(args, world, rank, local):
    import torch

    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    tune_loaded = False
    if args.tune_file and os.path.exists(args.tune_file):
        L.lqcd_tune_load(args.tune_file)
        tune_loaded = True
    try:
        _run_lqcd(args, world, rank, local, L, F, dev, stream)
    finally:
        if args.tune_file and not tune_loaded and rank == 0:
            L.lqcd_tune_save(args.tune_file)


def _run_lqcd(args, world, rank, local, L, F, dev, stream):
    import torch
    if args.mode == "hops":
        # profiling mode: the three hop shapes of the hot path on zero-filled fields
        # (the kernels do the same work whatever the values), args.steps launches each
        flush = L2Flush(dev)
        shapes = {
            "f32r12_24x24x24x48": lambda: _hop_gbs(L, F, L.lattice((24, 24, 24, 48), bc=BC), 1, 12, 576, flush,
                                                   stream, n=args.steps),
            "f16r12_24x24x24x48": lambda: _hop_gbs(L, F, L.lattice((24, 24, 24, 48), bc=BC), 2, 12, 296, flush,
                                                   stream, n=args.steps),
            "dwf_f32r12_16x4_ls16": lambda: _hop_gbs(L, F, L.lattice((16, 16, 16, 16), n5=16, bc=BC), 1, 12,
                                                     8 * 48 / 16 + 192, flush, stream, kind=L.LQCD_DWF, n=args.steps),
            "f32r12_32x4_12rhs": lambda: _hop_gbs(L, F, L.lattice((32, 32, 32, 32), n5=12, bc=BC), 1, 12,
                                                  8 * 48 / 12 + 192, flush, stream, n=args.steps)}
        names = [args.hop_shape] if args.hop_shape else list(shapes)
        res = {name: shapes[name]() for name in names}
        if rank == 0:
            print(json.dumps({"mode": "hops", "hops": res}), flush=True)
        return
    if args.mode == "blockcg":
        # profiling mode: one block CG solve of the 32^4 x 12-RHS workload (FP32 inner, double-float
        # updates), honouring --no-graph / --check-interval
        res = block_cg_bench(L, F, L2Flush(dev), stream, use_graph=0 if args.no_graph else 1,
                             check_interval=args.check_interval)
        if rank == 0:
            print(json.dumps({"mode": "blockcg", "block_cg": res}), flush=True)
        return
    if args.mode == "dwf":
        # profiling mode: the domain-wall solve alone (FP32 inner), honouring --no-graph / --check-interval
        res = dwf_bench(L, F, L2Flush(dev), stream, use_graph=0 if args.no_graph else 1,
                        check_interval=args.check_interval, three_level=False)
        if rank == 0:
            print(json.dumps({"mode": "dwf", "dwf": res}), flush=True)
        return
    dims = tuple(args.dims)
    mass = args.mass
    U, b = make_inputs(dims)
    V = int(np.prod(dims))
    vh = V // 2
    lat = L.lattice(dims, bc=BC)
    op64 = L.operator(mass=mass, prec=L.LQCD_F64, recon=18)
    stream = torch.cuda.current_stream()

    # resident FP64 inputs in the user layout
    U_dev = torch.from_numpy(np.ascontiguousarray(U).view(np.float64).reshape(-1)).to(dev)
    b_dev = torch.from_numpy(np.ascontiguousarray(b).view(np.float64).reshape(-1)).to(dev)
    g64 = F.empty(L.lqcd_gauge_bytes(lat, L.LQCD_F64, 18))
    gs = {p: F.empty(L.lqcd_gauge_bytes(lat, p, 12)) for p in (L.LQCD_F32, L.LQCD_F16)}
    bfull = F.empty(L.lqcd_spinor_bytes(lat, L.LQCD_F64, L.LQCD_FULL))
    x = F.empty(L.lqcd_spinor_bytes(lat, L.LQCD_F64, L.LQCD_FULL))
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op64, L.LQCD_EVEN))
    # mixed solves run their reliable updates and source preparation in double-float arithmetic
    prms = {k: L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=q, sloppy_recon=12 if q else 18,
                               delta=d, delta_mid=dm, check_interval=args.check_interval,
                               use_graph=0 if args.no_graph else 1,
                               update_prec=L.LQCD_F64_DF if q else L.LQCD_F64)
            for k, (q, d, dm) in VARIANTS.items()}
    ws = F.empty(max(L.lqcd_eo_solve_workspace_bytes(lat, op64, prms[k]) for k in prms))
    flush = L2Flush(dev)

    def step(key):
        """One solve of D_W x = b from the resident FP64 inputs; returns hops executed."""
        sloppy = prms[key].sloppy_prec
        L.lqcd_gauge_pack(g64, L.LQCD_F64, 18, U_dev, lat)
        gsl = g64
        if sloppy:
            gsl = gs[sloppy]
            L.lqcd_gauge_pack(gsl, sloppy, 12, U_dev, lat)
        L.lqcd_spinor_pack(bfull, L.LQCD_F64, L.LQCD_FULL, b_dev, lat)
        info = L.lqcd_eo_solve(x, bfull, g64, gsl, lat, op64, prms[key], ws)
        # preparation, CGNR start, 4 per iteration, update and replacement; the odd half reuses the last
        # update's hop
        hops = 1 + 2 + 4 * (info.iterations + info.reliable_updates + info.residual_replacements)
        return hops, info

    def timed(fn, *a):
        # the flush is queued, not waited for: while the GPU runs it the host queues the
        # events and the step's first kernels, so no host latency lands between e0 and them
        torch.cuda.synchronize()
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn(*a)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    if args.mode == "hop":
        # profiling mode: only one hop's roofline loop
        if args.hop_prec in (0, 3):
            L.lqcd_gauge_pack(g64, L.LQCD_F64, 18, U_dev, lat)
            roof = (fp64_hop_roofline if args.hop_prec == 0 else df_hop_roofline)(L, F, lat, g64, flush, stream, vh,
                                                                                 launches=args.steps)
            if rank == 0:
                print(json.dumps({"mode": "hop", "roofline": roof}), flush=True)
            return
        L.lqcd_gauge_pack(gs[args.hop_prec], args.hop_prec, 12, U_dev, lat)
        roof = hop_roofline(L, F, lat, gs[args.hop_prec], args.hop_prec, flush, stream, vh, launches=args.steps)
        if rank == 0:
            print(json.dumps({"mode": "hop", "roofline": roof}), flush=True)
        return

    # ---- headline: the fastest mixed precision solve (FP16 storage, three levels)
    for _ in range(args.warmup):
        step(HEADLINE)
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.lqcd_launch_count()
    total_ms, total_hops, infos = 0.0, 0, []
    for _ in range(args.steps):
        ms, (hops, info) = timed(step, HEADLINE)
        total_ms += ms
        total_hops += hops
        infos.append(info)
    launches = L.lqcd_launch_count() - launches0
    clk = clocks.stop()
    barrier(world)
    max_ms, flops_all, value = aggregate(total_ms, float(total_hops) * FLOP_PER_SITE * vh, world)

    # the solve must meet the FP64 true residual of the full system (checked on the device result)
    res = full_residual(L, F, lat, op64, g64, x, b_dev, tmp)
    if args.mode == "step":
        # profiling mode: only the timed solves
        if rank == 0:
            print(json.dumps({"mode": "step", "value": round(value, 1), "ms_per_step": max_ms / args.steps,
                              "iterations": infos[-1].iterations, "full_system_rel_residual": res,
                              "gpu_launches": int(launches)}), flush=True)
        return

    # ---- mixed vs FP64 comparison (median of five timed solves each after one warm-up)
    cgcmp = {}
    for p, name in VARIANT_NAMES.items():
        if p != HEADLINE:
            step(p)
        runs = sorted((timed(step, p) for _ in range(5)), key=lambda r: r[0])
        ms, (hops, info) = runs[2]  # median of 5 after one warm-up
        cgcmp[name] = {"ms": round(ms, 3), "iterations": info.iterations,
                       "reliable_updates": info.reliable_updates, "delta": prms[p].delta,
                       "true_rel_residual_full_system": info.true_rel_residual,
                       "dslash_gflops": round(hops * FLOP_PER_SITE * vh / (ms * 1e-3) / 1e9, 1)}
        if p == 3:
            cgcmp[name].update({"delta_mid": prms[p].delta_mid,
                                "fp32_replacements": info.residual_replacements})
    for name in ("mixed_fp32", "mixed_fp16", "mixed_fp16_three_level"):
        cgcmp["speedup_" + name[6:] + "_vs_fp64"] = round(cgcmp["fp64"]["ms"] / cgcmp[name]["ms"], 2)

    # ---- roofline of the dominant kernel: the inner hop (12-real links, the headline's storage
    # precision), one checkerboard; the FP32 storage hop beside it; and the FP64 hop of the
    # reliable updates, bound by the FP64 pipe
    roof = hop_roofline(L, F, lat, gs[HEADLINE_PREC], HEADLINE_PREC, flush, stream, vh)
    L.lqcd_gauge_pack(gs[1], 1, 12, U_dev, lat)
    roof32 = hop_roofline(L, F, lat, gs[1], 1, flush, stream, vh)
    roof64 = fp64_hop_roofline(L, F, lat, g64, flush, stream, vh)
    roofdf = df_hop_roofline(L, F, lat, g64, flush, stream, vh)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(L, F, lat, op64, U, b, prms[HEADLINE], ws, tmp, x, gs[HEADLINE_PREC], g64, bfull,
                      flush, stream, vh, args, world)

    # ---- the other hot-path workloads (domain wall, multi-RHS, uneven batch, force)
    extras = None
    if not args.no_extras:
        del U_dev, g64, gs, ws, tmp, x, bfull
        torch.cuda.empty_cache()
        extras = run_extras(L, F, flush, stream)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 arithmetic on f16 storage (per-site norm, 12-real links) in the inner iteration, "
                 "f32-arithmetic residual replacements, f64 reliable updates and true residual",
        "data": "synthetic (seeded exp(0.3 i H) links, Gaussian source)",
        "config": workload_config(dims, mass, world),
        "full_system_rel_residual": res,
        "iterations_per_step": infos[-1].iterations, "reliable_updates_per_step": infos[-1].reliable_updates,
        "fp32_replacements_per_step": infos[-1].residual_replacements,
        "cg": cgcmp,
        "roofline": roof,
        "roofline_fp32_hop": roof32,
        "roofline_fp64_hop": roof64,
        "roofline_df_hop": roofdf,
        "gpu_launches": int(launches),
        "clocks": clk,
        "tuned_hop_shapes": solve_hop_shapes(L, dims),
    }
    if e2e is not None:
        line["e2e"] = e2e
    if extras is not None:
        line["extras"] = extras
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
        big = cb["hop_gflops"]["24x24x24x48"]
        allc = [k for k in big if k.endswith("_cores")]
        key16 = "16x16x16x16"
        if allc:
            value, cores, where = big[allc[0]], cb["host"]["nproc"], "24^3 x 48"
        else:  # not enough host memory for one 24^3 x 48 oracle process per core
            allc16 = [k for k in cb["hop_gflops"][key16] if k.endswith("_cores")]
            value, cores, where = cb["hop_gflops"][key16][allc16[0]], cb["host"]["nproc"], "16^4"
        line["cpu_baseline"] = {
            "value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"even-odd hops of the FP64 numpy oracle on {where} (exp(0.3 i H) links), one process "
                      f"per core, each timing its own hops on memory-mapped shared fields; aggregate flops "
                      f"(1320 per output site) over the wall time",
            "detail": cb}
    if rank == 0:
        print(json.dumps(line), flush=True)


def packed_full_residual(L, F, lat, op64, g64, x, bd):
    """||b - M x|| / ||b|| for x and b both in the FP64 device layout (full lattice):
    M x with the FP64 operator, both unpacked to the host layout, whose size is
    2 x the complex entries of host_spinor_shape (padding sites never enter)."""
    import torch
    dx = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_FULL))
    L.lqcd_M(dx, x, g64, lat, op64, L.LQCD_FULL, 0, None)
    n = 2 * int(np.prod(F.host_spinor_shape(lat, L.LQCD_FULL)))
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    bb = torch.empty(n, dtype=torch.float64, device="cuda")
    L.lqcd_spinor_unpack(a, dx, L.LQCD_F64, L.LQCD_FULL, lat)
    L.lqcd_spinor_unpack(bb, bd, L.LQCD_F64, L.LQCD_FULL, lat)
    return float(torch.linalg.vector_norm(a - bb) / torch.linalg.vector_norm(bb))


def full_residual(L, F, lat, op64, g64, x, b_dev, tmp):
    """||b - D_W x|| / ||b|| of the step's result, computed with the FP64 operator
    and compared in the host layout (padding sites never enter)."""
    import torch
    dx = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    L.lqcd_M(dx, x, g64, lat, op64, L.LQCD_FULL, 0, None)
    a = torch.empty_like(b_dev)
    L.lqcd_spinor_unpack(a, dx, L.LQCD_F64, L.LQCD_FULL, lat)
    return float(torch.linalg.vector_norm(a - b_dev) / torch.linalg.vector_norm(b_dev))


L2_BYTES = 129e6  # GB300 L2 (nvidia-smi / device properties: 126.5 MiB)


def _cold_hop_seconds(L, F, lat, g, prec, recon, flush, stream, launches, rotate=True):
    """Event-timed duration of one checkerboard hop launch with its inputs not in L2.

    rotate=True: the launches run back to back, one event pair around all of
    them, cycling through enough copies of the links and the input spinor that
    the copy a launch reads was last touched more than 2 x L2 bytes of traffic
    earlier (inputs larger than L2); the mean per launch carries no event or
    launch latency. rotate=False: the L2 is flushed before every launch, each
    launch timed alone with its own event pair (that adds the events' and the
    launch's own latency, a few us, and the timer's resolution), mean over the
    launches."""
    import torch
    op = L.operator(prec=prec, recon=recon)
    fprec = L.LQCD_F64 if prec == L.LQCD_F64_DF else prec  # double-float arithmetic on FP64 fields
    rng = np.random.default_rng(5)
    shape = F.host_spinor_shape(lat, L.LQCD_ODD)
    host = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    fin = F.spinor_to_device(host, lat, fprec, L.LQCD_ODD)
    out = F.empty(L.lqcd_spinor_bytes(lat, fprec, L.LQCD_EVEN))
    for _ in range(3):
        L.lqcd_dslash(out, fin, g, lat, op, L.LQCD_EVEN, 0)
    if rotate:
        per_copy = g.numel() * g.element_size() + fin.numel() * fin.element_size()
        ncopy = max(2, int(np.ceil(2 * L2_BYTES / per_copy)) + 1)
        gs, fins = [g] + [g.clone() for _ in range(ncopy - 1)], [fin] + [fin.clone() for _ in range(ncopy - 1)]
        for k in range(ncopy):
            L.lqcd_dslash(out, fins[k], gs[k], lat, op, L.LQCD_EVEN, 0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(launches):
            L.lqcd_dslash(out, fins[i % ncopy], gs[i % ncopy], lat, op, L.LQCD_EVEN, 0)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / launches
        del gs, fins
        return t * 1e-3
    times = []
    for _ in range(launches):
        # flush queued behind a synchronize, events and launch queued while it runs: e0 -> e1
        # spans the kernel on the device, not the host's launch latency
        torch.cuda.synchronize()
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.lqcd_dslash(out, fin, g, lat, op, L.LQCD_EVEN, 0)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.mean(times)) * 1e-3


def hop_roofline(L, F, lat, gsl, prec, flush, stream, vh, launches=40):
    t = _cold_hop_seconds(L, F, lat, gsl, prec, 12, flush, stream, launches)
    t_flush = _cold_hop_seconds(L, F, lat, gsl, prec, 12, flush, stream, 20, rotate=False)
    # 8 links of 12 reals + input and output spinor, in the inner precision
    bytes_per_site = {1: 8 * 48 + 96 + 96, 2: 8 * 24 + 52 + 52}[prec]
    achieved = bytes_per_site * vh / t / 1e9
    peak, peak_src = measured_peak()
    traffic = None
    try:
        with open(PROFILE_JSON[prec]) as fh:
            prof = json.load(fh)
        if prof.get("source_hash") == dslash_sources_hash(prec) and list(prof.get("lattice", [])) == list(lat.dims):
            traffic = prof.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    name = {1: "F32", 2: "F16"}[prec]
    shape = L.lqcd_tune_get(hop_key(prec, 12, 0, 0, 0, lat.dims, 1))
    # no-reuse model: every neighbour spinor fetched once per use (8 in, 8 links, 1 out)
    no_reuse = {1: 8 * 48 + 8 * 96 + 96, 2: 8 * 24 + 8 * 52 + 52}[prec]
    return {"bound": "hbm", "kernel": f"hop_kernel<{name}, recon 12> (one checkerboard, inputs not in L2)",
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "peak_source": peak_src, "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_site * vh,
            "no_reuse_bytes_per_launch": no_reuse * vh,
            "launch_us": round(t * 1e6, 2), "gflops": round(FLOP_PER_SITE * vh / t / 1e9, 1),
            "timing": f"{launches} launches back to back, inputs rotated over copies totalling more than 2 x L2, "
                      f"one event pair (mean per launch)",
            "launch_us_flush_each": round(t_flush * 1e6, 2),
            "frac_flush_each": round(bytes_per_site * vh / t_flush / 1e9 / peak, 4),
            "launch_shape": {"index": shape, "meaning": HOP_SHAPE_MEANING.get(shape, "default")}}


HOP_SHAPE_MEANING = {0: "128 threads, one site per thread", 1: "128 threads, one site per thread, <= 72 registers",
                     2: "128 threads, one site per thread, spin components paired in packed FP32x2 arithmetic, "
                        "<= 72 registers", 3: "128 threads, one site per thread, <= 102 registers",
                     4: "128 threads, two sites per thread in packed FP32x2 arithmetic",
                     5: "128 threads, one site per thread, links staged in shared memory when n5 >= 4",
                     6: "128 threads, one site per thread, spin components paired in packed FP32x2 arithmetic",
                     7: "128 threads, one site per thread, <= 72 registers, neighbour spinors and links copied "
                        "asynchronously (cp.async) through a shared-memory ring",
                     8: "128 threads, one site per thread, spin-paired packed FP32x2 arithmetic, <= 72 registers, "
                        "neighbour data copied asynchronously through a shared-memory ring"}


def hop_key(prec, recon, dagger, epi, red, dims, n5, full=0):
    """The autotuner table's key of one hop kernel launch (include/lqcd.h)."""
    X, Y, Z, T = (int(d) for d in dims)
    return f"hop prec={prec} recon={recon} dagger={dagger} epi={epi} red={red} full={full} lat={X}x{Y}x{Z}x{T} n5={n5}"


def solve_hop_shapes(L, dims):
    """The launch shapes the tuner chose for the inner iteration's FP16 hops and the FP32 level's hops."""
    out = {}
    for prec in (2, 1):
        for dag, epi, red, what in ((0, 0, 0, "H_oe p"), (0, 1, 1, "M_hat p with |.|^2"), (1, 0, 0, "H^dag"),
                                    (1, 1, 2, "M_hat^dag with the fused CG update")):
            v = L.lqcd_tune_get(hop_key(prec, 12, dag, epi, red, dims, 1))
            if v >= 0:
                out[f"prec{prec} dagger{dag} epi{epi} red{red} ({what})"] = v
    return out


# GB300 FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA per SM per clock x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def fma_peak(L, F, prec, stream):
    """Measured FMA-chain rate (TFLOP/s) of the FMA probe (paper_1512_03487_gb300/measure, a library of its
    own): 152 x 8 blocks of 256 threads, best of 3."""
    import torch
    from paper_1512_03487_gb300 import measure as probe
    blocks = 152 * 8
    iters = 4096 if prec == 0 else 262144
    sink = torch.empty(blocks * 256, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    probe.fma_probe(sink, prec, iters, blocks)
    best = None
    for _ in range(3):
        t, _ = _events_time(lambda: probe.fma_probe(sink, prec, iters, blocks), stream)
        best = t if best is None else min(best, t)
    return 16.0 * iters * blocks * 256 / (best * 1e-3) / 1e12


def fp64_hop_roofline(L, F, lat, g64, flush, stream, vh, launches=5):
    """The FP64 hop of the reliable updates against the FP64 pipe: 1320 flop per site over the
    GB300 FP64 rate from unit counts and clock (FP64_PEAK_TFLOPS), the measured FMA-chain rate beside it."""
    t = _cold_hop_seconds(L, F, lat, g64, L.LQCD_F64, 18, flush, stream, launches)
    tf = FLOP_PER_SITE * vh / t / 1e12
    meas = fma_peak(L, F, 0, stream)
    return {"bound": "alu", "kernel": "hop_kernel<F64, recon 18> (one checkerboard, cold L2)",
            "achieved": round(tf, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
            "frac": round(tf / FP64_PEAK_TFLOPS, 4),
            "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
            "measured_fma_chain_tflops": round(meas, 4), "frac_of_measured_fma": round(tf / meas, 4),
            "launch_us": round(t * 1e6, 2), "hbm_gbs": round((8 * 144 + 192 + 192) * vh / t / 1e9, 1)}


# GB300 FP32 peak from unit counts and clock: 152 SMs x 128 FP32 FMA per SM per clock x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def df_hop_roofline(L, F, lat, g64, flush, stream, vh, launches=5):
    """The reliable updates' hop: FP64 fields in double-float arithmetic (LQCD_F64_DF). Its
    1320 FP64-equivalent flop per site against the FP64 peak it replaces, and its FP32
    instruction rate (about 19,400 FP32 instructions per site, ncu) against the FP32 pipe."""
    t = _cold_hop_seconds(L, F, lat, g64, L.LQCD_F64_DF, 18, flush, stream, launches)
    t64 = _cold_hop_seconds(L, F, lat, g64, L.LQCD_F64, 18, flush, stream, 3)
    tf = FLOP_PER_SITE * vh / t / 1e12
    return {"bound": "alu", "kernel": "hop_kernel<F64_DF, recon 18> (one checkerboard, cold L2)",
            "achieved_fp64_equivalent_tflops": round(tf, 4), "fp64_peak": round(FP64_PEAK_TFLOPS, 4),
            "frac_of_fp64_peak": round(tf / FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
            "fp32_peak": round(FP32_PEAK_TFLOPS, 2), "launch_us": round(t * 1e6, 2),
            "fp64_hop_launch_us": round(t64 * 1e6, 2), "speedup_vs_fp64_hop": round(t64 / t, 2),
            "hbm_gbs": round((8 * 144 + 192 + 192) * vh / t / 1e9, 1)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s (of fallback)"


def run_e2e(L, F, lat, op64, U, b, prm, ws, tmp, x, gsl, g64, bfull, flush, stream, vh, args, world):
    """Same solve through the C ABI from pinned host buffers: H2D of the FP64
    gauge field and source, pack, solve, reconstruct, D2H of the solution."""
    import torch
    U_h = torch.from_numpy(np.ascontiguousarray(U).view(np.float64).reshape(-1)).pin_memory()
    b_h = torch.from_numpy(np.ascontiguousarray(b).view(np.float64).reshape(-1)).pin_memory()
    x_h = torch.empty(b_h.numel(), dtype=torch.float64).pin_memory()
    staging = torch.empty(U_h.numel(), dtype=torch.float64, device=bfull.device)

    def e2e_step():
        L.lqcd_gauge_upload(g64, L.LQCD_F64, 18, U_h, staging, lat)
        L.lqcd_gauge_pack(gsl, HEADLINE_PREC, 12, staging, lat)
        L.lqcd_spinor_upload(bfull, L.LQCD_F64, L.LQCD_FULL, b_h, staging, lat)
        info = L.lqcd_eo_solve(x, bfull, g64, gsl, lat, op64, prm, ws)
        L.lqcd_spinor_download(x_h, x, L.LQCD_F64, L.LQCD_FULL, staging, lat)
        return 1 + 2 + 4 * (info.iterations + info.reliable_updates + info.residual_replacements)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    total, hops = 0.0, 0
    for _ in range(args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hops += e2e_step()
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
    total = allreduce_max(total, world)
    flops = allreduce_sum(float(hops) * FLOP_PER_SITE * vh, world)
    return {"value": round(flops / total / 1e9, 1), "unit": "GFLOP/s",
            "h2d_bytes_per_step": int(U_h.numel() * 8 + b_h.numel() * 8),
            "d2h_bytes_per_step": int(x_h.numel() * 8), "ms_per_step": round(total / args.steps * 1e3, 3)}


# ------------------------------------------------------------------ other workloads

def _events_time(fn, stream, flush=None, reps=1):
    import torch
    best = None
    out = None
    for _ in range(reps):
        torch.cuda.synchronize()
        if flush is not None:
            flush()  # queued: the host queues e0 and fn's first launches while it runs
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best, out


def _hop_gbs(L, F, lat, prec, recon, bytes_per_site, flush, stream, kind=0, n=10):
    """Cold-L2 time of one hop launch (one checkerboard) and its algorithmic GB/s."""
    import torch
    op = L.operator(kind=kind, prec=prec, recon=recon)
    nsites = lat.dims[0] * lat.dims[1] * lat.dims[2] * lat.dims[3] // 2 * lat.n5
    g = F.empty(L.lqcd_gauge_bytes(lat, prec, recon))
    g.zero_()
    fin = F.empty(L.lqcd_spinor_bytes(lat, prec, L.LQCD_ODD))
    fin.zero_()
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, L.LQCD_EVEN))
    for _ in range(2):
        L.lqcd_dslash(out, fin, g, lat, op, L.LQCD_EVEN, 0)
    ts = []
    for _ in range(n):
        t, _ = _events_time(lambda: L.lqcd_dslash(out, fin, g, lat, op, L.LQCD_EVEN, 0), stream, flush)
        ts.append(t)
    t = float(np.mean(ts)) * 1e-3
    peak, _ = measured_peak()
    gbs = bytes_per_site * nsites / t / 1e9
    return {"launch_us": round(t * 1e6, 2), "algorithmic_bytes_per_site": bytes_per_site, "achieved_gbs": round(gbs, 1),
            "frac_of_measured_hbm": round(gbs / peak, 4), "gflops": round(FLOP_PER_SITE * nsites / t / 1e9, 1)}


def block_cg_bench(L, F, flush, stream, use_graph=1, check_interval=64):
    """32^4, 12 Gaussian right-hand sides, Haar links, m = 0.01: block CG on
    M_hat^dag M_hat X = B_e to 1e-10, FP32 / 12-real inner, double-float updates
    (delta 1e-5); one warm-up and one timed solve."""
    from synthetic import config_seed, gauge_field, gaussian_spinor
    dims, nr = (32, 32, 32, 32), 12
    U = gauge_field(dims, "haar", config_seed(3, 0))
    lat = L.lattice(dims, n5=nr, bc=BC)
    op = L.operator(mass=0.01)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    del U
    be = F.spinor_to_device(F.checkerboard(gaussian_spinor(dims, config_seed(3, 1), lead=(nr,)), 0), lat, 0, 0)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=1, sloppy_recon=12, delta=DELTA_NORMAL_FP32,
                          check_interval=check_interval, use_graph=use_graph, update_prec=L.LQCD_F64_DF)
    ws = F.empty(L.lqcd_block_cg_workspace_bytes(lat, op, prm))
    L.lqcd_block_cg_solve(x, be, g64, g32, lat, op, prm, ws)
    ms, info = _events_time(lambda: L.lqcd_block_cg_solve(x, be, g64, g32, lat, op, prm, ws), stream, flush)
    return {"ms": round(ms, 3), "iterations": info.iterations, "reliable_updates": info.reliable_updates,
            "max_true_rel_residual_normal_eq": info.true_rel_residual}


def run_extras(L, F, flush, stream):
    """Domain-wall, multi-RHS, uneven-batch and force workloads, one timed run each."""
    import torch
    from synthetic import config_seed, gauge_field, gaussian_spinor
    out = {}

    out["dwf_16x4_ls16_mixed_fp32"] = dwf_bench(L, F, flush, stream)
    torch.cuda.empty_cache()

    # 32^4 with 12 right-hand sides sharing the links, m = 0.01, mixed CG per RHS to 1e-10 on
    # M_hat^dag M_hat x = b_e: FP32 inner (delta 1e-5), FP16 inner (delta 0.003), FP16 inner with
    # FP32-arithmetic replacements (three levels), block CG with FP32 inner; and the full systems
    # D x = b by the even-odd solve
    dims, nr = (32, 32, 32, 32), 12
    U = gauge_field(dims, "haar", config_seed(3, 0))
    lat = L.lattice(dims, n5=nr, bc=BC)
    op = L.operator(mass=0.01)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gsl = {1: F.gauge_to_device(U, lat, 1, 12), 2: F.gauge_to_device(U, lat, 2, 12)}
    del U
    rhs = gaussian_spinor(dims, config_seed(3, 1), lead=(nr,))
    be = F.spinor_to_device(F.checkerboard(rhs, 0), lat, 0, 0)
    bfull = F.spinor_to_device(rhs, lat, 0, 2)
    del rhs
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    DF = L.LQCD_F64_DF
    prm = {q: L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=q, sloppy_recon=12,
                              delta=DELTA_NORMAL_FP32 if q == 1 else DELTA[q], check_interval=64, update_prec=DF)
           for q in (1, 2)}
    prm[3] = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=2, sloppy_recon=12, delta=DELTA_NORMAL_FP32,
                             delta_mid=DELTA_MID, check_interval=64, update_prec=DF)
    prm[0] = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=0, sloppy_recon=18, check_interval=64)
    ws = F.empty(max(L.lqcd_cg_workspace_bytes(lat, op, prm[q], 0) for q in prm))
    vh = 32 ** 4 // 2
    mr = {}
    for q, name in ((0, "fp64"), (1, "fp32_inner"), (2, "fp16_inner"), (3, "fp16_inner_three_level")):
        g = g64 if q == 0 else gsl[prm[q].sloppy_prec]
        L.lqcd_cg_solve(x, be, g64, g, lat, op, prm[q], 0, ws)
        ms, info = _events_time(lambda: L.lqcd_cg_solve(x, be, g64, g, lat, op, prm[q], 0, ws), stream, flush)
        nop = info.iterations + info.reliable_updates + info.residual_replacements
        mr[name] = {
            "ms": round(ms, 3), "iterations": info.iterations, "reliable_updates": info.reliable_updates,
            "fp32_replacements": info.residual_replacements, "delta": prm[q].delta, "delta_mid": prm[q].delta_mid,
            "max_true_rel_residual_normal_eq": info.true_rel_residual,
            "dslash_gflops_in_solve": round(4 * nop * FLOP_PER_SITE * vh * nr / (ms * 1e-3) / 1e9, 1)}
    for name in ("fp32_inner", "fp16_inner", "fp16_inner_three_level"):
        mr["speedup_" + name + "_vs_fp64"] = round(mr["fp64"]["ms"] / mr[name]["ms"], 2)
    # the full systems D x = b of the 12 right-hand sides by lqcd_eo_solve (CGNR, tolerance on each
    # even-odd system's FP64 residual, FP16 storage with three levels)
    pe = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=2, sloppy_recon=12, delta=DELTA_3LVL,
                         delta_mid=DELTA_MID, check_interval=64, update_prec=DF)
    xf = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    wse = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, pe))
    L.lqcd_eo_solve(xf, bfull, g64, gsl[2], lat, op, pe, wse)
    mse, infe = _events_time(lambda: L.lqcd_eo_solve(xf, bfull, g64, gsl[2], lat, op, pe, wse), stream, flush)
    mr["eo_solve_full_systems_fp16_three_level"] = {
        "ms": round(mse, 3), "iterations": infe.iterations, "reliable_updates": infe.reliable_updates,
        "fp32_replacements": infe.residual_replacements, "delta": pe.delta, "delta_mid": pe.delta_mid,
        "max_true_rel_residual_full_system": infe.true_rel_residual,
        "dslash_gflops_in_solve": round((3 + 4 * (infe.iterations + infe.reliable_updates + infe.residual_replacements))
                                        * FLOP_PER_SITE * vh * nr / (mse * 1e-3) / 1e9, 1)}
    del xf, wse, bfull
    wsb = F.empty(L.lqcd_block_cg_workspace_bytes(lat, op, prm[1]))
    L.lqcd_block_cg_solve(x, be, g64, gsl[1], lat, op, prm[1], wsb)
    msb, infb = _events_time(lambda: L.lqcd_block_cg_solve(x, be, g64, gsl[1], lat, op, prm[1], wsb), stream, flush)
    mr["block_cg_fp32_inner"] = {
        "ms": round(msb, 3), "iterations": infb.iterations, "reliable_updates": infb.reliable_updates,
        "max_true_rel_residual_normal_eq": infb.true_rel_residual}
    mr["hop_f32r12_12rhs"] = _hop_gbs(L, F, lat, 1, 12, 8 * 48 / nr + 96 + 96, flush, stream)
    mr["hop_f16r12_12rhs"] = _hop_gbs(L, F, lat, 2, 12, 8 * 24 / nr + 52 + 52, flush, stream)
    mr["hop_f32r12_1rhs"] = _hop_gbs(L, F, L.lattice(dims, n5=1, bc=BC), 1, 12, 8 * 48 + 96 + 96, flush, stream)
    out["multi_rhs_32x4_12rhs_mixed"] = mr
    del g64, gsl, be, x, ws, wsb
    torch.cuda.empty_cache()

    out["gparity_16x3x32_xy_mixed_fp32"] = gparity_bench(L, F, flush, stream)
    out["su3_mul_footprint"] = su3_sweep(L, F, flush, stream)
    out["hmc_16x4"] = hmc_bench(L, F, stream)
    out["multigrid_24x3x48_m0.01"] = mg_bench(L, F, flush, stream)

    # uneven batch: 4 each of 8^4, 12^4, 16^4, 20^4, Haar links, m = 0.05, FP32-inner, one persistent launch per
    # phase, double-float reliable updates (the 16 sequential solves likewise)
    shapes = [(n_, n_, n_, n_) for n_ in (8, 12, 16, 20) for _ in range(4)]
    entries = []
    for k, dims in enumerate(shapes):
        lat = L.lattice(dims, bc=BC)
        U = gauge_field(dims, "haar", config_seed(30 + k, 0))
        bsrc = F.checkerboard(gaussian_spinor(dims, config_seed(30 + k, 1), lead=(1,)), 0)
        entries.append(dict(lat=lat, mass=0.05, gauge=F.gauge_to_device(U, lat, 0, 18),
                            gauge_sloppy=F.gauge_to_device(U, lat, 1, 12),
                            x=F.empty(L.lqcd_spinor_bytes(lat, 0, 0)), b=F.spinor_to_device(bsrc, lat, 0, 0)))
    items = L.batch_items(entries)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=1, sloppy_recon=12, delta=DELTA_NORMAL_FP32,
                          check_interval=64, update_prec=L.LQCD_F64_DF)
    wsb = F.empty(L.lqcd_batch_cg_workspace_bytes(len(entries), items, 18, prm))
    L.lqcd_batch_cg_solve(len(entries), items, 18, prm, wsb)  # tunes the tile and grid, captures the graph
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    bkey = f"sms={sms} prec=1 recon=12 : " + " ".join("x".join(map(str, d)) for d in shapes)
    ms_b, infos = _events_time(lambda: L.lqcd_batch_cg_solve(len(entries), items, 18, prm, wsb), stream, flush)
    op = L.operator(mass=0.05)
    wss = [F.empty(L.lqcd_cg_workspace_bytes(e["lat"], op, prm, 0)) for e in entries]

    def sequential():
        its = []
        for e, w in zip(entries, wss):
            its.append(L.lqcd_cg_solve(e["x"], e["b"], e["gauge"], e["gauge_sloppy"], e["lat"], op, prm, 0, w))
        return its

    sequential()
    ms_s, seq = _events_time(sequential, stream, flush)
    out["uneven_batch_4x_8_12_16_20"] = {
        "ms_persistent_batch": round(ms_b, 3), "ms_16_sequential_solves": round(ms_s, 3),
        "speedup": round(ms_s / ms_b, 2), "iterations": infos[0].iterations,
        "reliable_updates": infos[0].reliable_updates,
        "max_true_rel_residual_normal_eq": max(i.true_rel_residual for i in infos),
        "tuned_tile_sites": [64, 128, 256][L.lqcd_tune_get("batch_tile " + bkey)],
        "tuned_blocks_per_sm": L.lqcd_tune_get("batch_hop " + bkey),
        "tune_table_entries": L.lqcd_tune_entries()}
    del entries, items, wsb, wss
    torch.cuda.empty_cache()

    # force on 16^4 and 24^3 x 32: X = (M^dag M)^-1 phi (FP32-inner mixed, FP64 reliable updates), Y = M X,
    # force kernel
    for dims, key in (((16, 16, 16, 16), "force_16x4"), ((24, 24, 24, 32), "force_24x3x32")):
        U = gauge_field(dims, "haar", config_seed(4, 0))
        phi = gaussian_spinor(dims, config_seed(4, 1), lead=(1,))
        lat = L.lattice(dims, bc=BC)
        op = L.operator(mass=0.05)
        g64 = F.gauge_to_device(U, lat, 0, 18)
        g32 = F.gauge_to_device(U, lat, 1, 18)
        phid = F.spinor_to_device(phi, lat, 0, 2)
        X = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
        Y = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
        Fo = F.empty(L.lqcd_gauge_bytes(lat, 0, 18))
        prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=1, sloppy_recon=18, delta=DELTA_NORMAL_FP32,
                              check_interval=64, update_prec=L.LQCD_F64_DF)
        ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 2))

        def force_step():
            info = L.lqcd_cg_solve(X, phid, g64, g32, lat, op, prm, L.LQCD_FULL, ws)
            L.lqcd_M(Y, X, g64, lat, op, L.LQCD_FULL, 0, None)
            L.lqcd_force(Fo, g64, X, Y, lat, op, L.LQCD_FORCE_TA)
            return info

        force_step()
        ms, info = _events_time(force_step, stream, flush)
        tk, _ = _events_time(lambda: L.lqcd_force(Fo, g64, X, Y, lat, op, L.LQCD_FORCE_TA), stream, flush, reps=5)
        V = int(np.prod(dims))
        fbytes = V * (2 * 192 + 4 * 144 + 4 * 144)  # X, Y once per site, 4 links in, 4 force matrices out
        # FP64 flop per link: 4 spin projections 48, two colour outer products 288, U A - B U^dag 432,
        # boundary phase 18, traceless anti-Hermitian part 40
        fflop = V * 4 * 826
        peak, _ = measured_peak()
        out[key] = {"ms_solve_and_force": round(ms, 3), "iterations": info.iterations,
                    "reliable_updates": info.reliable_updates,
                    "force_kernel_us": round(tk * 1e3, 2), "force_kernel_bound": "alu (FP64)",
                    "force_kernel_tflops": round(fflop / (tk * 1e-3) / 1e12, 4),
                    "force_kernel_frac_of_fp64_peak": round(fflop / (tk * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                    "force_kernel_algorithmic_gbs": round(fbytes / (tk * 1e-3) / 1e9, 1),
                    "force_kernel_frac_of_measured_hbm": round(fbytes / (tk * 1e-3) / 1e9 / peak, 4)}
        del U, phi, g64, g32, phid, X, Y, Fo, ws
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ reference arm

def dwf_bench(L, F, flush, stream, use_graph=1, check_interval=64, three_level=True):
    """16^4 x L_s = 16 domain wall, M5 = 1.8, mf = 0.02, Haar links: even-odd CGNR to 1e-10 with FP32
    inner storage (delta 3e-6) and, optionally, FP16 storage with three levels, reliable updates in
    double-float arithmetic; one warm-up, one timed run (and the plain FP64 solve beside them)."""
    import torch
    from synthetic import config_seed, gauge_field, gaussian_spinor
    dims, Ls = (16, 16, 16, 16), 16
    U = gauge_field(dims, "haar", config_seed(2, 0))
    b = gaussian_spinor(dims, config_seed(2, 1), lead=(Ls,))
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=1.8, mf=0.02)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    bd = F.spinor_to_device(b, lat, 0, 2)
    del b
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=1, sloppy_recon=12, delta=DELTA[1],
                          check_interval=check_interval, use_graph=use_graph, update_prec=L.LQCD_F64_DF)
    prm3 = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=2, sloppy_recon=12, delta=DELTA_3LVL,
                           delta_mid=DELTA_MID, check_interval=check_interval, use_graph=use_graph,
                           update_prec=L.LQCD_F64_DF)
    g16 = F.gauge_to_device(U, lat, 2, 12)
    ws = F.empty(max(L.lqcd_eo_solve_workspace_bytes(lat, op, q) for q in (prm, prm3)))

    def dwf_solve(p=prm, gs=g32):
        return L.lqcd_eo_solve(x, bd, g64, gs, lat, op, p, ws)

    if three_level:
        dwf_solve(prm3, g16)
        ms3, info3 = _events_time(lambda: dwf_solve(prm3, g16), stream, flush)
        # the plain FP64 GPU solve of the same system (FP64 inner iteration)
        prm64 = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=0, sloppy_recon=18,
                                check_interval=check_interval, use_graph=use_graph)
        ws64 = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm64))
        L.lqcd_eo_solve(x, bd, g64, g64, lat, op, prm64, ws64)
        ms64, info64 = _events_time(lambda: L.lqcd_eo_solve(x, bd, g64, g64, lat, op, prm64, ws64), stream, flush)
        del ws64
    dwf_solve()
    ms, info = _events_time(dwf_solve, stream, flush)
    res = packed_full_residual(L, F, lat, op, g64, x, bd)
    hops = 1 + 2 + 4 * (info.iterations + info.reliable_updates) + 1
    return {
        "ms": round(ms, 3), "iterations": info.iterations, "reliable_updates": info.reliable_updates,
        "full_system_rel_residual": res, "reported_rel_residual_full_system": info.true_rel_residual,
        "dslash_gflops_in_solve": round(hops * FLOP_PER_SITE * 16 ** 4 // 2 * Ls / (ms * 1e-3) / 1e9, 1),
        "hop_f32r12_ls16": _hop_gbs(L, F, lat, 1, 12, 8 * 48 / Ls + 96 + 96, flush, stream, kind=L.LQCD_DWF),
        "fp16_inner_three_level": {"ms": round(ms3, 3), "iterations": info3.iterations,
                                   "reliable_updates": info3.reliable_updates,
                                   "fp32_replacements": info3.residual_replacements,
                                   "true_rel_residual_full_system": info3.true_rel_residual} if three_level else None,
        "fp64": {"ms": round(ms64, 3), "iterations": info64.iterations,
                 "true_rel_residual_full_system": info64.true_rel_residual} if three_level else None,
        "speedup_fp32_inner_vs_fp64": round(ms64 / ms, 2) if three_level else None}


def su3_sweep(L, F, flush, stream):
    """SU(3) x SU(3) field product z = x y against memory footprint (the paper's first
    benchmark): FP32 L^4 fields from L2-resident to 3.6 GB, timed back to back (warm) and,
    beyond L2, after an L2 flush (cold); FP64 at 48^4 cold. 216 B and 198 flop per FP32 site."""
    import torch
    peak, _ = measured_peak()
    rows = []
    for prec, sizes in ((1, (8, 12, 16, 24, 32, 48, 64)), (0, (48,))):
        bps = 216 if prec == 1 else 432
        for n_ in sizes:
            lat = L.lattice((n_, n_, n_, n_))
            nsites = n_ ** 4
            f = [F.empty(L.lqcd_colour_matrix_bytes(lat, prec)) for _ in range(3)]
            for t in f:
                t.zero_()
            # warm: 50 launches captured in one CUDA graph and replayed back to back, so that
            # L2-resident sizes show the GPU's time rather than the host's launch rate
            reps = 50
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(3):
                    L.lqcd_su3_mul(f[2], f[0], f[1], lat, prec)
            torch.cuda.current_stream().wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                for _ in range(reps):
                    L.lqcd_su3_mul(f[2], f[0], f[1], lat, prec)
            graph.replay()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            warm = e0.elapsed_time(e1) / reps * 1e-3
            del graph
            row = {"prec": "f32" if prec == 1 else "f64", "lattice": [n_] * 4, "sites": nsites,
                   "footprint_mb": round(bps * nsites / 1e6, 2), "warm_us": round(warm * 1e6, 2),
                   "warm_gbs": round(bps * nsites / warm / 1e9, 1),
                   "warm_gflops": round(198 * nsites / warm / 1e9, 1)}
            if bps * nsites > 256e6:
                cold, _ = _events_time(lambda: L.lqcd_su3_mul(f[2], f[0], f[1], lat, prec), stream, flush, reps=5)
                cold *= 1e-3
                row.update({"cold_us": round(cold * 1e6, 2), "cold_gbs": round(bps * nsites / cold / 1e9, 1),
                            "frac_of_measured_hbm": round(bps * nsites / cold / 1e9 / peak, 4)})
                if prec == 0:  # 198 FP64 flop per 432 B: bound by the FP64 pipe, not by HBM
                    row.update({"bound": "alu", "cold_tflops": round(198 * nsites / cold / 1e12, 4),
                                "frac_of_fp64_peak": round(198 * nsites / cold / 1e12 / FP64_PEAK_TFLOPS, 4)})
            rows.append(row)
            del f
    torch.cuda.empty_cache()
    return rows


def gparity_bench(L, F, flush, stream):
    """Even-odd Wilson CG with G-parity boundary conditions in x and y (two flavours as
    n5 = 2), 16^3 x 32, Haar links, m = 0.05, FP32 / 12-real inner, delta 1e-5, to 1e-10;
    plus the cold-L2 G-parity hop (8 links read once for both flavours)."""
    import torch
    from synthetic import config_seed, gauge_field, gaussian_spinor
    dims, m, mask = (16, 16, 16, 32), 0.05, 3
    lat = L.lattice(dims, n5=2, bc=BC)
    op = L.operator(mass=m, gparity=mask)
    U = gauge_field(dims, "haar", config_seed(60, 0))
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    bd = F.spinor_to_device(gaussian_spinor(dims, config_seed(60, 1), lead=(2,)), lat, 0, 2)
    del U
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=1, sloppy_recon=12, delta=DELTA[1], check_interval=64)
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))

    def solve():
        return L.lqcd_eo_solve(x, bd, g64, g32, lat, op, prm, ws)

    solve()
    ms, info = _events_time(solve, stream, flush)
    res = packed_full_residual(L, F, lat, op, g64, x, bd)
    vh = int(np.prod(dims)) // 2
    hops = 1 + 2 + 4 * (info.iterations + info.reliable_updates)  # the odd half reuses the last update's hop
    opg = L.operator(prec=1, recon=12, gparity=mask)
    fin = F.empty(L.lqcd_spinor_bytes(lat, 1, L.LQCD_ODD))
    fin.zero_()
    out = F.empty(L.lqcd_spinor_bytes(lat, 1, L.LQCD_EVEN))
    for _ in range(2):
        L.lqcd_dslash(out, fin, g32, lat, opg, L.LQCD_EVEN, 0)
    ts = [_events_time(lambda: L.lqcd_dslash(out, fin, g32, lat, opg, L.LQCD_EVEN, 0), stream, flush)[0]
          for _ in range(10)]
    t = float(np.mean(ts)) * 1e-3
    bps = 8 * 48 / 2 + 96 + 96
    peak, _ = measured_peak()
    return {"ms": round(ms, 3), "iterations": info.iterations, "reliable_updates": info.reliable_updates,
            "full_system_rel_residual": res,
            "dslash_gflops_in_solve": round(hops * FLOP_PER_SITE * vh * 2 / (ms * 1e-3) / 1e9, 1),
            "hop_f32r12_gparity": {"launch_us": round(t * 1e6, 2), "algorithmic_bytes_per_site": bps,
                                   "achieved_gbs": round(bps * vh * 2 / t / 1e9, 1),
                                   "frac_of_measured_hbm": round(bps * vh * 2 / t / 1e9 / peak, 4)}}


def mg_bench(L, F, flush, stream):
    """Two-level multigrid (b = 4, 12 near-null vectors, 40 set-up CG iterations each, 4 MR
    post-smoothing steps, 16 coarse CGNR iterations) on the bench field, solving the full
    D_W x = b to a 1e-10 FP64 residual: set-up and solve time, and outer iterations."""
    import torch
    from synthetic import config_seed, gauge_field, gaussian_spinor
    dims, m, nv = (24, 24, 24, 48), 0.01, 12
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    U = gauge_field(dims, "exp", config_seed(1, 0), eps=0.3)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    del U
    bd = F.spinor_to_device(gaussian_spinor(dims, config_seed(1, 1), lead=(1,)), lat, 0, 2)
    rnd = torch.cat([F.spinor_to_device(v, lat, 0, 2) for v in gaussian_spinor(dims, config_seed(70, 0), lead=(nv,))])
    mgp = L.mg_params(block=4, nvec=nv, setup_iters=40, pre_smooth=0, post_smooth=4, coarse_iters=16, restart=16)
    ws = F.empty(L.lqcd_mg_workspace_bytes(lat, op, mgp))
    setup_ms, _ = _events_time(lambda: L.lqcd_mg_setup(g64, g32, rnd, lat, op, mgp, ws), stream, flush)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    prm = L.solver_params(tol=1e-10, maxiter=500)
    L.lqcd_mg_solve(x, bd, g64, g32, lat, op, mgp, prm, ws)
    ms, info = _events_time(lambda: L.lqcd_mg_solve(x, bd, g64, g32, lat, op, mgp, prm, ws), stream, flush)
    return {"setup_ms": round(setup_ms, 1), "solve_ms": round(ms, 2), "outer_iterations": info.iterations,
            "true_rel_residual": info.true_rel_residual,
            "note": "full (not even-odd) operator; the even-odd CG of the headline needs 61 iterations here"}


def hmc_bench(L, F, stream, n_therm=12, n_meas=3):
    """HMC on 16^4: Wilson gauge action (beta 5.6) plus one Wilson pseudofermion
    (m = 0.2), minimum-norm integrator, tau = 1 in 10 steps (21 force
    evaluations), FP32-inner CG to 1e-10 on the full lattice for every force.
    Fresh Gaussian momenta and a fresh pseudofermion phi = M^dag eta before every
    trajectory (host random numbers, seeded). The start, links exp(0.3 i H), is
    far from equilibrium at beta 5.6, so n_therm trajectories are accepted
    unconditionally first; the n_meas timed trajectories then take the
    Metropolis test exp(-dH) with a seeded uniform number."""
    import torch
    from synthetic import config_seed, gauge_field, gaussian_spinor, make_rng, random_su3_algebra
    dims, beta, mass = (16, 16, 16, 16), 5.6, 0.2
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=mass)
    U = gauge_field(dims, "exp", config_seed(50, 0), eps=0.3)
    rng = make_rng(config_seed(50, 1))
    prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=1, sloppy_recon=12, delta=DELTA_NORMAL_FP32,
                          check_interval=64, update_prec=L.LQCD_F64_DF)
    hp = L.hmc_params(beta, 1.0, 10, L.LQCD_MINNORM2, 1)
    Ud = F.gauge_to_device(U, lat, 0, 18)
    Uprev = torch.empty_like(Ud)
    phid = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    ws = F.empty(L.lqcd_hmc_workspace_bytes(lat, op, prm))

    def refresh():
        P = random_su3_algebra(rng, U.size // 9).reshape(U.shape)
        eta = (rng.standard_normal(gaussian_shape) + 1j * rng.standard_normal(gaussian_shape)) / np.sqrt(2.0)
        L.lqcd_M(phid, F.spinor_to_device(eta, lat, 0, 2), Ud, lat, op, L.LQCD_FULL, 1, None)  # phi = M^dag eta
        return F.gauge_to_device(P, lat, 0, 18)

    gaussian_shape = F.host_spinor_shape(lat, L.LQCD_FULL)
    dH_therm = []
    for _ in range(n_therm):
        Pd = refresh()
        info = L.lqcd_hmc_trajectory(Ud, Pd, phid, lat, op, hp, prm, ws)
        dH_therm.append(info.H1 - info.H0)
    rows, ms_total, accepted = [], 0.0, 0
    for _ in range(n_meas):
        Pd = refresh()
        Uprev.copy_(Ud)
        ms, info = _events_time(lambda: L.lqcd_hmc_trajectory(Ud, Pd, phid, lat, op, hp, prm, ws), stream)
        dH = info.H1 - info.H0
        acc = bool(rng.uniform() < np.exp(min(0.0, -dH)))
        if not acc:
            Ud.copy_(Uprev)
        accepted += acc
        ms_total += ms
        rows.append({"ms": round(ms, 2), "dH": dH, "accepted": acc, "cg_iterations": info.cg_iterations})
    return {"ms_per_trajectory": round(ms_total / n_meas, 2), "trajectories": rows,
            "acceptance": round(accepted / n_meas, 3), "force_evaluations": info.force_evaluations,
            "thermalisation": {"trajectories": n_therm, "dH": [round(d, 2) for d in dH_therm]},
            "plaquette_action_share_last": round(info.gauge1 / info.H1, 4)}


def _oracle_schur_once(args):
    """One application of the oracle's even-odd Schur operator M_hat (two even-odd
    hops) on memory-mapped fields; returns its seconds."""
    path, mass = args
    from oracle import wilson
    U = np.load(path + ".U.npy", mmap_mode="r")
    be = np.load(path + ".be.npy", mmap_mode="r")
    t0 = time.perf_counter()
    wilson.schur(U, be, mass, BC)
    return time.perf_counter() - t0


def run_reference(args, world, rank):
    """The FP64 numpy oracle, as it stands, timed on the host cores on the same
    workload and metric. Each step is a bounded sample: every process of a spawn
    pool (one per core, fewer if the host lacks the ~3 GB of temporaries each
    needs at 24^3 x 48) applies the oracle's M_hat (two even-odd hops) once to the
    workload's fields, memory-mapped from one copy; the step time is the wall time
    of the whole pool's work, the value all processes' hop flops over it."""
    if rank != 0:
        return
    import multiprocessing as mp
    import shutil
    import tempfile
    from oracle import wilson
    dims = tuple(args.dims)
    info = host_info()
    procs = max(1, min(int(info["nproc"]), int(info.get("mem_available_gb", 3.0 * info["nproc"]) // 3.0)))
    U, b = make_inputs(dims)
    vh = int(np.prod(dims)) // 2
    tmpdir = tempfile.mkdtemp(prefix="lqcd_ref_")
    try:
        path = os.path.join(tmpdir, "fields")
        np.save(path + ".U.npy", U)
        np.save(path + ".be.npy", wilson.restrict(b[0], 0))
        del U, b
        with mp.get_context("spawn").Pool(procs) as pool:
            work = [(path, args.mass)] * procs
            for _ in range(args.warmup):
                pool.map(_oracle_schur_once, work)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                pool.map(_oracle_schur_once, work)
            dt = time.perf_counter() - t0
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)
    value = procs * 2 * args.steps * FLOP_PER_SITE * vh / dt / 1e9
    line = {"metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(dims, args.mass, world),
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": procs, "kind": "oracle",
                             "sample": f"per step one M_hat application (2 even-odd hops) of the FP64 numpy oracle "
                                       f"in each of {procs} processes (one per core), memory-mapped shared fields",
                             "host": info},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ distributed plumbing

def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(v, world):
    return _allreduce(v, world, "max")


def allreduce_sum(v, world):
    return _allreduce(v, world, "sum")


def _allreduce(v, world, op):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(local_ms, local_flop, world):
    """Whole-job figures of a replicated run: the slowest rank's time, the flops of
    all ranks, and the aggregate GFLOP/s (all ranks' work over the slowest time)."""
    max_ms = allreduce_max(local_ms, world)
    flop = allreduce_sum(local_flop, world)
    return max_ms, flop, flop / (max_ms * 1e-3) / 1e9


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    run_lqcd(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
