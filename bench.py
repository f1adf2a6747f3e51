#!/usr/bin/env python3
"""Benchmark: Wilson-AMG solves/s at 1e-10 relative error on one GB300 (and
on N GPUs as independent replicas).  A right-hand side counts as solved at a
relative residual of 3e-12, the tolerance whose solutions are within 1e-10
relative error of the exact one on this workload (measured in the same run
against a 1e-13 oracle solve: rel_err_vs_exact).

A step is one call of the solver's public entry point amg_solve on one batch
of right-hand sides: odd-even reduction, FGMRES(16) (FP64 true residual,
double-float Gram-Schmidt) preconditioned by the FP32 V(4,4) Kaczmarz AMG
cycle (tile-coloured ordering), reconstruction; the batch runs as two
concurrent lanes of 32.
The hierarchy is set up once before the timed region (the setup is cached
per gauge field); its time is reported separately.

Default workload (C4): 512x512 lattice, beta = 10 U(1) links from 500
seeded Metropolis sweeps, m at smallest |eigenvalue| 1e-3, 4 grids (4x4,
4x4, 2x2 cells), k = 12 test vectors, 64 complex Gaussian right-hand sides
per step, FP32 cycle inside FP64 FGMRES.  The plain FP64 single-RHS solve of
the same lattice is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import faulthandler
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Wilson-AMG solves/s at 1e-10 rel err (mixed+batched vs plain FP64); p99 ms"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the kernels the
# roofline reports, by (kernel, right-hand sides per launch), from one ncu capture each of the
# C4 workload (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on bench.py
# --kernel-only); None until captured for the current kernel
TRAFFIC = {("k_mdot", 64): 3228150000, ("k_kacz_tile", 32): 55593728, ("k_mdot_df", 32): 1751585024}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="C4")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--serve-configs", type=int, default=16,
                    help="resident configurations S00.. of the serving mix (16 = all five lattice sizes)")
    ap.add_argument("--serve-hbm-gb", type=float, default=160.0, help="device-memory budget of the server")
    ap.add_argument("--serving-only", action="store_true", help="run the serving leg alone (one JSON line)")
    ap.add_argument("--serve-setup-mu", default="",
                    help="override the serving mix's setup relaxations per visit, 'mu1,mu2'")
    ap.add_argument("--tol", type=float, default=3e-12,
                    help="relative residual at which a right-hand side counts as solved (3e-12 gives solutions "
                         "within 1e-10 relative error on the default workload; the line reports the error)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="timed CPU work per oracle variant (at least one solve each)")
    ap.add_argument("--nrhs", type=int, default=0, help="override the workload's RHS per step")
    ap.add_argument("--kacz-order", type=int, default=-1, help="override the Kaczmarz ordering (0 or 1)")
    ap.add_argument("--set", default="",
                    help="override integer solve parameters of the workload, 'key=value,...' (e.g. "
                         "'overlap=0,gs_arith=1')")
    ap.add_argument("--study", default="", choices=["", "rho"],
                    help="rho: Sec. 4's experiment (rho, GMRES(32) iterations, residual and error "
                         "across an eta_min sweep) instead of the benchmark; one JSON line per case")
    ap.add_argument("--kernel-only", default="",
                    choices=["", "dot", "axpy", "kacz", "tile", "dhat", "agg_tc", "agg_tc1", "agg_simt"],
                    help="set up the workload, then time one kernel family (wl_time_kernel, or agg_time_apply "
                         "for the aggregation block-stencil apply of 4x4 aggregates with k = 8) inside an NVTX "
                         "range 'cap' for profilers; prints one JSON line")
    ap.add_argument("--sweep-forms", default="",
                    help="pin the Kaczmarz launch form per level for the benchmark's batch width, "
                         "'form,param;form,param;...' from level 0 (as the JSON line's sweep_forms "
                         "reports them), so that a profiled run uses the plain run's forms")
    ap.add_argument("--study-sizes", default="128,256")
    ap.add_argument("--study-configs", type=int, default=3)
    ap.add_argument("--study-setup", default="W", choices=["W", "superV"],
                    help="setup cycles of the study: W (Sec. 4.1) or super-V (Sec. 4.2)")
    return ap.parse_args()


# ----------------------------------------------------------- oracle (CPU)
def _host_info():
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Model name", "Architecture", "Socket(s)", "Core(s) per socket"):
                info[k.strip()] = v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return info


def _oracle_leg(variant, name, hier, cyc, tol, seconds, nmax, ref_rhs, out_q):
    """Runs in a spawned process.  The oracle build `variant` ("plain": one
    thread; "omp": every host core) loads the GPU's exported hierarchy (so
    both arms solve on the same operators) and times single right-hand-side
    solves of the workload's first right-hand sides with the cycle `cyc`
    until `seconds` of solve time are spent (at least one, at most nmax).
    With ref_rhs it then solves that right-hand side to 1e-13 (untimed) as
    the reference solution the GPU's error is measured against."""
    try:
        from oracle import oracle as O
        from oracle.hierfile import read, gauge_hash
        from wl_inputs import workload, rhs_batch
        O.use_variant(variant)
        w = workload(name)
        d = read(hier)
        if d["gauge_hash"] != gauge_hash(w["U"]):
            raise ValueError("hierarchy file belongs to another gauge field")
        t0 = time.time()
        h = O.Hierarchy.from_arrays(w["N"], w["U"], d["m"], d["Nl"], d["Bl"], d["Pw"], d["As"])
        load_s = time.time() - t0
        times, iters = [], []
        for i in range(nmax):
            b = rhs_batch(w["N"], 1, 100, first=i)[0]
            t0 = time.perf_counter()
            _, info = h.solve(b, tol=tol, **cyc)
            times.append(time.perf_counter() - t0)
            iters.append(info["iters"])
            if info["status"] != 0:
                raise RuntimeError("oracle solve did not converge: %s" % info)
            if sum(times) >= seconds:
                break
        res = dict(ok=True, variant=variant, threads=O.threads(), load_s=load_s, times=times, iters=iters)
        if ref_rhs is not None:
            b = rhs_batch(w["N"], 1, 100, first=ref_rhs)[0]
            ref, info = h.solve(b, tol=1e-13, **cyc)
            res.update(ref=ref, ref_relres=info["relres"])
        out_q.put(res)
    except Exception as e:  # reported, never silently replaced
        out_q.put(dict(ok=False, variant=variant, error=repr(e)))


def _child_result(target, args, timeout):
    """Run target(*args, queue) in a spawned process and return what it put
    on the queue; a child that dies without a result is reported, not waited
    for."""
    import queue as _queue
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=target, args=args + (q,), daemon=True)
    p.start()
    t_end = time.time() + timeout
    res = None
    while res is None and time.time() < t_end:
        try:
            res = q.get(timeout=2)
        except _queue.Empty:
            if not p.is_alive():
                try:
                    res = q.get(timeout=1)
                except _queue.Empty:
                    res = dict(ok=False, error="oracle process exited with code %s" % p.exitcode)
    if res is None:
        p.terminate()
        res = dict(ok=False, error="oracle process timed out after %g s" % timeout)
    p.join(timeout=60)
    return res


def run_oracle_leg(*args, timeout=1800):
    return _child_result(_oracle_leg, args, timeout)


# ------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------- main arm
def job_throughput(units_per_rank, local_ms, world):
    """Whole-job throughput of `world` independent replicas that each
    processed `units_per_rank` units in `local_ms` milliseconds: the job time
    is the slowest rank's (MAX all-reduce on the default process group; a
    CUDA tensor under NCCL, a host tensor under gloo).  Returns (units per
    second over all ranks, job milliseconds)."""
    total = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return units_per_rank * world / (total / 1e3), total


def run_gb300(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1308_5992_gb300 import wilson_amg as W
    from wl_inputs import workload, rhs_batch

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    if w["m"] is None:
        raise SystemExit("no shift for workload %s (run oracle/make_shifts.py)" % args.workload)
    if args.kacz_order >= 0:
        w["kacz_order"] = args.kacz_order
    for kv in filter(None, args.set.split(",")):
        key, _, val = kv.partition("=")
        if key not in w:
            raise SystemExit("--set: unknown workload parameter %r" % key)
        w[key] = int(val)
    N, nrhs = w["N"], max(1, args.nrhs or w["nrhs"])
    prec = {"fp64": W.WL_FP64, "fp32": W.WL_FP32, "bf16": W.WL_FP32_BF16}[w["precision"]]

    TOL = args.tol
    op = W.wilson_create(torch.from_numpy(w["U"]).to(dev), N, w["m"])

    def params(precision, plain=False):
        # plain: the method as the paper states it (16-colour Kaczmarz, FP64 throughout)
        p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], zero_guess=1, setup_mu=w["setup_mu"],
                                 precision=precision, nu_pre=w["nu"], nu_post=w["nu"],
                                 cycle=W.WL_CYCLE_W if w["cycle"] == "W" else W.WL_CYCLE_V,
                                 fgmres_m=w["fgmres_m"], gs_passes=w["gs_passes"],
                                 kacz_order=0 if plain else w["kacz_order"],
                                 arnoldi_matvec=0 if plain else w["arnoldi_matvec"],
                                 overlap=0 if plain else w["overlap"],
                                 gs_arith=0 if plain else w["gs_arith"])
        p.levels = len(w["blocks"]) + 1
        for l, b in enumerate(w["blocks"]):
            p.block[l] = b
        return p

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    amg = W.amg_setup(op, params(prec))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    hier = os.path.join("/tmp", "wl_bench_%d_%d.wlh" % (os.getpid(), rank))
    W.amg_export(amg, hier)
    amg64 = W.amg_import(op, hier, params(W.WL_FP64, plain=True))  # same hierarchy, plain FP64 method

    b_host = torch.from_numpy(rhs_batch(N, nrhs, 100 + 1000 * rank)).pin_memory()
    b = b_host.to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def step(amg_, bb, xx, n):
        rc, info = W.amg_solve(amg_, bb, xx, n, TOL)
        if rc != W.WL_OK:
            raise RuntimeError("solve did not converge: %s" % info)
        return info

    # right-hand sides per solve lane: with overlap the batch runs as two concurrent halves,
    # so every kernel of the step is launched at that width
    lane = (nrhs + 1) // 2 if w["overlap"] and nrhs >= 32 else nrhs
    pin_sweep_forms(W, amg, args.sweep_forms, lane, prec)
    for _ in range(args.warmup):
        step(amg, b, x, nrhs)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = W.wl_launch_count()
    times, infos = [], []
    barrier()
    # profilers select the timed steps by this range: a start/end range, which (unlike a push/pop
    # range) covers the kernels every host thread launches, the second solve lane's included
    timed_range = torch.cuda.nvtx.range_start("timed")
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        infos.append(step(amg, b, x, nrhs))
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_end(timed_range)
    barrier()
    launches = W.wl_launch_count() - launches0
    clk = clocks.stop()
    value, total_ms = job_throughput(nrhs * args.steps, sum(times), world)
    iters = [i["iters"] for inf in infos for i in inf]
    relres = max(i["true_relres"] for inf in infos for i in inf)

    # e2e: the public call with host buffers (pinned): amg_solve_host copies b in and x out
    # inside the timed region of every step (one solve lane's copies beside the other
    # lane's solve); warm-up steps as for the device-timed loop
    x_host = torch.empty_like(b_host).pin_memory()
    e2e_ms = []
    for it in range(args.warmup + max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc, _ = W.amg_solve_host(amg, b_host, x_host, nrhs, TOL)
        e1.record()
        torch.cuda.synchronize()
        if rc != W.WL_OK:
            raise RuntimeError("host-buffer solve did not converge")
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    bd = torch.empty_like(b)
    e2e_value, _ = job_throughput(nrhs * len(e2e_ms), sum(e2e_ms), world)
    # the copies alone (CUDA events around each), to split the e2e time
    h2d_ms, d2h_ms = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        bd.copy_(b_host, non_blocking=True)
        e1.record()
        x_host.copy_(bd, non_blocking=True)
        e2.record()
        torch.cuda.synchronize()
        h2d_ms.append(e0.elapsed_time(e1))
        d2h_ms.append(e1.elapsed_time(e2))
    e2e = {"value": e2e_value, "unit": "solves/s", "call": "amg_solve_host (pinned host b and x)",
           "h2d_bytes_per_step": b_host.numel() * 16, "d2h_bytes_per_step": x_host.numel() * 16,
           "h2d_ms_alone": round(min(h2d_ms), 3), "d2h_ms_alone": round(min(d2h_ms), 3)}

    # The same step with the Gram-Schmidt in FP64 instead of double-float (the precision
    # split that keeps FP64 there), on the same hierarchy, timed the same way
    gs64 = None
    if w["gs_arith"]:
        p_gs = params(prec)
        p_gs.gs_arith = 0
        amg_gs = W.amg_import(op, hier, p_gs)
        pin_sweep_forms(W, amg_gs, args.sweep_forms, lane, prec)
        for _ in range(args.warmup):
            step(amg_gs, b, x, nrhs)
        t_gs, it_gs = [], []
        for _ in range(max(1, min(args.steps, 5))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            inf = step(amg_gs, b, x, nrhs)
            e1.record()
            torch.cuda.synchronize()
            t_gs.append(e0.elapsed_time(e1))
            it_gs += [i["iters"] for i in inf]
        gs64 = {"value": round(nrhs * len(t_gs) / (sum(t_gs) * 1e-3), 3), "unit": "solves/s",
                "ms_per_step": round(sum(t_gs) / len(t_gs), 3), "iters_mean": round(sum(it_gs) / len(it_gs), 2),
                "what": "the same step with FP64 Gram-Schmidt (gs_arith = 0), same hierarchy and lanes"}
        W.amg_destroy(amg_gs)

    # plain FP64 single-RHS solve of the same lattice (the method's baseline)
    b1, x1 = b[:1].contiguous(), torch.zeros_like(b[:1])
    for _ in range(2):
        step(amg64, b1, x1, 1)
    p64 = []
    for _ in range(3):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        inf64 = step(amg64, b1, x1, 1)
        e1.record()
        torch.cuda.synchronize()
        p64.append(e0.elapsed_time(e1))

    # Roofline.  The ncu launch list of this workload ranks the tile-coloured Kaczmarz
    # kernel first (28 % of kernel time on level 0, 37 % over levels 0 and 1), then the
    # FP64 Gram-Schmidt update k_maxpy and the multi-dots k_mdot; with the 16-colour
    # ordering k_mdot and the colour passes lead.
    # Every kernel is timed at the width the timed step launches it (lane right-hand sides).
    n0 = N * N // 2
    E = 2 * n0 * lane
    hbm, src = peaks()
    eb = 16 if prec == W.WL_FP64 else 8          # bytes of one complex value of the cycle
    sb = 16 if prec == W.WL_FP64 else (8 if prec == W.WL_FP32 else 4)  # stencil storage
    # k_mdot: FP64-ALU bound, peak derived from the unit counts (152 SMs x 2 FP64 FMA per
    # clock x 2 flop x 2070 MHz = 1259 GFLOP/s); one launch computes kc = 11 conjugate dot
    # products of length E = 2 n0 nrhs complex numbers, 8 flop per complex term
    kc = 11
    dot_ms = W.wl_time_kernel(amg, W.WL_K_GS_DOT, 0, lane, prec, 20)
    fp64_peak = 152 * 2 * 2 * 2070e6 / 1e9
    dot_gflops = 8.0 * kc * E / (dot_ms * 1e-3) / 1e9
    # the derived peak checked in this run: the library's FP64 FMA probe (8 blocks of 256
    # threads per SM, 8 independent chains of 4096 FMAs per thread)
    fma_ms = W.wl_time_kernel(amg, W.WL_K_FP64_FMA, 0, lane, prec, 5)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fma_gflops = nsm * 8 * 256 * 8 * 4096 * 2 / (fma_ms * 1e-3) / 1e9
    if w["gs_arith"]:
        # double-float Gram-Schmidt on the FP32 pipes: bound by HBM; the 11 dots run as two
        # launches (at most 8 per launch), each reading w once: (11 + 2) vectors of E complex
        # double-floats (16 B)
        nl = -(-kc // 8)
        dot_bytes = (kc + nl) * E * 16
        ach = dot_bytes / (dot_ms * 1e-3) / 1e9
        roof_dot = {"kernel": "k_mdot_df (double-float Gram-Schmidt, 11 dots in %d launches)" % nl, "bound": "hbm",
                    "achieved": round(ach, 1), "peak": hbm, "peak_source": src, "unit": "GB/s",
                    "frac": round(ach / hbm, 4), "traffic": TRAFFIC.get(("k_mdot_df", lane)),
                    "avg_launch_ms": round(dot_ms, 4), "algorithmic_bytes": int(dot_bytes),
                    "fp64_equivalent_gflops": round(dot_gflops, 1), "fp64_fma_probe_gflops": round(fma_gflops, 1)}
    else:
        roof_dot = {"kernel": "k_mdot<double> (Gram-Schmidt, 11 dots)", "bound": "alu",
                    "achieved": round(dot_gflops, 1), "peak": round(fp64_peak, 1),
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
                    "fp64_fma_probe_gflops": round(fma_gflops, 1), "frac_of_probe": round(dot_gflops / fma_gflops, 4),
                    "unit": "GFLOP/s", "frac": round(dot_gflops / fp64_peak, 4),
                    "traffic": TRAFFIC.get(("k_mdot", lane)), "avg_launch_ms": round(dot_ms, 4),
                    "algorithmic_flops": int(8 * kc * E)}
    # k_kacz: one colour pass (1/16 of the sites): r read and written on 9/16 of the sites,
    # x on 1/16, stencil rows and denominators of 1/16 of the sites (each operand once)
    kacz_ms = W.wl_time_kernel(amg, W.WL_K_KACZ, 0, lane, prec, 160)
    kacz_bytes = n0 * lane * (9 / 16 * 2 * 2 * eb + 1 / 16 * 2 * 2 * eb) + n0 / 16 * (36 * sb + 2 * (eb // 2))
    achieved = kacz_bytes / (kacz_ms * 1e-3) / 1e9
    roof_kacz = {"kernel": "k_kacz (fine level, one of 16 colour passes)", "bound": "hbm",
                 "achieved": round(achieved, 1), "peak": hbm, "peak_source": src, "unit": "GB/s",
                 "frac": round(achieved / hbm, 4), "traffic": None, "avg_launch_ms": round(kacz_ms, 5),
                 "algorithmic_bytes": int(kacz_bytes)}
    # k_kacz_tile: one tile colour (1/4 of the sites, a quarter of a sweep).  Algorithmic
    # bytes per even site and right-hand side of one Kaczmarz pass: r and x read and
    # written once (4 x 2 spins x 8 B = 64 B in FP32), plus the site's links and column
    # norms (40 B) shared by the right-hand sides; the kernel itself reads the explicit
    # 9-point stencil row (288 B) in place of the links, so its own count is higher
    def roof_tile_at(width):  # at a width the step runs, so with the launch form it tuned or pinned
        ms = W.wl_time_kernel(amg, W.WL_K_KACZ_TILE, 0, width, prec, 80)
        tb = n0 / 4 * (width * 2 * 2 * eb * 2 + 40 * (eb // 8))
        tbs = n0 / 4 * (width * 2 * 2 * eb * 2 + 36 * sb + 2 * (eb // 2))
        ach = tb / (ms * 1e-3) / 1e9
        return {"kernel": "k_kacz_tile (fine level, one of 4 tile colours), %d RHS" % width, "bound": "hbm",
                "achieved": round(ach, 1), "peak": hbm, "peak_source": src, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": TRAFFIC.get(("k_kacz_tile", width)),
                "avg_launch_ms": round(ms, 5), "algorithmic_bytes": int(tb), "nrhs": width,
                "bytes_per_site_per_rhs": 64, "bytes_per_site": 40,
                "achieved_with_stencil_rows": round(tbs / (ms * 1e-3) / 1e9, 1)}
    roof_tile = roof_tile_at(lane)
    # k_stencil on level 0 (residual f - A x with the 9-point Dhat stencil; the same gather
    # computes the FP32 Arnoldi matvec): x read once (its 9 neighbours come from cache), f
    # read, y written, the stencil row (36 complex) read once per site
    st_ms = W.wl_time_kernel(amg, W.WL_K_STENCIL, 0, lane, prec, 40)
    st_bytes = n0 * (lane * 2 * 3 * eb + 36 * sb)
    achieved = st_bytes / (st_ms * 1e-3) / 1e9
    roof_st = {"kernel": "k_stencil (fine level, residual f - Dhat x)", "bound": "hbm",
               "achieved": round(achieved, 1), "peak": hbm, "peak_source": src, "unit": "GB/s",
               "frac": round(achieved / hbm, 4), "traffic": None, "avg_launch_ms": round(st_ms, 5),
               "algorithmic_bytes": int(st_bytes)}
    if w["kacz_order"] == 1:
        roof, roof_more = roof_tile, [roof_dot, roof_kacz, roof_st]
    else:
        roof, roof_more = roof_dot, [roof_kacz, roof_tile, roof_st]

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64" if prec == W.WL_FP64 else
                  "f32 cycle + f32-pair (double-float) Gram-Schmidt + f64 Hessenberg and true residual"
                  if w["gs_arith"] else "f32 cycle + f64 Krylov"),
        "data": "synthetic (seeded U(1) Metropolis gauge, complex Gaussian right-hand sides)",
        "config": {"workload": "%s: %dx%d lattice, beta=%g, %d Metropolis sweeps, m=%.6f (smallest |eig| %g), "
                               "%d grids, blocks %s, k=%d, setup relaxations %s, %d RHS/step, %s(%d,%d) %s "
                               "Kaczmarz cycle in %s, FGMRES(%d) with %d Gram-Schmidt pass(es) in %s, Arnoldi "
                               "matvec %s, FP64 true residual at restarts, relative residual %g (error vs exact "
                               "in rel_err_vs_exact), %s"
                               % (args.workload, N, N, w["beta"], w["sweeps"], w["m"], w["target"],
                                  len(w["blocks"]) + 1, w["blocks"], w["k"], list(w["setup_mu"]), nrhs, w["cycle"],
                                  w["nu"], w["nu"], ["16-colour", "tile-coloured (8x8 tiles)"][w["kacz_order"]],
                                  ["fp64", "fp32", "fp32+bf16-storage"][prec], w["fgmres_m"], w["gs_passes"],
                                  "double-float" if w["gs_arith"] else "FP64",
                                  "fp32" if w["arnoldi_matvec"] and prec != W.WL_FP64 else "fp64", TOL,
                                  "two concurrent solve lanes of %d RHS" % lane if lane < nrhs else "one solve lane"),
                   "tol": TOL, "rhs_per_lane": lane,
                   "nrhs": nrhs, "L": N, "precision": ["fp64", "fp32", "fp32_bf16"][prec],
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": "replicas"},
        "iters_mean": round(sum(iters) / len(iters), 2), "iters_max": max(iters),
        "true_relres_max": relres, "setup_s": round(setup_s, 3),
        "step_ms_p50": sorted(times)[len(times) // 2], "step_ms_p99": sorted(times)[min(len(times) - 1,
                                                                                         int(0.99 * len(times)))],
        "gram_schmidt_fp64": gs64,
        "plain_fp64_single_rhs": {"value": round(1e3 / (sorted(p64)[1]), 3), "unit": "solves/s",
                                  "ms": sorted(p64)[1], "iters": inf64[0]["iters"]},
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "roofline_more": roof_more, "clocks": clk,
        "sweep_forms": [list(W.amg_sweep_form(amg, l, lane, prec)) for l in range(len(w["blocks"]))],
    }
    # The other single-configuration workloads, beside the headline: C3 (this lattice, one
    # right-hand side, the same FP32 cycle on the same hierarchy) and C2 (128x128, the plain
    # FP64 method with one right-hand side: the plain-method GPU baseline); solves/s at the
    # same tolerance, each solve timed with CUDA events after warm-up
    if args.workload == "C4" and rank == 0:
        def time_solves(amg_, bb, reps):
            xx = torch.zeros_like(bb)
            for _ in range(2):
                step(amg_, bb, xx, 1)
            ts, its = [], []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                inf = step(amg_, bb, xx, 1)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                its.append(inf[0]["iters"])
            ts.sort()
            return {"value": round(1e3 / ts[len(ts) // 2], 3), "unit": "solves/s", "ms_p50": round(ts[len(ts) // 2], 3),
                    "iters": its[0]}
        extra = {"C3": dict(time_solves(amg, b[:1].contiguous(), 5),
                            workload="512x512, 1 RHS, FP32 V(4,4) tile-coloured cycle in FGMRES(16) with "
                                     "%s Gram-Schmidt, the C4 hierarchy"
                                     % ("double-float" if w["gs_arith"] else "FP64"))}
        try:
            w2 = workload("C2")
            op2 = W.wilson_create(torch.from_numpy(w2["U"]).to(dev), w2["N"], w2["m"])
            p2 = W.amg_params_default(k_r=w2["k"], k_e=w2["k"], seed=w2["seed"], zero_guess=1, precision=W.WL_FP64)
            p2.levels = len(w2["blocks"]) + 1
            for l, bk in enumerate(w2["blocks"]):
                p2.block[l] = bk
            amg2 = W.amg_setup(op2, p2)
            b2 = torch.from_numpy(rhs_batch(w2["N"], 1, 100)).to(dev)
            extra["C2"] = dict(time_solves(amg2, b2, 10),
                               workload="128x128, beta=6, smallest |eig| 1e-3, 3 grids (4x4, 2x2), k=8, FP64 "
                                        "V(2,2) 16-colour cycle, FGMRES(20) with two Gram-Schmidt passes, 1 RHS")
            amg2.close()
            op2.close()
        except Exception as e:  # reported, never silently replaced
            extra["C2"] = {"error": repr(e)}
        out["other_workloads"] = extra

    # Aggregation coarse space (Sec. 4's "more interpolation variables per coarse point"):
    # the 9-point stencil of 16 x 16 blocks of 4 x 4 aggregates with k = 8 spin-split test
    # vectors of this lattice (8192 coarse sites), applied to this batch's 64 right-hand
    # sides on CUDA cores (FP32) and on the tensor cores (tcgen05: TF32 operands split
    # into high and low parts, FP32 accuracy; and the single-term TF32 form)
    if nrhs >= 16 and N % 8 == 0:
        try:
            from wl_inputs import cgauss
            V = torch.from_numpy(np.stack([cgauss(92, j, N * N) for j in range(8)])).to(dev)
            g = W.agg_create(amg, 0, 4, 8, V)
            del V
            ca = {"operator": "4x4 aggregates, k = 8 (16 x 16 complex blocks, 9-point stencil), %d coarse sites, "
                              "%d right-hand sides" % (g.nc, nrhs)}
            flops = 8.0 * g.nc * nrhs * 9 * 256
            byts = g.nc * (9 * 256 * 8 + 2 * nrhs * 16 * 8)
            for name, kern in (("cuda_cores_fp32", W.WL_AGG_FP32), ("tensor_cores_3xtf32", W.WL_AGG_TC),
                               ("tensor_cores_tf32", W.WL_AGG_TC1)):
                ms = W.agg_time_apply(g, nrhs, kern, 20)
                ca[name] = {"ms": round(ms, 4), "tflops": round(flops / (ms * 1e-3) / 1e12, 2),
                            "gbs": round(byts / (ms * 1e-3) / 1e9, 1), "frac_hbm": round(byts / (ms * 1e-3) / 1e9 / hbm, 4)}
            ca["algorithmic"] = {"flops": int(flops), "bytes": int(byts)}
            g.close()
            out["coarse_apply"] = ca
        except Exception as e:  # reported, never silently replaced
            out["coarse_apply"] = {"error": repr(e)}

    # CPU baseline: the oracle on the host cores, after the GPU's timed region (nothing else
    # runs meanwhile), on the GPU's exported hierarchy; two builds: one thread with the
    # lexicographic Kaczmarz ordering, and every core with the 16-colour ordering.  The
    # all-cores run also solves the batch's first right-hand side to 1e-13, the reference
    # the GPU solution's error is measured against.
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        cyc = dict(m=w["fgmres_m"], nu1=w["nu"], nu2=w["nu"], gamma=2 if w["cycle"] == "W" else 1,
                   gs_passes=w["gs_passes"])
        legs = [run_oracle_leg("plain", args.workload, hier, dict(cyc, order=O.ORDER_LEX), TOL, args.cpu_seconds,
                               3, None),
                run_oracle_leg("omp", args.workload, hier, dict(cyc, order=O.ORDER_COLOUR), TOL, args.cpu_seconds,
                               8, 0)]
        variants = []
        for res in legs:
            if not res.get("ok"):
                variants.append({"variant": res.get("variant"), "error": res.get("error")})
                continue
            ts = res["times"]
            variants.append({"variant": res["variant"], "value": round(len(ts) / sum(ts), 4), "unit": "solves/s",
                             "cores": res["threads"],
                             "order": "lexicographic" if res["variant"] == "plain" else "16-colour",
                             "solves": len(ts), "seconds": round(sum(ts), 2), "iters": res["iters"]})
        best = max((v for v in variants if "value" in v), key=lambda v: v["value"], default=None)
        out["cpu_baseline"] = {
            "value": best["value"] if best else None, "unit": "solves/s", "cores": best["cores"] if best else None,
            "kind": "oracle",
            "sample": "single-RHS solves of the workload's first right-hand sides on the GPU's exported "
                      "hierarchy, %s(%d,%d) cycle, FGMRES(%d) with %d Gram-Schmidt pass(es), tol %g, about %g s "
                      "of solve time per build, run after the GPU's timed region"
                      % (w["cycle"], w["nu"], w["nu"], w["fgmres_m"], w["gs_passes"], TOL, args.cpu_seconds),
            "variants": variants, "host": _host_info()}
        omp = legs[1]
        if omp.get("ok"):
            one = torch.zeros_like(b[:1])
            step(amg, b[:1].contiguous(), one, 1)
            got = one[0].cpu().numpy()
            ref = omp["ref"]
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            out["rel_err_vs_exact"] = {
                "value": err, "max_elementwise": float(np.abs(got - ref).max() / np.abs(ref).max()),
                "tol": TOL, "reference": "oracle FP64 solve of the batch's first right-hand side to a relative "
                                         "residual of %.1e on the same hierarchy" % omp["ref_relres"],
                "meets_1e-10": err <= 1e-10}
    os.remove(hier)
    if not args.no_serving:
        out["serving"] = run_serving(args, rank, dev, W, torch)
    return out


def _cache_gauge(name):
    from wl_inputs import workload
    workload(name)
    return name


def run_serving(args, rank, dev, W, torch):
    """Continuous-batching serving over resident hierarchies of several lattice
    sizes: a closed-loop burst measures capacity, then a seeded Poisson stream
    of 1-32 RHS requests arrives at 70% of it for --serve-seconds."""
    import numpy as np
    from wl_inputs import workload, rhs_batch, uniform01
    # S00..S15 cycle over 64, 128, 256, 512, 1024 lattices, beta 6/10, targets 1e-2/1e-3
    names = ["S%02d" % i for i in range(args.serve_configs)]
    # generate (and cache) the gauge fields in parallel host processes; spawn,
    # since this process already holds a CUDA context
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(len(names), os.cpu_count() or 1))) as pool:
        pool.map(_cache_gauge, names)
    srv = W.srv_create(int(args.serve_hbm_gb * (1 << 30)), 32)
    cfgs, pools = [], []
    for nm in names:
        w = workload(nm)
        if w["m"] is None:
            return {"unavailable": "no shift for %s" % nm}
        op = W.wilson_create(torch.from_numpy(w["U"]).to(dev), w["N"], w["m"])
        mu = tuple(int(v) for v in args.serve_setup_mu.split(",")) if args.serve_setup_mu else w["setup_mu"]
        p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], precision=W.WL_FP32, gs_passes=1,
                                 nu_pre=4, nu_post=4, kacz_order=1, arnoldi_matvec=1, setup_mu=mu, gs_arith=1,
                                 fgmres_m=16)
        p.levels = len(w["blocks"]) + 1
        for l, b in enumerate(w["blocks"]):
            p.block[l] = b
        amg = W.amg_setup(op, p)
        cfgs.append((nm, w, W.srv_add(srv, amg)))
        pools.append(torch.from_numpy(rhs_batch(w["N"], 32, 7000 + len(pools))).to(dev))
    slots, reserved = [], 0
    for _, _, cid in cfgs:
        n_, b_ = W.srv_info(srv, cid)
        slots.append(n_)
        reserved += b_
    W.srv_start(srv)
    seed = 9000 + rank

    def requests(n, stream):
        u = uniform01(seed, stream, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
        return [(int(u[i, 0] * len(cfgs)), 1 + int(u[i, 1] * 32), u[i, 2]) for i in range(n)]

    def submit(c, nr):
        nm, w, cid = cfgs[c]
        b = pools[c][:nr].contiguous()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        return W.srv_submit(srv, cid, b, x, nr, args.tol), nr, x

    # capacity: a closed-loop burst
    burst = requests(16, 1)
    t0 = time.perf_counter()
    live = [submit(c, nr) for c, nr, _ in burst]
    W.srv_drain(srv)
    cap = sum(nr for _, nr, _ in live) / (time.perf_counter() - t0)
    # open loop: Poisson arrivals at 70% of capacity (in right-hand sides per second)
    mean_rhs = 16.5
    rate = 0.7 * cap / mean_rhs
    n = max(8, int(rate * args.serve_seconds))
    reqs = requests(n, 2)
    live, t = [], time.perf_counter()
    tstart = t
    for c, nr, u in reqs:
        t += -np.log(max(u, 1e-12)) / rate
        dt = t - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        live.append(submit(c, nr))
    W.srv_drain(srv)
    wall = time.perf_counter() - tstart
    lats, solved, worst = [], 0, 0.0
    its = {}
    for (rid, nr, x), (c, _, _) in zip(live, reqs):
        done, info, lat = W.srv_poll(srv, rid, nr)
        lats.append(lat)
        solved += nr
        worst = max([worst] + [i["true_relres"] for i in info])
        its.setdefault(cfgs[c][0], []).extend(i["iters"] for i in info)
    lats.sort()
    srv.close()
    return {"configs": ["%s:%dx%d" % (nm, w["N"], w["N"]) for nm, w, _ in cfgs], "requests": len(lats),
            "rhs_per_request": "uniform 1..32", "arrival": "Poisson, seeded, %.2f req/s (70%% of %.1f solves/s "
            "closed-loop capacity)" % (rate, cap), "p50_ms": round(lats[len(lats) // 2], 2),
            "p99_ms": round(lats[min(len(lats) - 1, int(0.99 * len(lats)))], 2),
            "solves_per_s": round(solved / wall, 2), "true_relres_max": worst,
            "cycle": "V(4,4) FP32 tile-coloured Kaczmarz, FGMRES(16) (FP32 Arnoldi matvec, one double-float "
                     "Gram-Schmidt pass, FP64 true residual)", "slots_per_config": slots,
            "hbm_budget_gb": args.serve_hbm_gb, "hbm_reserved_gb": round(reserved / (1 << 30), 2),
            "setup_mu": list(mu), "tol": args.tol,
            "mean_iters_by_config": {k: round(sum(v) / len(v), 1) for k, v in sorted(its.items())}}


def _reference_leg(name, nsolves, tol, out_q):
    """Runs in a spawned process: the all-cores oracle build, its own setup of
    the workload (untimed), then `nsolves` timed single right-hand-side
    solves with the GPU arm's cycle (V(nu,nu), FGMRES(m), Gram-Schmidt passes)
    and the 16-colour Kaczmarz ordering."""
    try:
        from oracle import oracle as O
        from wl_inputs import workload, rhs_batch
        O.use_variant("omp")
        w = workload(name)
        p = O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"], seed=w["seed"], mu1=w["setup_mu"][0],
                           mu2=w["setup_mu"][1])
        t0 = time.time()
        h = O.Hierarchy.setup(w["N"], w["U"], w["m"], p)
        setup_s = time.time() - t0
        times, iters = [], []
        for i in range(nsolves):
            b = rhs_batch(w["N"], 1, 100, first=i)[0]
            t0 = time.perf_counter()
            _, info = h.solve(b, tol=tol, m=w["fgmres_m"], nu1=w["nu"], nu2=w["nu"],
                              gamma=2 if w["cycle"] == "W" else 1, order=O.ORDER_COLOUR, gs_passes=w["gs_passes"])
            times.append(time.perf_counter() - t0)
            iters.append(info["iters"])
        out_q.put(dict(ok=True, setup_s=setup_s, times=times, iters=iters, threads=O.threads()))
    except Exception as e:  # reported, never silently replaced
        out_q.put(dict(ok=False, error=repr(e)))


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, same metric and workload."""
    if rank != 0:
        return None
    from wl_inputs import workload
    w = workload(args.workload, with_gauge=False)
    res = _child_result(_reference_leg, (args.workload, args.warmup + args.steps, args.tol), 3600)
    if not res.get("ok"):
        return {"impl": "reference", "unavailable": "oracle failed: %s" % res.get("error")}
    ts = res["times"][args.warmup:]
    value = len(ts) / sum(ts)
    sample = ("one single-RHS solve per step, %d threads (oracle setup untimed: %.1f s); iterations %s"
              % (res["threads"], res["setup_s"], res["iters"][args.warmup:]))
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(ts) / len(ts), 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s: %dx%d lattice, beta=%g, %d Metropolis sweeps, m=%.6f (smallest |eig| %g), "
                                   "%d grids, blocks %s, k=%d, 1 RHS per solve (the first right-hand sides of the "
                                   "GPU arm's batch), FP64 CPU oracle on every host core: %s(%d,%d) 16-colour "
                                   "Kaczmarz cycle, FGMRES(%d) with %d Gram-Schmidt pass(es), tol %g"
                                   % (args.workload, w["N"], w["N"], w["beta"], w["sweeps"], w["m"], w["target"],
                                      len(w["blocks"]) + 1, w["blocks"], w["k"], w["cycle"], w["nu"], w["nu"],
                                      w["fgmres_m"], w["gs_passes"], args.tol),
                       "name": args.workload, "L": w["N"], "nrhs_per_step": 1},
            "cpu_baseline": {"value": round(value, 4), "unit": "solves/s", "cores": res["threads"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def pin_sweep_forms(W, amg, spec, nrhs, prec):
    """Apply --sweep-forms ('form,param;...' from level 0) before the first cycle."""
    for level, item in enumerate(v for v in spec.split(";") if v):
        form, param = (int(t) for t in item.split(","))
        W.amg_pin_sweep_form(amg, level, nrhs, prec, form, param)


def run_kernel_only(args):
    """Set up the workload's hierarchy, run one cycle of the batch width (so
    the autotuner has chosen its launch forms) and time one kernel family on
    level 0 (three warm-up launches, then two inside the NVTX range 'cap').
    agg_*: the aggregation block-stencil apply of the fine level (4x4
    aggregates, k = 8 random test vectors) on the tensor cores (agg_tc: FP32
    accurate, agg_tc1: TF32) or on CUDA cores (agg_simt)."""
    import torch
    from paper_1308_5992_gb300 import wilson_amg as W
    from wl_inputs import workload
    w = workload(args.workload)
    if args.kernel_only.startswith("agg"):
        import numpy as np
        from wl_inputs import cgauss
        dev = torch.device("cuda", 0)
        N, nrhs = w["N"], max(1, args.nrhs or w["nrhs"])
        op = W.wilson_create(torch.from_numpy(w["U"]).to(dev), N, w["m"])
        p = W.amg_params_default(k_r=4, k_e=4, seed=1, setup_mu=(2, 1))
        p.levels = len(w["blocks"]) + 1
        for l, b in enumerate(w["blocks"]):
            p.block[l] = b
        amg = W.amg_setup(op, p)
        g = W.agg_create(amg, 0, 4, 8, torch.from_numpy(np.stack([cgauss(92, j, N * N) for j in range(8)])).to(dev))
        kern = {"agg_tc": W.WL_AGG_TC, "agg_tc1": W.WL_AGG_TC1, "agg_simt": W.WL_AGG_FP32}[args.kernel_only]
        W.agg_time_apply(g, nrhs, kern, 3)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("cap")
        ms = W.agg_time_apply(g, nrhs, kern, 2)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"kernel_only": args.kernel_only, "workload": args.workload, "nrhs": nrhs,
                          "coarse_sites": g.nc, "avg_launch_ms": ms}))
        return
    if args.kacz_order >= 0:
        w["kacz_order"] = args.kacz_order
    for kv in filter(None, args.set.split(",")):
        key, _, val = kv.partition("=")
        if key not in w:
            raise SystemExit("--set: unknown workload parameter %r" % key)
        w[key] = int(val)
    dev = torch.device("cuda", 0)
    N, nrhs = w["N"], max(1, args.nrhs or w["nrhs"])
    prec = {"fp64": W.WL_FP64, "fp32": W.WL_FP32, "bf16": W.WL_FP32_BF16}[w["precision"]]
    kind = {"dot": W.WL_K_GS_DOT, "axpy": W.WL_K_GS_AXPY, "kacz": W.WL_K_KACZ, "tile": W.WL_K_KACZ_TILE,
            "dhat": W.WL_K_DHAT}[args.kernel_only]
    op = W.wilson_create(torch.from_numpy(w["U"]).to(dev), N, w["m"])
    p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], zero_guess=1, precision=prec,
                             kacz_order=w["kacz_order"], arnoldi_matvec=w["arnoldi_matvec"],
                             gs_arith=w["gs_arith"])
    p.levels = len(w["blocks"]) + 1
    for l, b in enumerate(w["blocks"]):
        p.block[l] = b
    amg = W.amg_setup(op, p)
    pin_sweep_forms(W, amg, args.sweep_forms, nrhs, prec)
    f = torch.ones((nrhs, N * N), dtype=torch.complex128, device=dev)
    W.amg_cycle(amg, f, torch.zeros_like(f), nrhs, prec)  # runs the autotuner for this width
    W.wl_time_kernel(amg, kind, 0, nrhs, prec, 3)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("cap")
    ms = W.wl_time_kernel(amg, kind, 0, nrhs, prec, 2)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"kernel_only": args.kernel_only, "workload": args.workload, "nrhs": nrhs,
                      "avg_launch_ms": ms, "level0_sweep_form": list(W.amg_sweep_form(amg, 0, nrhs, prec))}))


def run_study_rho(args):
    """Sec. 4's experiment on seeded stand-ins for its gauge ensembles:
    N = 128 / 256, beta = 3 / 6 / 10, up to three configurations each, 2x2
    cells down to N = 16, k_r = k_e = 8, setup mu = 10 / 5 with the W(4,4)
    adaptive step, FP64 W(4,4) solve cycle.  For every eta_min(D) of the
    sweep: rho of the stand-alone cycle (to 1e-8 or 100 iterations), the
    GMRES(32) iterations to a 1e-8 relative residual, that residual, and the
    relative error against a 1e-13 solve of the same hierarchy."""
    import numpy as np
    import torch
    from paper_1308_5992_gb300 import wilson_amg as W
    from wl_inputs import workload, rhs_batch, cgauss
    from wl_inputs.workloads import WORKLOADS, PAPER_ETAS
    dev = torch.device("cuda", 0)
    sizes = [int(v) for v in args.study_sizes.split(",") if v]
    rows = []
    for name, spec in WORKLOADS.items():
        if not spec.get("eta_sweep") or spec["N"] not in sizes or int(name[-1]) >= args.study_configs:
            continue
        w0 = workload(name)
        if w0["eta0"] is None:
            print(json.dumps({"study": "rho", "workload": name, "unavailable": "no eta0 in shifts.json"}))
            continue
        Ud = torch.from_numpy(w0["U"]).to(dev)
        N = w0["N"]
        n = N * N  # level-0 unknowns (N^2 / 2 sites, 2 spins)
        for eta in PAPER_ETAS:
            w = workload(name, with_gauge=False, eta=eta)
            op = W.wilson_create(Ud, N, w["m"])
            p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], zero_guess=1, precision=W.WL_FP64,
                                     nu_pre=4, nu_post=4, cycle=W.WL_CYCLE_W, fgmres_m=32, max_restarts=20,
                                     setup_cycle=1 if args.study_setup == "superV" else 0)
            p.levels = len(w["blocks"]) + 1
            for l, b in enumerate(w["blocks"]):
                p.block[l] = b
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                amg = W.amg_setup(op, p)
            except W.WilsonAMGError as e:
                print(json.dumps({"study": "rho", "workload": name, "eta": eta, "error": str(e)}), flush=True)
                op.close()
                continue
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
            x0 = torch.from_numpy(cgauss(w["seed"], 77, n)[None, :]).to(dev)
            xe = torch.zeros_like(x0)
            rc_r, rho, nu, _ = W.amg_rho(amg, x0, xe, 1, 1e-8, 100)
            b = torch.from_numpy(rhs_batch(N, 1, w["seed"])).to(dev)
            psi = torch.zeros_like(b)
            rc, info = W.amg_solve(amg, b, psi, 1, 1e-8)
            ref = torch.zeros_like(b)
            rc2, info2 = W.amg_solve(amg, b, ref, 1, 1e-13)
            err = float(torch.linalg.vector_norm(psi - ref) / torch.linalg.vector_norm(ref))
            row = {"study": "rho", "setup": args.study_setup, "workload": name, "N": N, "beta": w["beta"],
                   "eta": eta, "m": w["m"],
                   "rho": float(rho[0]), "rho_iters": int(nu[0]), "rho_met": rc_r == W.WL_OK,
                   "diverged": bool(rho[0] > 1.0),
                   "gmres_iters": info[0]["iters"], "restarts": info[0]["restarts"],
                   "relres": info[0]["true_relres"], "relerr": err, "ref_relres": info2[0]["true_relres"],
                   "setup_s": round(setup_s, 3)}
            rows.append(row)
            print(json.dumps(row), flush=True)
            amg.close()
            op.close()
    summary = {}
    for r in rows:
        key = "N%d_beta%g" % (r["N"], r["beta"])
        summary.setdefault(key, []).append(r)
    out = {}
    for key, rs in summary.items():
        rh = [r["rho"] for r in rs]
        out[key] = {"cases": len(rs), "rho_median": round(float(np.median(rh)), 3),
                    "rho_max": round(max(rh), 3), "rho_above_0.6": sum(v > 0.6 for v in rh),
                    "diverged": sum(v > 1.0 for v in rh),
                    "gmres_iters_max": max(r["gmres_iters"] for r in rs),
                    "restarted": sum(r["restarts"] > 1 for r in rs),
                    "err_over_res_max": round(max(r["relerr"] / max(r["relres"], 1e-300) for r in rs), 1)}
    print(json.dumps({"study": "rho", "setup": args.study_setup, "summary": out}))


def main():
    faulthandler.enable()
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if args.kernel_only:
        if rank == 0:
            run_kernel_only(args)
        return
    if args.study == "rho":
        if rank == 0:
            run_study_rho(args)
        return
    if args.serving_only:
        if rank == 0:
            import torch
            from paper_1308_5992_gb300 import wilson_amg as W
            dev = torch.device("cuda", 0)
            torch.cuda.set_device(dev)
            print(json.dumps({"serving": run_serving(args, 0, dev, W, torch)}))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_gb300(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
