"""Benchmark: MPS Vlasov-Poisson RK4-C1 steps/s at n = 20 (1024 x 1024), chi = 64.

One "step" is one RK4 step with compression level C1 of the two-stream
workload on a 1024 x 1024 grid (10 + 10 bit sites, sequential mapping),
chi = 64, tol = 1e-10, dt = 0.002: four field solves (density, Poisson, E as
an MPS), four MPO applications and seven compressions (QR sweep + truncated
SVD sweep).  The state is the saturated-bond two-stream input of
``paper_2205_11990_gb300.inputs.saturated_two_stream`` (seeded), whose
middle bonds sit at the chi = 64 cap.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the same workload instead (bounded sample).  Multi-GPU runs are independent
replicas (the path does not shard): value = steps of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "saturated_two_stream_1024x1024_seq"
CHI, TOL, DT = 64, 1e-10, 0.002
FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2.070  # 2 DFMA/clk/SM x 2 flop x 152 SMs x 2070 MHz (nominal 1.26 TF/s)
# The factorisations (QR, Q formation, Jacobi) run in double-word FP32: their
# roof is the FP32 pipe (128 lanes/SM/clk x 152 SMs x 2070 MHz) over the FP32
# instructions per pair of FP64-equivalent flops of their work mix -- half
# compensated dot-product steps (12 instructions), half double-word axpy
# updates (29): 20.5 instructions per 2 flops, 3.93 TF/s.
DW_PEAK_GFLOPS = 128 * 152 * 2.070 * 2 / 20.5
# What the path computes in: FP64 storage, contractions, Poisson and truncation
# rule; the QR, Q formation and Jacobi SVD in double-word FP32 (~2^-48).
DTYPE = "f64 storage/contractions, df32 (~2^-48) factorisations"
PROFILES = os.path.join(ROOT, "profiles")
# the dominant kernel of each class on the headline path (streams = 0: the
# batched kernels of a one-member lockstep group) and on the two-stream path
KERNEL_OF_CLASS = {"qr_factor": "kb_qr_factor_cl", "jacobi": "kb_jacobi_dw", "gemm": "kb_gemm",
                   "qr_formq": "kb_qr_formq_reg", "apply": "kb_site_sum", "select": "kb_select"}
KERNEL_OF_CLASS_STREAMS = {k: v[1:] for k, v in KERNEL_OF_CLASS.items()}


def profile_traffic(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` on `workload`, from the
    `bench-traffic:` lines of the ncu summaries under profiles/ (None when no
    capture of that kernel and workload is committed)."""
    if not os.path.isdir(PROFILES):
        return None
    for fn in sorted(os.listdir(PROFILES)):
        if not fn.endswith(".md"):
            continue
        for line in open(os.path.join(PROFILES, fn)):
            parts = line.split()
            if len(parts) == 4 and parts[0] == "bench-traffic:" and parts[1] == kernel and parts[2] == workload:
                return float(parts[3])
    return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline (profiling runs)")
    p.add_argument("--mode", default="step", choices=["step", "batch", "serve", "precision", "species", "peaks",
                                                          "compressibility"],
                   help="step: the headline single-run steps/s; batch / serve: many runs on one GPU; "
                        "species: electrons and ions on one field (Buneman, Dougherty collisions)")
    p.add_argument("--species-workload", default="saturated_buneman_512x512_s3",
                   help="named workload of paper_2205_11990_gb300.inputs.SPECIES_WORKLOADS (--mode species)")
    p.add_argument("--instances", type=int, default=32)
    p.add_argument("--concurrency", type=int, default=8)
    p.add_argument("--time", type=float, default=4.0, help="compressibility: physical time of the runs")
    p.add_argument("--groups", type=int, default=4, help="batch / serve: lockstep groups (bucketed by site count)")
    p.add_argument("--bits", default="8,12", help="batch / serve: grid bits per dimension, min,max")
    p.add_argument("--chis", default="16,32,64,128", help="batch / serve: bond caps drawn uniformly")
    p.add_argument("--rate", type=float, default=20.0, help="serve: mean Poisson arrival rate (req/s)")
    p.add_argument("--window", type=float, default=20.0, help="serve: arrival window (s)")
    p.add_argument("--workload", default=WORKLOAD,
                   help="named workload of paper_2205_11990_gb300.inputs.WORKLOADS (profiling of smaller cases)")
    args = p.parse_args()
    set_workload(args.workload)
    return args


def set_workload(name):
    global WORKLOAD, CHI, DT
    from paper_2205_11990_gb300 import inputs as I
    w = I.WORKLOADS[name]
    WORKLOAD, CHI, DT = name, w["chi"], w["dt"]


def dist_init(n):
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    return rank, world


def barrier(world):
    """Barrier across the replicas (no-op for one process)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ms, world, device="cuda"):
    """The slowest replica's timed duration (ms): the job's duration."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, ms):
    """Whole-job throughput: the steps of every replica over the job's duration."""
    return world * steps / (ms / 1e3)


def metric_name(lay):
    from paper_2205_11990_gb300 import inputs as I
    mp = "seq" if lay.mapping == 0 else "interleaved"
    ic = I.WORKLOADS[WORKLOAD]["ic"]
    label = "two-stream" if "two_stream" in ic else ic.replace("_", " ")
    return f"MPS VP steps/s at n={lay.n} chi={CHI} (RK4-C1, {lay.Nx}x{lay.Nv} {label}, {mp})"


def workload():
    from paper_2205_11990_gb300 import inputs as I
    w = I.WORKLOADS[WORKLOAD]
    lay = w["layout"]
    return lay, I.initial_condition(w["ic"], lay)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        # raw samples: $VP_CLOCKS_DIR when set (kept with the run's other output), else the temp dir
        import tempfile
        d = os.environ.get("VP_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", idx, f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0].split()[0]))
                mx.append(float(parts[1].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps

    lay, f0 = workload()
    ctx = vpmps.Context()
    m = ctx.mps_from_grid(lay, f0, CHI, TOL)
    # streams=0: the step runs as a one-member lockstep group (both
    # compressions of a stage in every launch)
    sim = ctx.sim(lay, m, DT, CHI, TOL, TOL, streams=0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    # measured rates of the units the kernels run on (outside the timed region)
    probes = {k: ctx.peak_probe(k) for k in ("fp64_fma", "dw_dot", "dw_axpy", "fp32_fma", "dmma")}
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()

    clocks = Clocks()
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = ctx.kernel_launches
    ctx.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    recs = []
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # evict the L2 between timed steps (outside the event pair)
        ev[i][0].record(stream)
        recs += sim.step(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall
    prof = ctx.profile_read()
    ctx.profile(False)
    launches = ctx.kernel_launches - launches0
    clk = clocks.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    steps_per_s = job_rate(world, args.steps, ms)

    roof = roofline(prof, ms, world, WORKLOAD, probes)

    e2e = None
    if not args.no_e2e:
        # end to end through the public entry point vp_run: host f0 in, f(T)
        # and the per-step records out, MPS creation included
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fT, _ = ctx.run(lay, f0, DT, args.steps, CHI, TOL, TOL, want_f=True, streams=0)
        t1 = time.perf_counter() - t0
        nbytes = f0.size * 8
        e2e = {"value": world * args.steps / t1, "unit": "steps/s",
               "h2d_bytes_per_step": nbytes / args.steps,
               "d2h_bytes_per_step": (nbytes + 40 * args.steps) / args.steps}
    out = {
        "metric": metric_name(lay),
        "value": steps_per_s, "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE, "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": f"{lay.Nx}x{lay.Nv}", "sites": f"{lay.nx}+{lay.nv}",
                   "mapping": "seq" if lay.mapping == 0 else "interleaved", "chi": CHI,
                   "tol": TOL, "dt": DT, "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MB write)"},
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "diag": {"max_bond": max(r["max_bond"] for r in recs), "field_energy": recs[-1]["field_energy"],
                 "wall_s": t_wall, "kernel_ms": {k: round(v[0], 3) for k, v in prof.items()},
                 "flops_per_step": sim.flops / max(1, args.steps + args.warmup)},
    }
    if rank == 0:
        out["cpu_baseline"] = None if args.no_cpu else cpu_baseline(lay, f0, budget_s=25.0)
        print(json.dumps(out), flush=True)


def roofline(prof, ms, world, workload, probes=None, lockstep=True):
    """Roofline entry of the dominant kernel class of the profiled window."""
    top = max(prof, key=lambda k: prof[k][0])
    tms, tl, work = prof[top]
    if top == "apply":
        achieved = work / (tms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": 6789.6, "unit": "GB/s",
                "peak_basis": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    else:
        achieved = work / (tms / 1e3) / 1e12
        if top == "gemm":  # FP64 GEMMs on the FP64 pipe
            roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                    "peak_basis": "FP64 FMA: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (derived from unit counts)"}
        else:  # double-word factorisations on the FP32 pipe
            peak = DW_PEAK_GFLOPS / 1e3
            basis = ("double-word FP32: 128 FP32 lanes/clk/SM x 152 SMs x 2070 MHz x 2 flops / 20.5 FP32 "
                     "instructions (derived from unit counts)")
            if probes and probes.get("dw_dot") and probes.get("dw_axpy"):
                # the measured rate of the same dot/update mix, when higher
                # (the compiler fuses a few of the counted instructions)
                mix = 2.0 / (1.0 / probes["dw_dot"] + 1.0 / probes["dw_axpy"])
                if mix > peak:
                    peak = mix
                    basis = "double-word FP32 dot/update mix, measured by vp_peak_probe on this GPU (of measured)"
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "peak_basis": basis,
                    "peak_fp64": FP64_PEAK_GFLOPS / 1e3, "frac_fp64": achieved / (FP64_PEAK_GFLOPS / 1e3)}
    roof["frac"] = roof["achieved"] / roof["peak"]
    kernel = (KERNEL_OF_CLASS if lockstep else KERNEL_OF_CLASS_STREAMS).get(top, top)
    # DRAM bytes (read + write) per launch of the dominant kernel, from the ncu
    # captures summarised under profiles/
    roof["traffic"] = profile_traffic(kernel, workload)
    roof["kernel"] = kernel
    roof["class"] = top
    roof["launches"] = tl
    roof["share_of_step"] = tms / ms * world if ms else None
    if probes:
        roof["measured_tflops"] = {k: round(v, 4) for k, v in probes.items()}
    return roof


def run_species(args, rank, world):
    """Electrons and ions sharing one field: RK4-C1 steps of both species
    (Buneman set-up with Dougherty collisions), timed like the headline."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import inputs as I
    from paper_2205_11990_gb300 import vpmps

    name = args.species_workload
    lays, fs, species, chi, dt = I.species_workload(name)
    ctx = vpmps.Context()
    run = ctx.multi(lays, species, [ctx.mps_from_grid(l, f, chi, TOL) for l, f in zip(lays, fs)], dt, chi, TOL, TOL)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        run.step(1)
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = ctx.kernel_launches
    ctx.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    recs = []
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        recs += run.step(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    launches = ctx.kernel_launches - launches0
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    e2e = None
    if not args.no_e2e:
        # public API end to end: host grids in (MPS creation), steps, host grids out
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r2 = ctx.multi(lays, species, [ctx.mps_from_grid(l, f, chi, TOL) for l, f in zip(lays, fs)], dt, chi,
                       TOL, TOL)
        r2.step(args.steps)
        outs = [r2.state(s).to_grid(l) for s, l in enumerate(lays)]
        t1 = time.perf_counter() - t0
        r2.close()
        nb = sum(f.size * 8 for f in fs)
        e2e = {"value": world * args.steps / t1, "unit": "steps/s", "h2d_bytes_per_step": nb / args.steps,
               "d2h_bytes_per_step": (sum(o.size * 8 for o in outs) + 40 * len(lays) * args.steps) / args.steps}
    le = lays[0]
    out = {
        "metric": f"MPS VP two-species steps/s (RK4-C1, Buneman {le.Nx}x{le.Nv} electrons + {lays[1].Nx}x{lays[1].Nv} "
                  f"ions, S3, chi={chi}, Dougherty collisions)",
        "value": job_rate(world, args.steps, ms), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
        "config": {"workload": name, "species": species, "chi": chi, "tol": TOL, "dt": dt,
                   "parallelism": f"replicas x{world}", "l2": "flushed between timed steps (256 MB write)"},
        "roofline": roofline(prof, ms, world, name, lockstep=False),
        "gpu_launches": launches, "clocks": clk, "e2e": e2e,
        "diag": {"max_bond": [max(r["max_bond"][s] for r in recs) for s in range(len(lays))],
                 "field_energy": recs[-1]["field_energy"], "kernel_ms": {k: round(v[0], 3) for k, v in prof.items()}},
    }
    if rank == 0:
        if not args.no_cpu:
            from oracle import vp as OV
            cs = [OV.mps_from_f(f, l, chi, TOL) for f, l in zip(fs, lays)]
            done, t = 0, 0.0
            while t < 25.0:
                t0 = time.perf_counter()
                cs, _ = OV.multi_rk4_step(cs, lays, species, dt, chi, TOL, TOL)
                t += time.perf_counter() - t0
                done += 1
            out["cpu_baseline"] = {"value": done / t, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": f"{done} two-species RK4-C1 step(s) of the same workload "
                                             f"(numpy/LAPACK, all host cores), {t:.1f} s"}
        print(json.dumps(out), flush=True)


def oracle_steps(lay, f0, nsteps, budget_s):
    """Time up to nsteps oracle RK4-C1 steps (stop once budget_s is spent)."""
    from oracle import vp as OV
    c = OV.mps_from_f(f0, lay, CHI, TOL)
    done, t = 0, 0.0
    while done < nsteps:
        t0 = time.perf_counter()
        c, _ = OV.rk4_step(c, lay, DT, CHI, TOL, TOL)
        t += time.perf_counter() - t0
        done += 1
        if t > budget_s:
            break
    return done, t


def cpu_baseline(lay, f0, budget_s):
    from oracle import mps as OM
    OM.TIE_STATS.update(cuts=0, fired=0, min_gap=float("inf"))
    done, t = oracle_steps(lay, f0, 1000, budget_s)
    ts = dict(OM.TIE_STATS)
    return {"value": done / t, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} RK4-C1 step(s) of the same workload from the same initial MPS "
                      f"(numpy/LAPACK, all host cores), {t:.1f} s",
            # how often the truncation tie rule moved a cut in those steps, and
            # the smallest relative gap at a cut it left alone
            "tie_rule": {"cuts": ts["cuts"], "fired": ts["fired"], "min_gap_at_cut": ts["min_gap"]}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    lay, f0 = workload()
    for _ in range(min(args.warmup, 1)):
        oracle_steps(lay, f0, 1, 1e9)
    done, t = oracle_steps(lay, f0, args.steps, 150.0)
    v = done / t
    print(json.dumps({
        "impl": "reference", "metric": metric_name(lay),
        "value": v, "unit": "steps/s", "n_gpus": world, "steps": done, "warmup": min(args.warmup, 1),
        "ms_per_step": 1e3 * t / done, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (numpy/LAPACK oracle)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": f"{lay.Nx}x{lay.Nv}", "sites": f"{lay.nx}+{lay.nv}",
                   "mapping": "seq" if lay.mapping == 0 else "interleaved", "chi": CHI, "tol": TOL, "dt": DT,
                   "parallelism": "cpu"},
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{done} of {args.steps} requested steps (capped at 150 s of CPU work)"},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def mixed_request(rng, bits=(6, 9), chis=(16, 32, 64), amp_range=(1e-3, 0.5)):
    """One seeded request of the batching / serving mix (the batching
    configuration's distribution): grid bits per dimension uniform in
    bits[0]..bits[1] (square grids), chi uniform in chis, sequential or
    interleaved 50/50, Landau (k ~ U[0.3, 0.6], amplitude log-uniform in
    amp_range, v in [-6, 6]) or bump-on-tail (n_b = 0.1, v_b = 4.5,
    sigma_b = 0.5, k ~ U[0.3, 0.6], v in [-8, 8]) 50/50, dt = 0.6 dx / vmax."""
    import math
    from paper_2205_11990_gb300 import inputs as I
    nb = int(rng.integers(bits[0], bits[1] + 1))
    mapping = I.SEQ if rng.random() < 0.5 else I.INTERLEAVED
    k = float(rng.uniform(0.3, 0.6))
    if rng.random() < 0.5:
        amp = float(math.exp(rng.uniform(math.log(amp_range[0]), math.log(amp_range[1]))))
        lay = I.Layout(nb, nb, 0.0, 2 * math.pi / k, -6.0, 6.0, mapping)
        f0 = I.landau(lay, amp, k)
    else:
        lay = I.Layout(nb, nb, 0.0, 2 * math.pi / k, -8.0, 8.0, mapping)
        f0 = I.bump_on_tail(lay, 1e-3, k)
    dx = (lay.xmax - lay.xmin) / lay.Nx
    dt = 0.6 * dx / lay.vmax
    chi = int(rng.choice(list(chis)))
    return lay, f0, dt, chi


def _parse_range(s):
    a, b = (int(x) for x in s.split(","))
    return a, b


def run_batch(args):
    """Many independent runs on one GPU: the same seeded request set through
    the plain per-instance path (one run at a time, vp_step) and through the
    lockstep engine (bucketed groups, continuous batching); sims/s of each."""
    import numpy as np
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    ctx = vpmps.Context()
    rng = np.random.Generator(np.random.PCG64(0))
    bits = _parse_range(args.bits)
    chis = tuple(int(c) for c in args.chis.split(","))
    reqs = [mixed_request(rng, bits, chis) for _ in range(args.instances)]
    steps = max(1, args.steps)
    out = {}
    arms = [("lockstep", dict(max_concurrent=args.instances, lockstep=args.groups)),
            ("sequential", dict(max_concurrent=1, lockstep=0))]
    results = {}
    launches = 0
    for label, kw in arms:
        b = vpmps.Batch(ctx, kw["max_concurrent"], 200 << 30, lockstep=kw["lockstep"])
        ids = [b.submit(lay, f0, dt, steps, chi, keep_f=True) for lay, f0, dt, chi in reqs]
        t0 = time.perf_counter()
        b.start()
        b.wait()
        t = time.perf_counter() - t0
        res = {r["id"]: r for r in b.poll(4 * len(reqs))}
        assert all(r["status"] == 0 for r in res.values()), [r["status"] for r in res.values()]
        step_ms = np.concatenate([b.records(i)[1] for i in ids])
        results[label] = [b.records(i, want_f=True) for i in ids]
        out[label] = {"sims_per_s": len(reqs) / t, "instance_steps_per_s": len(reqs) * steps / t, "wall_s": t,
                      "step_ms_p50": float(np.percentile(step_ms, 50)),
                      "step_ms_p99": float(np.percentile(step_ms, 99)),
                      "run_ms_p50": float(np.median([r["queue_ms"] + r["run_ms"] for r in res.values()])),
                      "run_ms_p99": float(np.percentile([r["queue_ms"] + r["run_ms"] for r in res.values()], 99))}
        out[label]["gpu_launches"] = b.kernel_launches
        launches += b.kernel_launches
        b.close()
    # the two arms compute the same runs: every final state and record equal
    same = all(np.array_equal(a[2], c[2]) and a[0] == c[0] for a, c in zip(results["lockstep"], results["sequential"]))
    print(json.dumps({
        "metric": "batched sims/s (RK4-C1 runs, mixed sizes/chi/mappings)", "value": out["lockstep"]["sims_per_s"],
        "unit": "sims/s", "n_gpus": 1, "higher_is_better": True, "dtype": DTYPE, "data": "synthetic",
        "config": {"workload": f"mixed Landau/bump-on-tail, grid bits {bits[0]}..{bits[1]} per dim, chi {chis}, "
                               f"seq/interleaved", "instances": args.instances, "steps_per_run": steps,
                   "lockstep_groups": args.groups, "seed": 0},
        "lockstep": out["lockstep"], "sequential_fp64_per_instance": out["sequential"],
        "speedup_vs_sequential": out["lockstep"]["sims_per_s"] / out["sequential"]["sims_per_s"],
        "results_identical": bool(same), "gpu_launches": ctx.kernel_launches + launches}), flush=True)


def run_serve(args):
    import numpy as np
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    ctx = vpmps.Context()
    rng = np.random.Generator(np.random.PCG64(1))
    arrivals, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / args.rate))
        if t > args.window:
            break
        lay, f0, dt, chi = mixed_request(rng, _parse_range(args.bits), tuple(int(c) for c in args.chis.split(",")))
        arrivals.append((t, lay, f0, dt, chi, int(rng.integers(max(2, args.steps // 4), args.steps + 1))))
    b = vpmps.Batch(ctx, args.concurrency, 200 << 30, lockstep=args.groups)
    b.start()
    t0 = time.perf_counter()
    done, i = [], 0
    while len(done) < len(arrivals):
        now = time.perf_counter() - t0
        while i < len(arrivals) and arrivals[i][0] <= now:
            _, lay, f0, dt, chi, n = arrivals[i]
            b.submit(lay, f0, dt, n, chi)
            i += 1
        done += b.poll(256)
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    steps_ms = []
    for r in done:
        recs, ms, _ = b.records(r["id"])
        steps_ms += list(ms)
    run_lat = [r["queue_ms"] + r["run_ms"] for r in done]
    launches = ctx.kernel_launches + b.kernel_launches
    b.close()
    print(json.dumps({
        "metric": "served sims/s with p50/p99 step and run latency (continuous batching)",
        "value": len(done) / wall, "unit": "sims/s", "n_gpus": 1, "higher_is_better": True, "dtype": DTYPE,
        "data": "synthetic",
        "config": {"arrivals": "Poisson", "rate_per_s": args.rate, "window_s": args.window, "requests": len(done),
                   "steps_per_run": f"U[{max(2, args.steps // 4)}, {args.steps}]", "grid_bits": args.bits,
                   "chis": args.chis, "lockstep_groups": args.groups, "resident_per_group": args.concurrency,
                   "seed": 1},
        "step_ms_p50": float(np.percentile(steps_ms, 50)), "step_ms_p99": float(np.percentile(steps_ms, 99)),
        "run_ms_p50": float(np.percentile(run_lat, 50)), "run_ms_p99": float(np.percentile(run_lat, 99)),
        "wall_s": wall, "gpu_launches": launches}), flush=True)


def run_precision(args):
    """FP64-contraction path vs the reduced-precision contraction modes
    (factorisations double-word FP32 in every mode) on the same state: steps/s of each and the field-energy and f errors
    against the FP64 run."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    lay, f0 = workload()
    ctx = vpmps.Context()
    out = {}
    for name, prec in vpmps.PRECISIONS.items():
        m = ctx.mps_from_grid(lay, f0, CHI, TOL)
        sim = ctx.sim(lay, m, DT, CHI, TOL, TOL, precision=prec)
        sim.step(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs = sim.step(args.steps)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out[name] = (args.steps / t, np.array([r["field_energy"] for r in recs]), sim.state().to_grid(lay),
                     max(r["max_bond"] for r in recs))
        sim.close()
        m.close()
    v64, we64, f64, _ = out["fp64"]
    modes = {}
    for name, (v, we, f, mb) in out.items():
        modes[name] = {"steps_per_s": v, "speedup_vs_fp64": v / v64, "max_bond": mb,
                       "field_energy_abs_err_max": float(np.max(np.abs(we - we64))),
                       "field_energy_rel_err_max": float(np.max(np.abs(we - we64) / we64)),
                       "f_rel_l2_err": float(np.linalg.norm(f - f64) / np.linalg.norm(f64))}
    best = out["tf32x3"][0]
    print(json.dumps({
        "metric": metric_name(lay) + " - contraction precision modes", "value": best, "unit": "steps/s",
        "n_gpus": 1, "steps": args.steps, "higher_is_better": True,
        "dtype": "tf32x3 contractions (tcgen05), df32 (~2^-48) factorisations", "data": "synthetic",
        "config": {"workload": WORKLOAD, "chi": CHI, "tol": TOL, "dt": DT,
                   "errors": "after 1 + steps steps, against the FP64 run from the same state"},
        "modes": modes}), flush=True)


def run_compressibility(args):
    """State compressibility (main text, "State Compressibility", the rms
    compression error against D): nonlinear Landau (A = 0.5, k = 0.5, the
    paper's set-up) run with no bond cap at tol = 1e-10 on several grids to
    the same time T = --time, then the rms error over the grid of f - f_D for
    each D."""
    import math
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import inputs as I
    from paper_2205_11990_gb300 import vpmps
    ctx = vpmps.Context()
    chis = [2, 4, 8, 16, 32, 64]
    out = {}
    for bits in (6, 7, 8):
        lay = I.Layout(bits, bits, 0.0, 4 * math.pi, -6.0, 6.0, I.SEQ)
        f0 = I.landau(lay, 0.5, 0.5)
        steps = max(1, int(math.ceil(args.time / (0.6 * (lay.xmax - lay.xmin) / lay.Nx / lay.vmax))))
        dt = args.time / steps
        full = 1 << bits
        sim = ctx.sim(lay, ctx.mps_from_grid(lay, f0, full, TOL), dt, full, TOL, TOL, streams=0)
        t0 = time.perf_counter()
        recs = sim.step(steps)
        t = time.perf_counter() - t0
        st = sim.state()
        f = st.to_grid(lay)
        rms_f = float((f * f).mean() ** 0.5)
        err = ctx.compression_error(st, chis, 0.0)
        out[f"{lay.Nx}x{lay.Nv}"] = {"t": recs[-1]["t"] + dt, "max_bond": max(st.bonds()), "rms_f": rms_f,
                                    "rms_error": {str(c): float(e) for c, e in zip(chis, err)},
                                    "steps": steps, "steps_per_s": steps / t}
        sim.close()
    print(json.dumps({"metric": "rms compression error vs bond dimension (nonlinear Landau)", "unit": "rms of f - f_D",
                      "dtype": DTYPE, "data": "synthetic", "config": {"ic": "Landau A=0.5 k=0.5, seq",
                      "time": args.time, "tol": TOL, "D": chis}, "grids": out}), flush=True)


def run_peaks(args):
    """Measured rates of the arithmetic units the kernels run on."""
    import __graft_entry__ as g
    g.build()
    from paper_2205_11990_gb300 import vpmps
    ctx = vpmps.Context()
    probes = {k: ctx.peak_probe(k) for k in vpmps.Context.PROBES}
    print(json.dumps({"metric": "measured arithmetic rates", "unit": "TFLOP/s (FP64-equivalent flops)",
                      "measured": probes,
                      "derived": {"fp64_fma": FP64_PEAK_GFLOPS / 1e3, "dw_factorisation_mix": DW_PEAK_GFLOPS / 1e3,
                                  "fp32_fma": 128 * 152 * 2.070 * 2 / 1e3}}), flush=True)


def main():
    args = parse()
    if args.mode == "peaks":
        return run_peaks(args)
    if args.mode == "compressibility":
        return run_compressibility(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.mode == "species":
        run_species(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
