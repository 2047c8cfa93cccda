"""Benchmark: cell-steps/s of the implicit FLD + ionisation + heating step.

Workload: the reionization-like field at 256^3 (periodic 14.4 Mpc comoving box at z = 9,
log-normal density, 2000 density-peak sources, Gaussian velocities; see ``workloads``),
one implicit step (v) per timed step: setup, globalised Newton with nonlinear
elimination of the local block, Schur-reduced FP64 CG with a multigrid preconditioner,
and the gas-energy hand-over e_h += e_c.  ``value`` is the mixed path (FP32 multigrid
inside FP64 Newton/CG); the all-FP64 path is timed the same way and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--size 256]
Under torchrun each rank runs an independent replica on its own GPU ("replicas only":
the step has no cross-GPU exchange on one GPU per problem).  ``--impl reference`` times
the FP64 CPU oracle on host cores instead (bounded sub-block samples of the workload).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s of implicit FLD+chem solve, 256^3, mixed vs FP64; V-cycle HBM GB/s"


def parse():
    """Command line: the driver's --gpus/--steps/--warmup/--impl plus size, tolerances and
    switches for the optional measurements."""
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=256)
    p.add_argument("--newton-tol", type=float, default=1e-6)
    p.add_argument("--lin-rtol", type=float, default=1e-3)
    p.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 comparison run")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--no-advect", action="store_true", help="skip the advection pre-step measurement")
    p.add_argument("--helium", action="store_true",
                   help="time the hydrogen + helium version of the field (Y = 0.24); no CPU baseline")
    return p.parse_args()


L2_BYTES = 129e6   # GB300 L2


def workload_sources(n):
    """Source count of the n^3 field: 2000, scaled down with the volume below 128^3."""
    return 2000 if n >= 128 else max(2, 2000 * n**3 // 256**3)


def workload(n):
    """The bench's reionization field at n^3 (the 256^3 cell size; box and photon rate scale
    with the volume)."""
    import workloads as W
    return W.reionization_field(n=n, nsrc=workload_sources(n), box_mpc=14.4 * n / 256,
                                ndot_total=1e52 * (n / 256) ** 3)


def l2_note(n):
    """How the timed steps stand to the L2 (the timing rule: inputs larger than L2, or a flush):
    the working set is taken as the DRAM traffic of one Newton evaluation."""
    ws = ASSEMBLE_DRAM_BYTES_PER_CELL * n**3
    field = 8.0 * n**3 / 1e6
    if ws > L2_BYTES:
        return (f"inputs larger than L2 (one Newton evaluation moves {ws / 1e6:.0f} MB, each FP64 field "
                f"{field:.1f} MB; L2 {L2_BYTES / 1e6:.0f} MB)")
    return f"inputs smaller than L2 at this size (one Newton evaluation moves {ws / 1e6:.0f} MB); L2 not flushed"


# FP64 flops per cell of one newton_assemble launch on this workload: the work the kernel
# executes (2 x DFMA + DADD + DMUL thread instructions counted by ncu), mean over the five
# launches of one step at 128^3 (743-1419 per launch: one or two evaluations of the local
# equations per cell); the kernel is FP64-ALU bound
ASSEMBLE_FP64_FLOPS_PER_CELL = 1107.0
# its DRAM traffic per cell (dram__bytes_read.sum + dram__bytes_write.sum), mean over the five
# launches of one warm 256^3 step (ncu, the timed step only), scaled to a launch by the cells
ASSEMBLE_DRAM_BYTES_PER_CELL = 243.5
# the same two figures for the hydrogen + helium kernel (--helium): mean over the four launches
# of one step of the 128^3 field with helium (ncu), 2347-5469 flops per launch
ASSEMBLE_HE_FP64_FLOPS_PER_CELL = 4227.0
ASSEMBLE_HE_DRAM_BYTES_PER_CELL = 220.1
# FP64 flops per cell of the advection kernel with rho_b (three face Courant numbers and three
# donor-cell updates of three densities per axis: 3 x (6 + 3 x 4)), counted from the source
ADVECT_FP64_FLOPS_PER_CELL = 54.0
# FP64 peak from unit counts and clock: 2 FP64 FMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz
FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2.07


def load_peaks():
    """MEASURED_PEAKS.json at the repository root, or None."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ------------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi sampling of SM clocks, power and throttle reasons every 200 ms while the
    timed region runs (a context manager); summary() gives the median clock and reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        """{sm_mhz: median under load, sm_max_mhz, reasons: active throttle reasons, samples}."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------ mixed against FP64 final states


def _final_state(s):
    """(E, x_HI, T) of a solver's current state on the host (CGS E, temperature in K)."""
    from paper_0908_2654_gb300.units import temperature
    st = s.state_cgs()
    nHI, E = st[1], st[-1]
    u = s.units
    rho = s.rho.cpu().numpy() * u.u_d
    v = tuple(x.cpu().numpy() * u.u_v for x in s.v)
    T = temperature(s.e_h.cpu().numpy() * u.u_v**2, rho, nHI, v)
    return E, nHI / (rho / 1.6735575e-24), T


def state_errors(a, b):
    """Differences of state a from the reference b: E normwise (2 and max, relative), x_HI and T
    pointwise relative (x_HI with a floor of 1e-8)."""
    Ea, xa, Ta = a
    Eb, xb, Tb = b
    return {"E_rel_2": float(np.linalg.norm(Ea - Eb) / np.linalg.norm(Eb)),
            "E_rel_inf": float(np.max(np.abs(Ea - Eb)) / np.max(np.abs(Eb))),
            "xHI_rel_max": float(np.max(np.abs(xa - xb) / np.maximum(xb, 1e-8))),
            "T_rel_max": float(np.max(np.abs(Ta - Tb) / Tb))}


# ----------------------------------------------------------- whole-job numbers


def reduce_max(value, world, device):
    """Largest value over the ranks: the job takes as long as its slowest replica."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, cells, steps, ms_max):
    """Cell-steps per second of the whole job: every replica advances its own grid."""
    return world * cells * steps / (ms_max * 1e-3)


# -------------------------------------------------------------------- GPU arm


def run_gpu(args, rank, world, local_rank):
    """The GPU arm on this rank: W warm-up and K timed mixed-precision steps of the field
    (barrier and synchronise around the timed region; the library's per-kernel CUDA events
    run on its stream inside that region, giving the kernel durations of the rooflines), then
    the all-FP64 comparison, the end-to-end run from pinned host memory and the advection
    pre-step.  Returns the results bench_line turns into the JSON line."""
    import torch
    import torch.distributed as dist

    from paper_0908_2654_gb300.solver import Solver

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.size
    w = workload(n)
    if args.helium:
        import workloads as W
        w = W.with_helium(w)
    cells = n**3

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(precision, steps, warmup, profile):
        s = Solver(w, precision=precision, newton_tol=args.newton_tol, lin_rtol=args.lin_rtol, max_newton=40,
                   max_lin=400, device=local_rank)
        for _ in range(warmup):
            s.step()
        torch.cuda.synchronize()
        if profile:
            s.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as clk:
            torch.cuda.nvtx.range_push(f"timed_{precision}")   # lets a profiler select these steps
            e0.record(s.stream)
            for _ in range(steps):
                stats.append(s.step())
            e1.record(s.stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        barrier()
        ms = e0.elapsed_time(e1)
        prof = s.profile() if profile else None
        final = _final_state(s)
        s.close()
        return ms, stats, prof, clk.summary(), final

    ms_mixed, st_mixed, prof, clocks, final_mixed = timed("mixed", args.steps, args.warmup, profile=True)
    ms_max = reduce_max(ms_mixed, world, dev)
    value = job_rate(world, cells, args.steps, ms_max)

    fp64 = None
    if not args.no_fp64:
        ms64, st64, _, _, final64 = timed("fp64", args.steps, args.warmup, profile=False)
        ms64 = reduce_max(ms64, world, dev)
        v64 = job_rate(world, cells, args.steps, ms64)
        fp64 = {"value": v64, "ms_per_step": ms64 / args.steps,
                "newton_iters": [x["newton_iters"] for x in st64], "linear_iters": [x["linear_iters"] for x in st64],
                "speedup_mixed_vs_fp64": value / v64,
                "mixed_vs_fp64_error": state_errors(final_mixed, final64)}

    advect = None if args.no_advect else run_advect(w, local_rank)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, w, local_rank, barrier, world)

    return dict(value=value, ms=ms_max, stats=st_mixed, prof=prof, clocks=clocks, fp64=fp64, e2e=e2e, w=w,
                advect=advect)


def run_advect(w, local_rank, calls=10, warmup=3):
    """The advection pre-step (rho_b, n_HI and E by donor cell) on the same field, timed per
    kernel with CUDA events: {kernel: (launches, ms, algorithmic bytes)}."""
    from paper_0908_2654_gb300.solver import Solver
    s = Solver(w, precision="fp64", device=local_rank)
    for _ in range(warmup):
        s.advect()
    s.set_profiling(True)
    for _ in range(calls):
        courant = s.advect()
    prof = s.profile()
    s.close()
    out = {k: prof[k] for k in ("advect", "advect_courant") if k in prof}
    out["courant_max"] = courant
    return out


def run_e2e(args, w, local_rank, barrier, world):
    """Same steps through the C ABI with host arrays: the step's inputs are copied from pinned host
    memory and the result read back inside the timed region."""
    import torch

    from paper_0908_2654_gb300.solver import Solver

    s = Solver(w, precision="mixed", newton_tol=args.newton_tol, lin_rtol=args.lin_rtol, max_newton=40,
               max_lin=400, device=local_rank)
    # the state lives in host memory between steps: E, n_HI and e_h go in and come back out
    host_in = {k: getattr(s, k).cpu().pin_memory() for k in ("E", "nHI", "rho", "e_h", "clump")}
    host_v = [v.cpu().pin_memory() for v in s.v]
    out = {k: host_in[k] for k in ("E", "nHI", "e_h")}
    out["ec"] = torch.empty_like(s.ec, device="cpu").pin_memory()
    bi = sum(t.numel() * t.element_size() for t in list(host_in.values()) + host_v)
    bo = sum(t.numel() * t.element_size() for t in out.values())
    stream = s.stream

    def one():
        with torch.cuda.stream(stream):
            for k, t in host_in.items():
                getattr(s, k).copy_(t, non_blocking=True)
            for dv, hv in zip(s.v, host_v):
                dv.copy_(hv, non_blocking=True)
        s.step()
        with torch.cuda.stream(stream):
            for k, t in out.items():
                t.copy_(getattr(s, k), non_blocking=True)
        stream.synchronize()

    for _ in range(max(1, args.warmup)):
        one()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = reduce_max(e0.elapsed_time(e1), world, torch.device("cuda", local_rank))
    s.close()
    cells = w["nx"] * w["ny"] * w["nz"]
    return {"value": job_rate(world, cells, args.steps, ms), "unit": "cell-steps/s",
            "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo}


# ------------------------------------------------------------------ CPU oracle


def oracle_sample(w, m, seed_corner=(0, 0, 0)):
    """An m^3 periodic sub-block of workload w (its fields and the sources inside it)."""
    z0, y0, x0 = seed_corner
    sl = (slice(z0, z0 + m), slice(y0, y0 + m), slice(x0, x0 + m))
    shape = (w["nz"], w["ny"], w["nx"])
    zc, yc, xc = np.unravel_index(w["src_index"], shape)
    inside = (zc >= z0) & (zc < z0 + m) & (yc >= y0) & (yc < y0 + m) & (xc >= x0) & (xc < x0 + m)
    sub = dict(w)
    sub.update(nx=m, ny=m, nz=m, periodic=(True, True, True), bc=None,
               rho_b=w["rho_b"][sl].copy(), T0=w["T0"][sl].copy(), v=tuple(v[sl].copy() for v in w["v"]),
               clump=w["clump"][sl].copy(), E=w["E"][sl].copy(), nHI=w["nHI"][sl].copy(),
               src_index=np.ravel_multi_index((zc[inside] - z0, yc[inside] - y0, xc[inside] - x0), (m, m, m)),
               src_ndot=np.asarray(w["src_ndot"])[inside])
    return sub


def densest_corner(w, m):
    """Corner of the m^3 block holding the most sources (so the sample contains fronts)."""
    shape = (w["nz"], w["ny"], w["nx"])
    zc, yc, xc = np.unravel_index(w["src_index"], shape)
    best, corner = -1, (0, 0, 0)
    for z0 in range(0, shape[0] - m + 1, m):
        for y0 in range(0, shape[1] - m + 1, m):
            for x0 in range(0, shape[2] - m + 1, m):
                c = int(np.sum((zc >= z0) & (zc < z0 + m) & (yc >= y0) & (yc < y0 + m) & (xc >= x0) & (xc < x0 + m)))
                if c > best:
                    best, corner = c, (z0, y0, x0)
    return corner


def time_oracle_steps(w, m, nsteps, tol):
    """Time nsteps oracle steps on the m^3 sub-block of w around its densest corner: returns
    (cell-steps/s, wall seconds, sources inside, cores used).  Cores used = process CPU time
    over wall time, which counts any threads numpy or SciPy start."""
    from oracle import driver
    sub = oracle_sample(w, m, densest_corner(w, m))
    r = driver.Run(sub)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(nsteps):
        r.advance(tol=tol)
    dt, cpu = time.perf_counter() - t0, time.process_time() - c0
    return m**3 * nsteps / dt, dt, int(len(sub["src_index"])), max(1, int(round(cpu / dt)))


def cpu_baseline(w, tol):
    """The oracle timed on a bounded sample of the bench workload (one step of a 24^3 block)."""
    m = 24
    value, secs, nsrc, cores = time_oracle_steps(w, m, 1, tol)
    return {"value": value, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"one implicit step of a {m}^3 periodic sub-block of the {w['nx']}^3 field "
                      f"({nsrc} sources inside), FP64 numpy/SciPy oracle, {secs:.1f} s"}


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores (16^3 sub-blocks of the
    same field, K timed steps after W warm-up steps); prints its JSON line."""
    n = args.size
    w = workload(n)
    m = 16
    for _ in range(args.warmup):
        time_oracle_steps(w, m, 1, args.newton_tol)
    value, secs, nsrc, cores = time_oracle_steps(w, m, args.steps, args.newton_tol)
    cpu = {"value": value, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
           "sample": f"{args.steps} implicit steps of a {m}^3 periodic sub-block of the {n}^3 field "
                     f"({nsrc} sources), FP64 numpy/SciPy oracle"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"reionization-like field {n}^3 (oracle on {m}^3 sub-blocks)", "grid": n},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def bench_line(args, res, world, peaks):
    """The JSON line of the GPU arm from run_gpu's results (rooflines from the per-kernel
    profile, kernel table, launch count)."""
    prof = res["prof"] or {}
    dom_name, dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else (None, None)
    helium = getattr(args, "helium", False)
    roof = None
    cells = args.size**3
    hbm_peak = (peaks or {}).get("hbm_gbs", 6800.0)
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"

    def hbm_roof(name, v):
        ms = v["ms"] / v["launches"]
        ach = v["bytes"] / v["launches"] / (ms * 1e-3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": None, "peak_source": peak_src, "share_of_step": v["ms"] / res["ms"]}

    if dom is not None:
        if dom_name == "newton_assemble":
            ms = dom["ms"] / dom["launches"]
            fpc = ASSEMBLE_HE_FP64_FLOPS_PER_CELL if helium else ASSEMBLE_FP64_FLOPS_PER_CELL
            bpc = ASSEMBLE_HE_DRAM_BYTES_PER_CELL if helium else ASSEMBLE_DRAM_BYTES_PER_CELL
            ach = fpc * cells / (ms * 1e-3) / 1e12
            roof = {"kernel": dom_name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS / 1e3,
                    "unit": "TFLOP/s", "frac": ach / (FP64_PEAK_GFLOPS / 1e3),
                    "traffic": bpc * cells,
                    "traffic_source": ("ncu DRAM bytes per cell of this kernel at 128^3" if helium else
                                       "ncu DRAM bytes per cell of this kernel in one warm 256^3 step") +
                                      " times the cells of one launch",
                    "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz (own probe: 1.19 TFLOP/s)",
                    "flops_per_cell": fpc, "share_of_step": dom["ms"] / res["ms"]}
        else:
            roof = hbm_roof(dom_name, dom)
    # the smoother over all levels, and its fine-level passes alone (the coarse levels are a few
    # microseconds each and latency-bound)
    parts = [prof[k] for k in ("mg_rbgs", "mg_rbgs_fine") if k in prof]
    roof_mg = None
    if parts:
        smooth = {key: sum(p[key] for p in parts) for key in ("launches", "ms", "bytes")}
        roof_mg = hbm_roof("mg_rbgs", smooth)
        if "mg_rbgs_fine" in prof:
            fine = hbm_roof("mg_rbgs_fine", prof["mg_rbgs_fine"])
            roof_mg["fine_level"] = {k: fine[k] for k in ("achieved", "frac", "share_of_step")}
    roof_adv = None
    if res["advect"] and "advect" in res["advect"]:
        v = res["advect"]["advect"]
        ms = v["ms"] / v["launches"]
        ach = ADVECT_FP64_FLOPS_PER_CELL * cells / (ms * 1e-3) / 1e12
        roof_adv = {"kernel": "advect", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS / 1e3,
                    "unit": "TFLOP/s", "frac": ach / (FP64_PEAK_GFLOPS / 1e3), "traffic": None,
                    "flops_per_cell": ADVECT_FP64_FLOPS_PER_CELL, "ms_per_call": ms,
                    "hbm_GBps": v["bytes"] / v["launches"] / (ms * 1e-3) / 1e9,
                    "courant_max": res["advect"]["courant_max"],
                    "note": "advection pre-step (rho_b, n_HI, E), timed apart from the implicit step"}
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None,
                   "share": v["ms"] / res["ms"]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    launches = sum(x["kernel_launches"] for x in res["stats"]) + len(res["stats"])
    w_desc = (f"reionization-like field {args.size}^3, {workload_sources(args.size)} sources, z=9, dt=1 Myr, "
              "theta=1" + (", hydrogen + helium (Y = 0.24)" if helium else ""))
    config = {"workload": w_desc, "grid": args.size, "precision": "mixed (FP32 multigrid in FP64 Newton/CG)",
              "newton_tol": args.newton_tol, "lin_rtol": args.lin_rtol, "parallelism": f"replicas x{world}",
              "l2": l2_note(args.size)}
    fp64 = res["fp64"]
    if fp64:
        # the all-FP64 arm and the mixed-vs-FP64 comparison, kept in the config block
        config["fp64_path"] = {"value": fp64["value"], "ms_per_step": fp64["ms_per_step"],
                               "speedup_mixed_vs_fp64": fp64["speedup_mixed_vs_fp64"],
                               "newton_iters": fp64["newton_iters"], "linear_iters": fp64["linear_iters"]}
        config["mixed_vs_fp64_error"] = fp64["mixed_vs_fp64_error"]
    config["mixed_iters"] = {"newton_iters": [x["newton_iters"] for x in res["stats"]],
                             "linear_iters": [x["linear_iters"] for x in res["stats"]]}
    # per kernel class: share of the step and achieved GB/s on its algorithmic bytes
    config["kernel_shares"] = {k: [round(v["share"], 4), round(v["GBps"], 1) if v["GBps"] else None]
                               for k, v in kernels.items()}
    if roof_mg is not None:
        config["vcycle_smoother"] = {k: roof_mg[k] for k in ("achieved", "frac", "share_of_step")}
        if "fine_level" in roof_mg:
            config["vcycle_smoother"]["fine_level"] = roof_mg["fine_level"]
    line = {
        "metric": METRIC, "value": res["value"], "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": config,
        "newton_iters": [x["newton_iters"] for x in res["stats"]],
        "linear_iters": [x["linear_iters"] for x in res["stats"]],
        "fp64": res["fp64"],
        "roofline": roof,
        "roofline_vcycle_smoother": roof_mg,
        "roofline_advect": roof_adv,
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": res["clocks"],
        "e2e": res["e2e"],
    }
    return line


def main():
    """Run the selected arm; under torchrun rank 0 prints the one JSON line."""
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_gpu(args, rank, world, local_rank)
    if rank != 0:
        return
    line = bench_line(args, res, world, load_peaks())
    if not args.no_cpu and not args.helium and world == 1:
        line["cpu_baseline"] = cpu_baseline(res["w"], args.newton_tol)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
