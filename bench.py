"""Benchmark: FP64 BDF2 projection steps of the 512 x 512 x 32 synthetic ocean basin.

A step is one pass of the whole hot path of Section 3's time loop: velocity right-hand side,
three velocity PCG solves (IC0), divergence right-hand side, the zero-mean pressure PCG
(vertical-line preconditioner), the pressure update and the lumped velocity correction. The loop
is spun up from rest (a BDF1 start step, then BDF2 steps) before the timed steps, which continue
it, so every timed step solves all four systems from a non-trivial state. The metric is the
algorithmic bandwidth of the steps' PCG iterations (GB/s), reported with its fraction of the
measured HBM peak; solves/s and latency come along. Operators (about 4.5 GB) exceed the 126 MB
L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only baseline this method has) on a bounded
window of the same basin, on one host core, running the same kind of steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG GB/s % of HBM peak; solves/s, p99 latency vs plain FP64 at 1e-8 residual"
WORKLOAD = "ocean basin 512x512 columns x 32 sigma layers, FP64 BDF2 projection steps of a spun-up time loop"
CPU_WINDOW = 64     # columns per side of the oracle's bounded sample (a few seconds per step on one core)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---- clocks during the timed region ------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="pm_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        try:
            self.proc.terminate()
            self.proc.wait(timeout=5)
        except Exception:
            pass
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = sorted(float(r[1]) for r in rows)
        out["sm_mhz"] = sm[len(sm) // 2]
        out["sm_max_mhz"] = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


# ---- the oracle's bounded sample (CPU baseline and reference arm) ------------------------------

def oracle_window_basin():
    """A CPU_WINDOW x CPU_WINDOW window of the same synthetic ocean basin (largest component)."""
    from workloads import ocean_basin
    from workloads.basins import _keep_largest_cell_component
    full = ocean_basin()
    m = full.mask
    best, bj, bi = -1, 0, 0
    for j0 in range(0, full.ny - CPU_WINDOW, 32):
        for i0 in range(0, full.nx - CPU_WINDOW, 32):
            s = int(m[j0:j0 + CPU_WINDOW, i0:i0 + CPU_WINDOW].sum())
            if s > best:
                best, bj, bi = s, j0, i0
    sl = (slice(bj, bj + CPU_WINDOW), slice(bi, bi + CPU_WINDOW))
    full.mask = _keep_largest_cell_component(m[sl].copy())
    full.depth = full.depth[sl].copy()
    full.coriolis = full.coriolis[sl].copy()
    full.theta = full.theta[(slice(None),) + sl].copy()
    full.nx = full.ny = CPU_WINDOW
    full.name = f"ocean512-window{CPU_WINDOW}x{CPU_WINDOW}x{full.nz}"
    return full


def oracle_step_bytes(n, rep):
    """Algorithmic PCG bytes of a step, the same per-row model as the GPU path."""
    spmv = 15 * 8 + 8 + 8
    per_ic0 = spmv + 48 + 2 * 8 * 8 + 4 * 8 + 16 + 24
    per_line = spmv + 48 + 3 * 8 + 8 + 24 + 8      # pressure: m'z adds m
    its_vel = sum(r.iters for r in rep.vel)
    return n * (its_vel * per_ic0 + rep.pres.iters * per_line)


def cpu_worker(steps: int, warmup: int):
    """The oracle's time loop on the window: a BDF1 start step and max(warmup, 1) - 1 more steps
    untimed, then `steps` timed BDF2 steps; prints one JSON line (GB/s, seconds per step)."""
    from oracle import fem, step
    basin = oracle_window_basin()
    ops = fem.assemble(basin)
    opts = step.StepOptions(vel_rtol=1e-8, pres_rtol=1e-8, vel_prec="ic0", pres_prec="line")
    st = step.initial_state(ops.n)
    for _ in range(max(warmup, 1)):
        step.project_step(ops, st, opts)
    rates, secs = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        rep = step.project_step(ops, st, opts)
        dt = time.perf_counter() - t0
        rates.append(oracle_step_bytes(ops.n, rep) / dt / 1e9)
        secs.append(dt)
    print(json.dumps({"gbs": sum(rates) / len(rates), "seconds": sum(secs) / len(secs), "n": ops.n,
                      "sample": basin.name, "iters": [r.iters for r in rep.vel] + [rep.pres.iters]}))


def run_cpu_oracle(steps: int, warmup: int):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--steps", str(steps),
                        "--warmup", str(warmup)], capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_cpu_oracle_all_cores(max_workers: int = 16):
    """The oracle on every host core at once: one single-threaded worker process per core, each
    running one projection step on the same window. Returns the aggregate algorithmic GB/s (all
    workers' bytes over the slowest worker's time) and the core count."""
    cores = min(len(os.sched_getaffinity(0)), max_workers)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--steps", "1", "--warmup", "0"]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for _ in range(cores)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=3600)
        if p.returncode != 0:
            raise RuntimeError("oracle worker failed:\n" + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    total_bytes = sum(o["gbs"] * o["seconds"] for o in outs)
    slowest = max(o["seconds"] for o in outs)
    return {"value": round(total_bytes / slowest, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} single-threaded oracle processes, one projection step each on "
                      f"{outs[0]['sample']} ({outs[0]['n']} nodes), concurrently",
            "seconds_slowest": round(slowest, 2)}


# ---- our arm -----------------------------------------------------------------------------------

# live timing classes of the library (index = KT_* value) and the kernels they stand for
KT_NAMES = ("k_cg_spmv", "k_cg_update", "k_cg_rho+k_cg_pupd", "k_ic0_sweep", "k_update_line")
SMS, FP64_FMA_PER_CLK_SM = 152, 2


def fp64_peak_tflops(sm_mhz):
    """FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA per SM per clock x 2 flop
    (GB300's nominal FP64 rate, 1.25 TFLOP/s at 2070 MHz)."""
    return SMS * FP64_FMA_PER_CLK_SM * 2 * float(sm_mhz) * 1e6 / 1e12


def roofline_of(kt, n, steps, ms_total, peak, peak_kind, sm_mhz=None):
    """Roofline of the dominant kernel class. kt: {class: (total ms, launches)} over `steps`
    steps of an n-row basin. Algorithmic bytes per launch per class (each array once); the FP64
    SpMV is bound by the FP64 pipe (ncu: 83 % busy, DRAM 44 %), so when it dominates it is
    reported as "alu" against the FP64 peak, with its HBM-equivalent rate beside it."""
    per_launch_bytes = {
        0: n * (15 * 8 + 8 + 8),            # SpMV: values, p (gathers cached), w
        1: n * (4 * 8 + 2 * 8),             # IC0 path update: x, r, p, w read; x, r written
        2: n * (3 * 8 + 8) / 2,             # (r, z) dot + p update, two launches
        3: n * (2 * 8 * 8 + 4 * 8) / 16,    # IC0 colour phase: F (8 per row per sweep), r / y / z
        4: n * (2 * 8 + 2 * 8 + 8 + 8 + 3 * 8 + 8 + 8),      # fused update + line solve: x, r r/w; p, w,
                                                              # 3 factors, m read; z written
    }
    spmv_flops = 2 * 16 * n                 # 15 slot FMAs and the (p, Ap) FMA per row
    live = {k: v for k, v in kt.items() if v[1] > 0}
    dom = max(live, key=lambda k: live[k][0])
    dom_ms, dom_launches = live[dom]
    avg_s = dom_ms * 1e-3 / dom_launches
    gbs = per_launch_bytes[dom] / avg_s / 1e9
    out = {"kernel": KT_NAMES[dom], "traffic": dram_traffic(KT_NAMES[dom]),
           "kernel_share_of_step": round(dom_ms / max(ms_total, 1e-9), 4)}
    if dom == 0:
        pk = fp64_peak_tflops(sm_mhz or 2070.0)
        tf = spmv_flops / avg_s / 1e12
        out.update({"bound": "alu", "achieved": round(tf, 4), "peak": round(pk, 4), "unit": "TFLOP/s",
                    "frac": round(tf / pk, 4),
                    "peak_source": f"derived: {SMS} SMs x {FP64_FMA_PER_CLK_SM} FP64 FMA/clk x 2 flop x "
                                   f"{sm_mhz or 2070.0:.0f} MHz (nominal FP64 1.25 TFLOP/s)",
                    "hbm_equivalent": {"achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                                       "frac": round(gbs / peak, 4), "peak_source": peak_kind}})
    else:
        out.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(gbs / peak, 4), "peak_source": peak_kind})
    out["classes_ms_per_step"] = {KT_NAMES[k]: round(v[0] / steps, 3) for k, v in kt.items()}
    out["classes"] = {KT_NAMES[k]: {"launches_per_step": v[1] // max(steps, 1),
                                    "us_per_launch": round(v[0] * 1e3 / v[1], 1),
                                    "gbs": round(per_launch_bytes[k] / (v[0] * 1e-3 / v[1]) / 1e9, 1),
                                    "frac": round(per_launch_bytes[k] / (v[0] * 1e-3 / v[1]) / 1e9 / peak, 4)}
                      for k, v in live.items()}
    return out


def kernel_source_hash(path: str, names) -> str:
    """sha256[:12] of the source text of the named device functions (each from its name at a
    definition to the matching closing brace), so that a traffic figure follows the kernel's own
    code rather than the whole file."""
    import hashlib
    import re
    with open(path) as fh:
        src = fh.read()
    parts = []
    for name in names:
        m = None
        for cand in re.finditer(r"\b" + re.escape(name) + r"\s*\(", src):
            head = src[max(0, cand.start() - 400):cand.start()]
            if "__global__" in head.split(";")[-1] or "__device__" in head.split(";")[-1]:
                m = cand
                break
        if m is None:
            raise ValueError(f"{name} not found in {path}")
        k = src.index("{", m.end())
        depth = 0
        for e in range(k, len(src)):
            depth += {"{": 1, "}": -1}.get(src[e], 0)
            if depth == 0:
                break
        parts.append(src[m.start():e + 1])
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()[:12]


def dram_traffic(kernel: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kernel` from the
    ncu summary in profiles/traffic.md, or None when the kernel's source (the functions listed
    beside the figure) has changed since the counters were taken (its hash is recorded there)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 5 and cells[0] == f"`{kernel}`":
                src = os.path.join(ROOT, "paper_1207_0486_gb300", "csrc", cells[2])
                names = [n.strip().strip("`") for n in cells[3].split(",")]
                try:
                    return int(cells[1]) if kernel_source_hash(src, names) == cells[4] else None
                except (OSError, ValueError):
                    return None
    return None


def _reduce(dist, v, op):
    """All-reduce one number over the replicas (NCCL on GPUs, gloo on CPU); v itself without
    a process group."""
    import torch
    if not dist:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _gather_max(dist, v):
    return _reduce(dist, v, dist.ReduceOp.MAX) if dist else v


def _gather_sum(dist, v):
    return _reduce(dist, v, dist.ReduceOp.SUM) if dist else v


def run_small_leg():
    """The 16x16x8 box (2,048 nodes): latency-bound, so reported as microseconds per solve and
    solves/s, not as a fraction of HBM. One solve per call to 1e-10 (FP64) or 1e-8 (mixed) from
    x = 0, seeded N(0, 1) right-hand sides; velocity u1 with IC0, pressure with the line
    preconditioner and with Jacobi. The mixed-precision rows are the same geometry with FP32 / BF16
    operator values (FP64 dots and refinement), with their error against the FP64 solution. The
    mms_* rows solve right-hand sides manufactured from a smooth seeded field u* (b = A u*, the
    small configuration's form) and report the error against u*."""
    import torch
    import paper_1207_0486_gb300 as pm
    from workloads import box_basin, manufactured_field, mms_modes

    basin = box_basin()
    op = pm.assemble_operator(basin)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1207)
    out = {"workload": "box 16x16x8 (2,048 nodes), x0 = 0, seeded N(0, 1) right-hand side; mms_* rows: "
                       "b = A u* for the seeded sinusoid field u* (workloads.manufactured_field)"}
    cases = [(pm.OP_VEL_U1, "velocity_ic0", pm.PREC_IC0, pm.FP64, 1e-10),
             (pm.OP_PRESSURE, "pressure_line", pm.PREC_LINE, pm.FP64, 1e-10),
             (pm.OP_PRESSURE, "pressure_jacobi", pm.PREC_JACOBI, pm.FP64, 1e-10),
             (pm.OP_VEL_U1, "velocity_ic0_fp64_1e-8", pm.PREC_IC0, pm.FP64, 1e-8),
             (pm.OP_VEL_U1, "velocity_ic0_fp32", pm.PREC_IC0, pm.FP32_REFINE, 1e-8),
             (pm.OP_VEL_U1, "velocity_ic0_bf16", pm.PREC_IC0, pm.BF16_REFINE, 1e-8),
             (pm.OP_PRESSURE, "pressure_line_fp64_1e-8", pm.PREC_LINE, pm.FP64, 1e-8),
             (pm.OP_PRESSURE, "pressure_line_fp32", pm.PREC_LINE, pm.FP32_REFINE, 1e-8),
             (pm.OP_PRESSURE, "pressure_line_bf16", pm.PREC_LINE, pm.BF16_REFINE, 1e-8)]
    rhs = {w: torch.randn(op.n, dtype=torch.float64, device="cuda", generator=gen) for w in (pm.OP_VEL_U1, pm.OP_PRESSURE)}
    ref = {}
    for which, label, prec, precision, rtol in cases:
        b = rhs[which]
        x = torch.zeros_like(b)
        opts = pm.Options(rtol=rtol, prec=prec, precision=precision, max_iter=100000, inner_rtol=1e-2)
        op.solve(which, b, x, opts)
        torch.cuda.synchronize()
        reps = 50
        t0 = time.perf_counter()
        for _ in range(reps):
            x.zero_()
            st = op.solve(which, b, x, opts)
        dt = (time.perf_counter() - t0) / reps
        row = {"us_per_solve": round(dt * 1e6, 1), "solves_per_s": round(1.0 / dt, 1), "iters": int(st.iters),
               "rel_residual_true": float(f"{st.rel_residual_true:.3e}")}
        if precision == pm.FP64 and rtol == 1e-8:
            ref[which] = x.clone()
        elif precision != pm.FP64:
            r = ref[which]
            row["rel_err_vs_fp64"] = float(f"{float((x - r).norm() / r.norm()):.3e}")
            row["outer_iters"] = int(st.outer_iters)
        out[label] = row
    # manufactured right-hand sides: b = A u*, so the exact solution is u* (the pressure's is u*
    # minus its M-weighted mean, m = M 1)
    ci, cj = op.columns()
    us = torch.from_numpy(manufactured_field(basin, ci, cj, mms_modes())).cuda()
    m = torch.zeros_like(us)
    op.spmv(pm.OP_MASS, torch.ones_like(us), m)
    for which, label, prec in ((pm.OP_VEL_U1, "mms_velocity_ic0", pm.PREC_IC0),
                               (pm.OP_PRESSURE, "mms_pressure_line", pm.PREC_LINE)):
        b = torch.zeros_like(us)
        op.spmv(which, us, b)
        exact = us - (m @ us) / m.sum() if which == pm.OP_PRESSURE else us
        x = torch.zeros_like(us)
        opts = pm.Options(rtol=1e-10, prec=prec, max_iter=100000)
        op.solve(which, b, x, opts)
        torch.cuda.synchronize()
        reps = 50
        t0 = time.perf_counter()
        for _ in range(reps):
            x.zero_()
            st = op.solve(which, b, x, opts)
        dt = (time.perf_counter() - t0) / reps
        out[label] = {"us_per_solve": round(dt * 1e6, 1), "solves_per_s": round(1.0 / dt, 1), "iters": int(st.iters),
                      "rel_residual_true": float(f"{st.rel_residual_true:.3e}"),
                      "rel_err_vs_manufactured": float(f"{float((x - exact).norm() / exact.norm()):.3e}")}
    op.close()
    return out


def run_batched_leg(dist, world, rank):
    """Many basins x 4 right-hand sides (3 velocity components + pressure) in one persistent,
    graph-captured launch (FP32 inner PCG, FP64 refinement to 1e-8, autotuned tile x block), against
    the same systems solved one after another by the single-system FP64 path. Basins are dealt to
    replicas round-robin."""
    import torch
    import paper_1207_0486_gb300 as pm
    from workloads import batch_basins

    basins = batch_basins()[rank::world]
    ops = [pm.assemble_operator(b) for b in basins]
    which = [pm.OP_VEL_U1, pm.OP_VEL_U2, pm.OP_VEL_U3, pm.OP_PRESSURE]
    sys_ops = [op for op in ops for _ in which]
    sys_w = [w for _ in ops for w in which]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1207 + rank)
    bs = [torch.randn(op.n, dtype=torch.float64, device="cuda", generator=gen) for op in sys_ops]
    xs = [torch.zeros_like(b) for b in bs]
    opts = pm.Options(rtol=1e-8, prec=pm.PREC_LINE, precision=pm.FP32_REFINE, inner_rtol=1e-4, max_iter=200000)
    batch = pm.Batch(sys_ops, sys_w, opts, autotune=True)
    info = batch.info()
    batch.solve(bs, xs, allow_not_converged=True)  # warm-up (graph capture)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    stats = batch.solve(bs, xs, allow_not_converged=True)
    torch.cuda.synchronize()
    t_batch = _gather_max(dist, time.perf_counter() - t0)
    batch.close()
    seq = pm.Options(rtol=1e-8, prec=pm.PREC_LINE, precision=pm.FP64, max_iter=200000, max_restarts=5)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    sst = [op.solve(w, b, x, seq, allow_not_converged=True) for op, w, b, x in zip(sys_ops, sys_w, bs, xs)]
    torch.cuda.synchronize()
    t_seq = _gather_max(dist, time.perf_counter() - t0)
    nsys = _gather_sum(dist, len(sys_ops))
    nodes = _gather_sum(dist, sum(op.n for op in ops))
    bad = _gather_sum(dist, sum(1 for s in stats if s.status != pm.PM_OK))
    # the same batch with BF16 operator values (FP32 vectors, FP64 refinement), autotuned too
    bf = pm.Batch(sys_ops, sys_w, pm.Options(rtol=1e-8, prec=pm.PREC_LINE, precision=pm.BF16_REFINE,
                                             inner_rtol=1e-4, max_iter=200000), autotune=True)
    bf.solve(bs, xs, allow_not_converged=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    bf_stats = bf.solve(bs, xs, allow_not_converged=True)
    torch.cuda.synchronize()
    t_bf = _gather_max(dist, time.perf_counter() - t0)
    bf.close()
    bf16 = {"batched_s": round(t_bf, 3), "solves_per_s": round(nsys / t_bf, 2),
            "speedup_vs_sequential_fp64": round(t_seq / t_bf, 3), "iters_max": max(int(s.iters) for s in bf_stats),
            "failed": int(_gather_sum(dist, sum(1 for s in bf_stats if s.status != pm.PM_OK)))}
    mass = _consistent_mass_batch(dist, ops, gen)
    for op in ops:
        op.close()
    return {"workload": "64 seeded basins, sides log-uniform 48-384, 8-48 layers, 4 right-hand sides each",
            "systems": int(nsys), "nodes": int(nodes), "precision": "fp32 inner / fp64 refinement, rtol 1e-8",
            "preconditioner": "vertical-line block-Jacobi",
            "batched_s": round(t_batch, 3), "sequential_fp64_s": round(t_seq, 3),
            "solves_per_s": round(nsys / t_batch, 2), "sequential_solves_per_s": round(nsys / t_seq, 2),
            "speedup_vs_sequential_fp64": round(t_seq / t_batch, 3), "failed": int(bad),
            "iters_max": max(int(s.iters) for s in stats), "sequential_iters_max": max(int(s.iters) for s in sst),
            "autotuned": info, "bf16_refine": bf16, "consistent_mass_ic0": mass}


def _consistent_mass_batch(dist, ops, gen):
    """The consistent-mass velocity correction of every basin (M u = rhs for the three components,
    IC0-PCG to 1e-10) in one batched launch, FP64 and FP32-with-refinement, against the same solves
    one after another on the single-system FP64 path."""
    import torch
    import paper_1207_0486_gb300 as pm

    sys_ops = [op for op in ops for _ in range(3)]
    bs = [torch.randn(op.n, dtype=torch.float64, device="cuda", generator=gen) for op in sys_ops]
    xs = [torch.zeros_like(b) for b in bs]
    sys_w = [pm.OP_MASS] * len(sys_ops)
    out = {"systems": int(_gather_sum(dist, len(sys_ops))), "preconditioner": "multicolour IC0", "rtol": 1e-10,
           "workload": "the batched leg's 64 basins, M u_c = rhs_c for c = 1, 2, 3, seeded N(0, 1) right-hand sides"}
    for label, precision in (("fp64", pm.FP64), ("fp32_refine", pm.FP32_REFINE)):
        batch = pm.Batch(sys_ops, sys_w, pm.Options(rtol=1e-10, prec=pm.PREC_IC0, precision=precision,
                                                    inner_rtol=1e-4, max_iter=10000), autotune=True)
        batch.solve(bs, xs, allow_not_converged=True)  # warm-up (graph capture)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        stats = batch.solve(bs, xs, allow_not_converged=True)
        torch.cuda.synchronize()
        t = _gather_max(dist, time.perf_counter() - t0)
        batch_info = batch.info()
        batch.close()
        out[label] = {"batched_s": round(t, 4), "solves_per_s": round(out["systems"] / t, 1), "autotuned": batch_info,
                      "failed": int(_gather_sum(dist, sum(1 for st in stats if st.status != pm.PM_OK))),
                      "iters_max": max(int(st.iters) for st in stats)}
    seq = pm.Options(rtol=1e-10, prec=pm.PREC_IC0, precision=pm.FP64, max_iter=10000, max_restarts=5)
    for op, b, x in zip(sys_ops[:1], bs[:1], xs[:1]):  # factors built outside the timed region
        op.solve(pm.OP_MASS, b, x, seq, allow_not_converged=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sst = [op.solve(pm.OP_MASS, b, x, seq, allow_not_converged=True) for op, b, x in zip(sys_ops, bs, xs)]
    torch.cuda.synchronize()
    t_seq = _gather_max(dist, time.perf_counter() - t0)
    out["sequential_fp64_s"] = round(t_seq, 4)
    out["sequential_iters_max"] = max(int(st.iters) for st in sst)
    for label in ("fp64", "fp32_refine"):
        out[label]["speedup_vs_sequential_fp64"] = round(t_seq / out[label]["batched_s"], 3)
    return out


def run_serving_leg(dist, world, rank, n_requests):
    """Poisson request stream (200 req/s, lognormal basin sizes, 1-4 right-hand sides, 8 sessions
    of consecutive steps) served by continuous batching (FP32 inner / FP64 refinement to 1e-8)
    and by plain serial FP64 solves, in real time on this GPU; sessions are dealt to replicas."""
    import numpy as np
    from paper_1207_0486_gb300.serve import GpuBackend, Scheduler, shard
    from workloads import request_stream

    def serve(correction, max_rhs):
        sessions, reqs = request_stream(n_requests=n_requests, max_rhs=max_rhs)
        mine = [reqs[i] for i in shard(sessions, reqs, rank, world)]
        out = {}
        for mode in ("continuous", "serial"):
            be = GpuBackend(slots=64, nz_cap=48, correction=correction)
            if dist:
                dist.barrier()
            rep = Scheduler(be, sessions, mine, slots=64, quantum=16, mode=mode).run()
            be.close()
            lat = rep.latencies_ms().tolist()
            if dist:
                gathered = [None] * world
                dist.all_gather_object(gathered, lat)
                lat = [v for part in gathered for v in part]
            span = _gather_max(dist, rep.makespan)
            solves = _gather_sum(dist, rep.solves)
            sm = rep.summary()
            out[mode] = {"solves": int(solves), "solves_per_s": round(solves / span, 2),
                         "p50_ms": round(float(np.percentile(lat, 50)), 1),
                         "p99_ms": round(float(np.percentile(lat, 99)), 1),
                         "makespan_s": round(span, 3), "mean_iters": round(sm["mean_iters"], 1),
                         "failed_solves": int(_gather_sum(dist, sm["failed_solves"])),
                         "host_seconds": sm["host_seconds"]}
        c, s_ = out["continuous"], out["serial"]
        out["workload"] = (f"{n_requests} requests, Poisson 200 req/s, lognormal nodes (median 1.5e5), "
                           f"1-{max_rhs} rhs, 8 concurrent sessions of consecutive steps, operators and Krylov "
                           "state resident")
        out["continuous"]["precision"] = "fp32 inner / fp64 refinement (restart at 1e-4), rtol 1e-8"
        out["serial"]["precision"] = "fp64, rtol 1e-8"
        out["throughput_vs_serial_fp64"] = round(c["solves_per_s"] / s_["solves_per_s"], 3)
        out["p99_vs_serial_fp64"] = round(c["p99_ms"] / s_["p99_ms"], 3)
        return out

    out = serve("lumped", 4)
    cons = serve("consistent", 7)
    cons["systems"] = ("u1, u2, u3 and pressure (line preconditioner), three consistent-mass corrections "
                       "M u_c = rhs_c (IC0), all in one persistent kernel")
    out["consistent_mass_correction"] = cons
    return out


def _step_stats(stats):
    """Iterations, residuals and bytes of one step's four solves (u1, u2, u3, q)."""
    return {"iters": [int(s.iters) for s in stats[:4]],
            "restarts": [int(s.outer_iters) for s in stats[:4]],
            "rel_residual_true": [float(f"{s.rel_residual_true:.3e}") for s in stats[:4]],
            "rel_residual_floor": [float(f"{s.rel_residual_floor:.3e}") for s in stats[:4]],
            "status": [int(s.status) for s in stats[:4]],
            "bytes": sum(s.bytes_moved for s in stats[:4]),
            "solves_with_work": sum(1 for s in stats[:4] if s.iters > 0)}


def run_resident_leg(args):
    """A fixed load on the resident solve server, for timing and profiling its persistent kernel:
    `--systems` copies of one box basin's pressure (or velocity) system kept resident and run for
    `--quanta` launches of `--quantum` iterations, with a tolerance out of reach so that every
    system stays active. Prints microseconds per iteration of the timed launches."""
    import torch

    import paper_1207_0486_gb300 as pm
    from workloads import box_basin, random_vector

    torch.cuda.set_device(0)
    op = pm.assemble_operator(box_basin(nh=args.nh, nz=args.nz))
    prc = pm.FP32_REFINE if args.precision == "fp32" else pm.FP64
    srv = pm.Server(slots=max(args.systems, 1), nz_cap=max(args.nz, 2),
                    opts=pm.Options(rtol=1e-300, prec=pm.PREC_LINE, precision=prc, max_iter=10 ** 8,
                                    inner_rtol=1e-2), tile_cols=64, block=128)
    b = torch.from_numpy(random_vector(op.n, 1207)).cuda()
    xs = [torch.zeros(op.n, dtype=torch.float64, device="cuda") for _ in range(args.systems)]
    ws = [torch.empty(srv.workspace_bytes(op), dtype=torch.uint8, device="cuda") for _ in range(args.systems)]
    for k in range(args.systems):
        srv.admit(op, args.which, b, xs[k], ws[k])
    srv.run(1)
    t0 = time.perf_counter()
    active = [srv.run(args.quantum) for _ in range(args.quanta)]
    us = (time.perf_counter() - t0) / (args.quanta * args.quantum) * 1e6
    srv.close()
    op.close()
    print(json.dumps({"resident_load": {"systems": args.systems, "basin": f"box{args.nh}x{args.nh}x{args.nz}",
                                        "which": args.which, "precision": args.precision,
                                        "us_per_iteration": round(us, 1), "active": min(active)}}))


def run_batch_load(args):
    """A batched solve for timing and profiling the persistent kernel: the first basins of the
    batched 64-basin set, up to `--max-rows` rows, one system of `--which` each (4: the
    consistent mass matrix), preconditioner `--prec`, FP64 or FP32 refinement, rtol 1e-10. Solves
    twice (the first captures the graph); the second solve's iteration launch is the fourth
    launch of k_batch. Prints the second solve's time."""
    import torch

    import paper_1207_0486_gb300 as pm
    from workloads import batch_basins

    torch.cuda.set_device(0)
    ops, rows = [], 0
    for b in batch_basins():
        op = pm.assemble_operator(b)
        if rows + op.n > args.max_rows:
            op.close()
            continue
        ops.append(op)
        rows += op.n
    prec = {"ic0": pm.PREC_IC0, "jacobi": pm.PREC_JACOBI, "line": pm.PREC_LINE}[args.prec]
    prc = pm.FP32_REFINE if args.precision == "fp32" else pm.FP64
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    bs = [torch.randn(op.n, dtype=torch.float64, device="cuda", generator=gen) for op in ops]
    xs = [torch.zeros_like(b) for b in bs]
    bt = pm.Batch(ops, [args.which] * len(ops), pm.Options(rtol=1e-10, prec=prec, precision=prc, max_iter=10000))
    bt.solve(bs, xs, allow_not_converged=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = bt.solve(bs, xs, allow_not_converged=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    info = bt.info()
    bt.close()
    for op in ops:
        op.close()
    print(json.dumps({"batch_load": {"systems": len(ops), "rows": rows, "which": args.which, "prec": args.prec,
                                     "precision": args.precision, "seconds": round(dt, 4),
                                     "iters_max": max(int(s.iters) for s in st), **info}}))


def run_ours(args):
    import numpy as np
    import torch

    import paper_1207_0486_gb300 as pm
    from paper_1207_0486_gb300 import api
    from workloads import ocean_basin

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()

    basin = ocean_basin() if args.nx == 512 else ocean_basin(nx=args.nx, ny=args.nx, dx=1e4 * 512 / args.nx)
    launches_start = pm.kernel_launch_count()
    op = pm.assemble_operator(basin)
    st = pm.State(op)
    t1 = torch.from_numpy(op.column_field(basin.theta[0])).cuda()
    t2 = torch.from_numpy(op.column_field(basin.theta[1])).cuda()
    vel = pm.Options(rtol=1e-8, prec=pm.PREC_IC0, max_iter=500000)
    pres = pm.Options(rtol=1e-8, prec=pm.PREC_LINE, max_iter=500000)

    def one_step(v=vel, p=pres, allow=False):
        return pm.project_step(op, st, t1, t2, v, p, allow_not_converged=allow)

    # spin-up: the time loop from rest (BDF1 start step, then BDF2), untimed; the timed steps
    # continue it, so every step solves all four systems from a non-trivial state
    spin = max(args.warmup, 2)
    for _ in range(spin):
        one_step()
    torch.cuda.synchronize()
    snap = st.snapshot()

    clocks = ClockSampler(dev_index)
    clocks.start()
    time.sleep(0.3)
    api.kernel_timing(True)
    launches0 = pm.kernel_launch_count()
    launches_before = launches0 - launches_start
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record()
    all_stats = []
    for k in range(args.steps):
        all_stats.append(one_step())
        ev[k + 1].record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = pm.kernel_launch_count() - launches0
    ms_total = ev[0].elapsed_time(ev[-1])
    ms_steps = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    kt = {k: api.kernel_timing_get(k) for k in (api.KT_SPMV, api.KT_UPDATE, api.KT_PUPDATE, api.KT_IC0,
                                                 api.KT_LINE)}
    api.kernel_timing(False)
    clk = clocks.stop()

    per_step = [_step_stats(s) for s in all_stats]
    bytes_step = sum(p["bytes"] for p in per_step) / args.steps
    solves_step = sum(p["solves_with_work"] for p in per_step) / args.steps
    ms_step = ms_total / args.steps
    if dist:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * bytes_step / (ms_step * 1e-3) / 1e9

    # roofline of the dominant kernel class, timed live with events on the solve stream
    n = op.n
    peak, peak_kind = measured_peaks()
    roofline = roofline_of(kt, n, args.steps, ms_total, peak, peak_kind, (clk or {}).get("sm_mhz"))

    # end to end through the C ABI with host buffers: the same timed steps replayed from the
    # snapshot, theta in and (u1, u2, u3, p) out every step; diagnostics read after each step
    e2e = None
    time_loop = None
    fp64_fields_at = {}
    k_m = max(1, min(args.steps, 3))
    if not args.no_e2e:
        st.restore(snap)
        th_h = [torch.from_numpy(op.column_field(basin.theta[c])).pin_memory() for c in range(2)]
        outs_h = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(4)]
        th_d = [torch.empty(op.ncols, dtype=torch.float64, device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        e2e_bytes = 0.0
        for k in range(args.steps):
            for c in range(2):
                th_d[c].copy_(th_h[c], non_blocking=True)
            s_e = pm.project_step(op, st, th_d[0], th_d[1], vel, pres)
            e2e_bytes += sum(s.bytes_moved for s in s_e[:4])
            for h, d in zip(outs_h, st.get()):
                h.copy_(d, non_blocking=True)
        f1.record()
        torch.cuda.synchronize()
        ms_e2e = f0.elapsed_time(f1) / args.steps
        if dist:
            t = torch.tensor([ms_e2e], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        e2e = {"value": round(world * (e2e_bytes / args.steps) / (ms_e2e * 1e-3) / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": 2 * op.ncols * 8, "d2h_bytes_per_step": 4 * n * 8,
               "ms_per_step": round(ms_e2e, 3), "steps": args.steps,
               "note": "the same timed steps, replayed from a snapshot of the spun-up state"}

    # the time loop's monitors and its checkpoint (replaying the timed steps once more)
    if not args.no_e2e:
        st.restore(snap)
        diags = []
        for k in range(args.steps):
            one_step()
            if k + 1 == k_m:
                fp64_fields_at[k_m] = [t.clone() for t in st.get()]
            diags.append(st.diagnostics())
        time_loop = {"first_timed_step": spin, "steps": args.steps,
                     "kinetic_energy": [float(f"{d['kinetic_energy']:.6e}") for d in diags],
                     "div_u": [float(f"{d['div_u']:.3e}") for d in diags],
                     "div_u_tilde": [float(f"{d['div_u_tilde']:.3e}") for d in diags],
                     "p_mean": [float(f"{d['p_mean']:.3e}") for d in diags]}
        try:
            with tempfile.TemporaryDirectory() as td:
                path = os.path.join(td, "state.pmck")
                c0 = time.perf_counter()
                st.save(path)
                c1 = time.perf_counter()
                probe = pm.State(op)
                probe.load_checkpoint(path)
                c2 = time.perf_counter()
                same = all(bool(torch.equal(a, b)) for a, b in zip(st.snapshot()[0], probe.snapshot()[0]))
                time_loop["checkpoint"] = {"bytes": os.path.getsize(path), "save_s": round(c1 - c0, 3),
                                           "load_s": round(c2 - c1, 3), "round_trip_identical": same}
                probe.close()
        except Exception as ex:  # reported, never fatal for the headline number
            time_loop["checkpoint"] = {"error": str(ex)[:200]}

    # the same steps with mixed precision (form 1): FP32 / BF16 operator values and inner PCG,
    # FP64 dots, alpha/beta and outer refinement to the same rule; error vs the FP64 steps
    mixed = {}
    if not args.no_mixed and fp64_fields_at:
        ref = fp64_fields_at[k_m]
        ms_fp64 = sum(ms_steps[:k_m]) / k_m
        for label, prc in (("fp32", pm.FP32_REFINE), ("bf16", pm.BF16_REFINE)):
            vm = pm.Options(rtol=1e-8, prec=pm.PREC_IC0, precision=prc, max_iter=60000)
            pmo = pm.Options(rtol=1e-8, prec=pm.PREC_LINE, precision=prc, max_iter=60000)
            try:
                st.restore(snap)      # untimed first pass: operator copies, factors, workspace
                one_step(vm, pmo, True)
            except pm.PMError as ex:
                mixed[label] = {"error": str(ex)[:200]}
                continue
            st.restore(snap)
            torch.cuda.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record()
            m_stats = []
            for _ in range(k_m):
                m_stats.append(one_step(vm, pmo, True))
            g1.record()
            torch.cuda.synchronize()
            ms_m = g0.elapsed_time(g1) / k_m
            got = st.get()
            errs = {}
            for nm, g, o in zip(("u", "v", "w", "p"), got, ref):
                scale = float(o.abs().max())
                errs[nm] = 0.0 if scale == 0 else float((g - o).abs().max() / scale)
            last_m = m_stats[-1]
            mixed[label] = {"steps": k_m, "ms_per_step": round(ms_m, 3), "fp64_ms_per_step_same_steps": round(ms_fp64, 3),
                            "solves_per_s": round(sum(_step_stats(s)["solves_with_work"] for s in m_stats) / (k_m * ms_m * 1e-3), 3),
                            "speedup_vs_fp64_step": round(ms_fp64 / ms_m, 3),
                            "pcg_gbs": round(sum(sum(x.bytes_moved for x in s[:4]) for s in m_stats) / (k_m * ms_m * 1e-3) / 1e9, 1),
                            "inner_iters": [int(s.iters) for s in last_m[:4]],
                            "outer_iters": [int(s.outer_iters) for s in last_m[:4]],
                            "fp64_iters": per_step[k_m - 1]["iters"],
                            "rel_residual_true": [float(f"{s.rel_residual_true:.3e}") for s in last_m[:4]],
                            "rel_residual_floor": [float(f"{s.rel_residual_floor:.3e}") for s in last_m[:4]],
                            "status": [int(s.status) for s in last_m[:4]],
                            "per_field_max_rel_err_vs_fp64": {k: float(f"{v:.3e}") for k, v in errs.items()}}

    small = None
    if not args.no_small:
        try:
            small = run_small_leg()
        except Exception as ex:  # reported, never fatal for the headline number
            small = {"error": str(ex)[:300]}
    batched = None
    if not args.no_batch:
        try:
            batched = run_batched_leg(dist, world, rank)
        except Exception as ex:  # reported, never fatal for the headline number
            batched = {"error": str(ex)[:300]}
    serving = None
    if not args.no_serve:
        try:
            serving = run_serving_leg(dist, world, rank, args.serve_requests)
        except Exception as ex:
            serving = {"error": str(ex)[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            w = run_cpu_oracle(1, 0)
            cpu = {"value": round(w["gbs"], 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                   "sample": f"one oracle BDF2 projection step (FP64, IC0 velocity, line-preconditioned pressure, "
                             f"rtol 1e-8) after a BDF1 start step, on {w['sample']} ({w['n']} of the workload's "
                             f"{n} nodes), {w['seconds']:.1f} s; GB/s = the step's algorithmic PCG bytes / time",
                   "seconds_per_step": round(w["seconds"], 2), "iters": w["iters"]}
        except Exception as ex:  # the GPU number stands on its own
            cpu = {"value": None, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"[:200]}
        try:
            cpu["all_cores"] = run_cpu_oracle_all_cores()
        except Exception as ex:
            cpu["all_cores"] = {"error": str(ex)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded ocean basin: smoothed-noise land mask, sum-of-Gaussians bathymetry)",
            "config": {"workload": WORKLOAD, "basin": basin.name, "nodes": n, "columns": op.ncols,
                       "velocity": "IC0-PCG x3 (multicolour), rtol 1e-8",
                       "pressure": "vertical-line block-Jacobi PCG, zero-mean multiplier, rtol 1e-8 or the FP64 "
                                   "floor once restarts stall",
                       "correction": "lumped mass", "spin_up_steps": spin,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "operators 4.5 GB > L2, no flush needed"},
            "pct_hbm_peak": round(value / world / peak, 4),
            "solves_per_s": round(world * solves_step / (ms_step * 1e-3), 3),
            "iters": per_step[-1]["iters"],
            "rel_residual_true": per_step[-1]["rel_residual_true"],
            "rel_residual_floor": per_step[-1]["rel_residual_floor"],
            "per_step": {"ms": [round(v, 2) for v in ms_steps], "iters": [p["iters"] for p in per_step],
                         "restarts": [p["restarts"] for p in per_step]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "gpu_launches_before_timed": int(launches_before),
            "time_loop": time_loop,
            "mixed_precision": mixed,
            "small_case": small,
            "batched": batched,
            "serving": serving,
            "clocks": clk,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_reference(args):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    w = run_cpu_oracle(args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(w["gbs"], 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(w["seconds"] * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": w["sample"]},
        "cpu_baseline": {"value": round(w["gbs"], 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: one oracle projection step on {w['sample']} ({w['n']} nodes)"},
        "e2e": {"value": round(w["gbs"], 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--cpu-worker", action="store_true")
    ap.add_argument("--resident-load", action="store_true",
                    help="time a fixed load on the resident solve server (see run_resident_leg)")
    ap.add_argument("--systems", type=int, default=9)
    ap.add_argument("--nh", type=int, default=100)
    ap.add_argument("--nz", type=int, default=30)
    ap.add_argument("--which", type=int, default=3,
                    help="resident / batch load: 0-2 velocity component, 3 pressure, 4 mass")
    ap.add_argument("--quanta", type=int, default=3)
    ap.add_argument("--quantum", type=int, default=8)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--batch-load", action="store_true",
                    help="time one batched solve of the first batched basins (see run_batch_load)")
    ap.add_argument("--max-rows", type=int, default=12_000_000)
    ap.add_argument("--prec", default="ic0", choices=["ic0", "jacobi", "line"])
    ap.add_argument("--nx", type=int, default=512,
                    help="basin columns per side (512 = the benchmark workload; smaller for profiling)")
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args.steps, args.warmup)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.resident_load:
        run_resident_leg(args)
        return
    if args.batch_load:
        run_batch_load(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
