#!/usr/bin/env python
"""Benchmark of the panel-interaction hot path on one GB300 (or N replicas).

Workload (one "step"): the large matrix-free run -- the multi-domain device
(conductor sphere R=1 at V0=1, floating torus (R=2, r=0.3) with its
charge-neutrality row, dielectric cylinder eps_r=4) meshed with about 200k flat
triangles (seeded), then
  1. the matrix-free solve: GMRES on the mixed-precision matvec (FP32 regular
     pairs, FP64 near pairs and Arnoldi) inside an FP64-accurate iterative
     refinement to a relative residual of 1e-8,
  2. the surface field E+ at every centroid,
  3. phi and E at 1e6 points uniform in [-4,4]^3 outside the conductors.
Metric: Ginteractions/s = (target, triangle) pairs evaluated by all kernel
launches of the step / step time (whole job over all ranks).  The same step on
the 20k device, and the plain FP64 form of both, are reported beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMRES solve+field-eval time & Ginteractions/s, FP64 vs mixed on GB300 at rel err 1e-6"
UNIT = "Ginteractions/s"
FLOPS_PER_PAIR_OP = 18        # phi+E per (target, quadrature node): 3 sub, 5 for r^2, w/r, phi+=, 1/r^2, w/r^3, 6 in the 3 fma of E
PHI_FLOPS_PER_PAIR_OP = 10    # phi alone: 3 sub, 5 for r^2, w/r, phi+=
FP32_LANES_PER_SM = 128
TOL = 1e-8
C5_SCALE = (200000 / 20068.0) ** 0.5   # mesh scale of the ~200k-triangle device


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=None,
                    help="mesh scale (default: ~200k triangles, trace mode ~20k; 1.0: ~20k)")
    ap.add_argument("--points", type=int, default=1000000)
    ap.add_argument("--no-c2", action="store_true", help="skip the 20k-device comparison")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--far32-variant", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="FP32 regular-pair kernel variant (0: tuned at context creation)")
    ap.add_argument("--mode", default="step", choices=["step", "matvec", "batch", "report", "trace"],
                    help="matvec: only W+K mixed matvecs of the workload (a small case for ncu); "
                         "batch: the uneven device family solved and traced by the batched calls; "
                         "report: per-configuration times and errors of both GPU forms and the oracle")
    ap.add_argument("--report-configs", default="c1,c2,c3,bushing,p1,c5", help="report mode: configurations")
    ap.add_argument("--c5-lines", type=int, default=64, help="report mode: field lines traced on c5")
    ap.add_argument("--lines", type=int, default=512, help="trace mode: field lines")
    ap.add_argument("--seed-radius", type=float, default=1.05,
                    help="trace mode: radius of the sphere the Fibonacci seeds lie on")
    ap.add_argument("--batch-points", type=int, default=10000,
                    help="batch mode: field points per mesh for bem_batch_eval_field")
    ap.add_argument("--max-steps", type=int, default=200000, help="trace mode: RK4 step limit per line")
    ap.add_argument("--no-trace", action="store_true", help="skip the field-line block of the step's line")
    ap.add_argument("--trace-cluster", default="0",
                    help="trace mode: CTAs per tracer cluster (0 automatic); a comma list runs each")
    ap.add_argument("--instances", type=int, default=64, help="batch mode: meshes in the family")
    ap.add_argument("--nrhs", type=int, default=4, help="batch mode: right-hand sides per mesh")
    ap.add_argument("--seeds", type=int, default=8, help="batch mode: field lines traced per mesh")
    ap.add_argument("--n-min", type=int, default=2000)
    ap.add_argument("--n-max", type=int, default=30000)
    return ap.parse_args()


def run_matvec(args):
    """W + K mixed-precision matrix-free products on the workload's mesh."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem
    mesh, _ = workload(args)
    ctx = bem.Context(mesh, far32_variant=args.far32_variant)
    x = torch.randn(ctx.nunk, dtype=torch.float64, device="cuda", generator=None)
    for _ in range(args.warmup + args.steps):
        ctx.matvec(x, bem.MIXED)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "matvec", "triangles": ctx.np, "launches": ctx.counters()["kernel_launches"]}))
    ctx.close()


def workload(args, scale=None, points=None):
    from paper_2003_12663_gb300 import meshgen as mg
    scale = scale if scale is not None else (args.scale if args.scale is not None else C5_SCALE)
    mesh = mg.device_mesh(scale=scale, seed=2)
    pts = mg.device_box_points(points if points is not None else args.points, seed=5)
    return mesh, pts


def workload_name(mesh):
    big = mesh.np_ > 100000
    return (("large matrix-free run: " if big else "") +
            f"multi-domain device (conductor sphere, floating torus, dielectric cylinder) at "
            f"{mesh.np_} triangles; mixed solve to {TOL}, surface field, field at box points")


def config_of(args, mesh, n_points, extra=None):
    cfg = {"workload": workload_name(mesh),
           "triangles": int(mesh.np_), "unknowns": int(mesh.n_unknowns),
           "counts_sphere_torus_cylinder": list(mesh.info["counts"]),
           "eval_points": int(n_points), "gmres_tol": TOL, "solver": "GMRES(100)+FP64-accurate refinement",
           "far_rule": "3x3 Duffy/Gauss, eta=4", "l2": "flushed (256 MB write) before every step",
           "parallelism": f"replicas x{args.gpus}"}
    if mesh.np_ > 100000:
        cfg["reading"] = ("the large configuration's device is the three-body device of the 20k "
                          "configuration refined to ~200k triangles; its field lines are reported by "
                          "--mode report, not in this step")
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return dist if world > 1 else None


def dist_max(dist, value, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(dist):
    if dist is not None:
        dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ roofline inputs
def fp32_peak_derived(num_sms):
    """FP32 CUDA-core peak from unit counts: SMs x 128 lanes x 2 flop (FFMA) x max SM clock."""
    mhz = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            mhz = float(json.load(open(p)).get("sm_max_mhz"))
        except Exception:
            mhz = None
    if not mhz:
        mhz = 2070.0
    return num_sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, mhz


def fp32_peak(bem, num_sms):
    """(peak TFLOP/s, basis): the FP32 rate measured by bem_measure_peaks (paired and
    scalar FP32 multiply-add chains at full occupancy), else the derived figure."""
    derived, mhz = fp32_peak_derived(num_sms)
    try:
        m = bem.measure_peaks()
    except Exception as e:  # the measurement is reported, never silently replaced
        return derived, f"derived ({num_sms} SMs x 128 lanes x 2 x {mhz:.0f} MHz); measurement failed: {e}", None
    basis = (f"measured: bem_measure_peaks, FP32 multiply-add chains at full occupancy "
             f"(paired {m['fp32_tflops']:.1f}, scalar {m['fp32_scalar_tflops']:.1f} TFLOP/s); "
             f"derived {derived:.1f} ({num_sms} SMs x 128 lanes x 2 x {mhz:.0f} MHz)")
    return m["fp32_tflops"], basis, m


def far_kernel_hash():
    """sha256[:16] of the packed FP32 kernel's source (from its section marker to
    the next kernel): the committed ncu counters stay valid while it is unchanged."""
    src = open(os.path.join(ROOT, "paper_2003_12663_gb300", "csrc", "far.cu")).read()
    a = src.index("// ---------------------------------------------------------------- packed FP32")
    b = src.index("k_far64(", a)
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def committed_traffic(profile):
    """DRAM bytes per launch of the FP32 regular-pair kernel, copied from the committed
    ncu summary profiles/<profile> when it was captured on the current kernel source
    (its 'k_far32p source sha256[:16]' line); else None.  This is a stored capture,
    not a measurement of this run, and the bench line says so."""
    p = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(": ", 1)
            vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
    if vals.get("k_far32p source sha256[:16]") != far_kernel_hash():
        return None
    try:
        return float(vals["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ CPU oracle
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_oracle_rate(mesh, seconds, seed=0, threads=0):
    """Oracle throughput (pairs/s) on a bounded sample: the pair integrals of a
    seeded sample of collocation rows against all triangles (classification,
    Duffy/Gauss rule, closed form), OpenMP on `threads` host cores (0: all)."""
    from oracle import oracle as O
    before = O.set_threads(threads) if threads > 0 else None
    try:
        P = O.Problem(mesh, eta=4.0, g=3)
        rng = np.random.default_rng(seed)
        rows = 4
        while True:
            idx = np.sort(rng.choice(P.N, size=min(rows, P.N), replace=False))
            t0 = time.perf_counter()
            P.pair_block(P.centroids[idx], idx, want_G=True)
            t = time.perf_counter() - t0
            if t > seconds / 4 or rows >= P.N:
                break
            rows *= 2
        # the timed sample
        idx = np.sort(rng.choice(P.N, size=min(rows * 2, P.N), replace=False))
        t0 = time.perf_counter()
        P.pair_block(P.centroids[idx], idx)
        t = time.perf_counter() - t0
    finally:
        if before is not None:
            O.set_threads(before)
    return len(idx) * P.N / t, len(idx), t


def events_ms(fn, stream, n, flush=None):
    """CUDA-event times (ms) of n calls of fn on stream, L2 flushed before each."""
    import torch
    out = []
    for _ in range(n):
        if flush is not None:
            flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    dist_barrier(dist)
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem

    mesh, pts = workload(args)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    peak, peak_basis, peaks = fp32_peak(bem, props.multi_processor_count)
    ctx = bem.Context(mesh, timing=1, far32_variant=args.far32_variant)
    Q = ctx.params.far_order ** 2
    pts_d = torch.tensor(pts, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()
    out = {}

    def step():
        u, it, rel = ctx.solve(bem.MIXED, tol=TOL)
        Es = ctx.surface_field(u[0], bem.MIXED)
        phi, E = ctx.eval_field(u[0], pts_d, bem.MIXED)
        out.update(u=u, it=it, rel=rel, Es=Es, phi=phi, E=E)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.reset_counters()
    clocks = ClockSampler(local) if local == 0 else None
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if clocks:
        clocks.start()
    dist_barrier(dist)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.add_(1.0)
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    dist_barrier(dist)
    clk = clocks.stop() if clocks else None
    times = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ms = dist_max(dist, float(np.mean(times)), dev)
    cnt = ctx.counters()
    pairs_step = sum(cnt["pairs"]) / args.steps
    value = world * pairs_step / (ms * 1e-3) / 1e9
    launches = cnt["kernel_launches"]

    # roofline of the dominant kernel: the FP32 regular-pair kernel
    far_pairs = cnt["pairs"][1] - cnt["near_pairs"][1]
    # tiles of conductor rows sum phi alone: 10 of the 18 flops of a pair-op
    phi_far = cnt["phi_pairs"][1] * (far_pairs / max(cnt["pairs"][1], 1))
    flops = Q * (FLOPS_PER_PAIR_OP * far_pairs - (FLOPS_PER_PAIR_OP - PHI_FLOPS_PER_PAIR_OP) * phi_far)
    far_ms = cnt["far_ms"][1]
    achieved = flops / (far_ms * 1e-3) / 1e12 if far_ms > 0 else None
    n_launch = max(cnt["far_launches"][1], 1)
    profile = "far32_device200k.md" if mesh.np_ > 100000 else "far32_device20k.md"
    traffic = committed_traffic(profile)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_source": (f"copied from the committed ncu capture profiles/{profile} "
                                   f"(same k_far32p source hash {far_kernel_hash()}), not measured in this run"
                                   if traffic is not None else
                                   f"null: no ncu capture of the current k_far32p source in profiles/{profile}"),
                "kernel": ("k_far32 (scalar)" if cnt["far32_variant"] == 1 else
                           f"k_far32p (packed f32x2, {cnt['far32_variant']} target pairs/thread)")
                          + ": FP32 regular pairs, phi+E",
                "peak_basis": peak_basis,
                "flops_basis": f"{Q} nodes x ({FLOPS_PER_PAIR_OP} x far pairs - 8 x far pairs of phi-only tiles)",
                "flops_per_launch": flops / n_launch, "avg_launch_ms": far_ms / n_launch,
                "launches_timed": cnt["far_launches"][1],
                "phi_only_pair_share": cnt["phi_pairs"][1] / max(cnt["pairs"][1], 1),
                "fast_chunk_share": (cnt["fast_chunks32p"] / cnt["chunks32p"]) if cnt["chunks32p"] else None,
                "fp64_far_ms_per_step": cnt["far_ms"][0] / args.steps,
                "df_residual_far_ms_per_step": cnt["far_ms"][2] / args.steps,
                "fp32_far_ms_per_step": far_ms / args.steps}
    if peaks:
        roofline["fp64_peak_tflops_measured"] = peaks["fp64_tflops"]
    roofline["tuning"] = ctx.tuning()   # the kernel shape bem_create's tuner chose, and the candidates' times

    rel = out["rel"][0]
    # the true residual of the step's result, with the double-FP32 product (untimed)
    b0 = ctx.rhs()[0]
    true_rel = ((b0 - ctx.matvec(out["u"][0], precision=bem.DF)).norm() / b0.norm()).item()
    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32 regular pairs + f64",
              "data": "synthetic (seeded meshes and points)",
              "config": config_of(args, mesh, len(pts),
                                  {"gmres_iters_per_step": cnt["gmres_iters"] / args.steps,
                                   "products_per_step": {"mixed": cnt["matvecs"][1] / args.steps,
                                                         "double_fp32_residual": cnt["matvecs"][2] / args.steps},
                                   "relres": rel, "relres_recomputed_double_fp32": true_rel,
                                   "pairs_per_step": pairs_step}),
              "roofline": roofline, "gpu_launches": launches}
    if clk:
        result["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}

    if not args.no_fp64_form and rank == 0:
        result["fp64_form"] = fp64_form(args, bem, ctx, mesh, pts_d, out, cnt, ms, stream, flush)
    if not args.no_c2 and rank == 0 and mesh.np_ > 100000:
        result["c2"] = c2_block(args, bem, stream, flush)

    if not args.no_trace and rank == 0:
        result["trace"] = trace_block(args, bem)

    if not args.no_e2e:
        result["e2e"] = e2e_block(args, bem, mesh, pts, dev, flush, dist, world, pairs_step)

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        rate, rows, secs = cpu_oracle_rate(mesh, args.cpu_seconds)
        rate1, rows1, secs1 = cpu_oracle_rate(mesh, args.cpu_seconds / 2, seed=1, threads=1)
        result["cpu_baseline"] = {"value": rate / 1e9, "unit": UNIT, "cores": os.cpu_count(),
                                  "kind": "oracle", "cpu_model": cpu_model(),
                                  "sample": f"oracle pair integrals (classification, Duffy/Gauss, closed form; "
                                            f"FP64, OpenMP) of {rows} seeded collocation rows x {mesh.np_} "
                                            f"triangles, {secs:.1f} s",
                                  "one_thread": {"value": rate1 / 1e9, "unit": UNIT, "cores": 1,
                                                 "sample": f"{rows1} rows x {mesh.np_} triangles, {secs1:.1f} s"}}
    ctx.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def fp64_form(args, bem, ctx, mesh, pts_d, out, cnt, ms_mixed, stream, flush):
    """The plain FP64 GPU form of the same step.  On the ~200k device it would take
    about half an hour, so it is extrapolated from measured parts: one FP64 product
    (timed), times the products of the mixed step (its GMRES products and refinement
    residuals) plus one for the surface field, plus the FP64 field at a sample of the
    points scaled to all of them.  Smaller meshes run it in full (median of 5)."""
    import torch
    M = pts_d.shape[0]
    if mesh.np_ <= 100000:
        res = {}

        def step64():
            u64, it64, rel64 = ctx.solve(bem.FP64, tol=TOL)
            ctx.surface_field(u64[0], bem.FP64)
            phi, E = ctx.eval_field(u64[0], pts_d, bem.FP64)
            res.update(u=u64, it=it64, rel=rel64, E=E)

        t = events_ms(step64, stream, 5, flush)
        ms64 = float(np.median(t))
        du = (torch.linalg.norm(out["u"][0] - res["u"][0]) / torch.linalg.norm(res["u"][0])).item()
        dE = ((out["E"] - res["E"]).abs().max() / res["E"].abs().max()).item()
        return {"ms_per_step": ms64, "runs_ms": t, "statistic": "median of 5", "gmres_iters": res["it"],
                "relres": res["rel"][0], "mixed_speedup": ms64 / ms_mixed,
                "sigma_rel_l2_mixed_vs_fp64": du, "E_rel_mixed_vs_fp64": dE}
    u = out["u"][0]
    t_mv = events_ms(lambda: ctx.matvec(u, bem.FP64), stream, 2, flush)
    t_mv64 = float(np.median(t_mv))
    products = (cnt["matvecs"][1] + cnt["matvecs"][2]) / args.steps
    n_sub = min(M, 20000)
    sub = pts_d[:n_sub]
    holder = {}
    t_ev = events_ms(lambda: holder.update(r=ctx.eval_field(u, sub, bem.FP64)), stream, 1, flush)[0]
    _, E64 = holder["r"]
    dE = ((out["E"][:n_sub] - E64).abs().max() / E64.abs().max()).item()
    ms64 = (products + 1) * t_mv64 + t_ev * (M / n_sub)
    return {"ms_per_step": ms64, "extrapolated": True,
            "basis": f"(products of the mixed step {products:.0f} + 1 surface field) x one FP64 product "
                     f"{t_mv64:.0f} ms (timed) + FP64 field at {n_sub} of the {M} points "
                     f"{t_ev:.0f} ms (timed) x {M / n_sub:.0f}",
            "fp64_product_ms": t_mv, "fp64_eval_sample_ms": t_ev, "mixed_speedup": ms64 / ms_mixed,
            "E_rel_mixed_vs_fp64_on_sample": dE}


def p1_vertex_weights(nodes, tri6, nv, body, nbody, g=8):
    """w[b, v] = integral of the linear basis function of vertex v over the curved
    six-node triangles of body b: a g x g Gauss rule on the square mapped onto each
    triangle (xi = s(1 - t), eta = s t, Jacobian s), times the area element
    |dy/dxi x dy/deta| of the quadratic map."""
    x, wx = np.polynomial.legendre.leggauss(g)
    x, wx = 0.5 * (x + 1.0), 0.5 * wx
    s, t = np.meshgrid(x, x, indexing="ij")
    ws = (wx[:, None] * wx[None, :] * s).ravel()
    xi, eta = (s * (1.0 - t)).ravel(), (s * t).ravel()
    l0 = 1.0 - xi - eta
    dxi = np.stack([1.0 - 4.0 * l0, 4.0 * xi - 1.0, 0.0 * xi, 4.0 * (l0 - xi), 4.0 * eta, -4.0 * eta], 1)
    deta = np.stack([1.0 - 4.0 * l0, 0.0 * xi, 4.0 * eta - 1.0, -4.0 * xi, 4.0 * xi, 4.0 * (l0 - eta)], 1)
    lam = np.stack([l0, xi, eta], 1)
    out = np.zeros((nbody, nv))
    for T in range(len(tri6)):
        P = nodes[tri6[T]]
        J = np.linalg.norm(np.cross(dxi @ P, deta @ P), axis=1)
        np.add.at(out[body[T]], tri6[T, :3], (ws * J) @ lam)
    return out


def trace_block(args, bem):
    """Field lines beside the step (untimed by the step's clock, CUDA events of their own):
    c3's 256 Fibonacci lines on the 1,280-triangle sphere (h = 1e-3, r_max = 10), and
    1,024 lines seeded on |x| = 1.05 around the conductor sphere of the 20k device; both
    mixed, each after a warm-up call on 8 lines."""
    import torch
    from paper_2003_12663_gb300 import meshgen as mg
    out = {}
    for key, mesh, seeds in (("c3_sphere_256_lines", mg.sphere_mesh(3), mg.fibonacci_seeds(256)),
                             ("device20k_1024_lines", mg.device_mesh(1.0, seed=2),
                              mg.fibonacci_seeds(1024, radius=1.05))):
        ctx = bem.Context(mesh)
        u, _, _ = ctx.solve(bem.MIXED, tol=1e-10)
        sd = torch.tensor(seeds)
        ctx.trace_lines(u[0], sd[:8], bem.MIXED)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        K, st, ns, _ = ctx.trace_lines(u[0], sd, bem.MIXED)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        steps = int(ns.sum().item())
        Q = ctx.params.far_order ** 2
        out[key] = {"triangles": int(mesh.np_), "lines": len(seeds), "ms": ms, "rk4_steps": steps,
                    "field_pair_ops_per_s": steps * 4 * mesh.np_ * Q / (ms * 1e-3),
                    "max_steps_of_a_line": int(ns.max().item()),
                    "lines_reaching_r_max": int((st == 1).sum().item())}
        ctx.close()
    out["note"] = ("field pair-ops: RK4 steps x 4 field evaluations x triangles x nodes "
                   "(event re-steps not counted)")
    return out


def c2_block(args, bem, stream, flush):
    """The same step on the 20k device, both GPU forms, each the median of 5 runs."""
    import torch
    mesh, pts = workload(args, scale=1.0, points=100000)
    pts_d = torch.tensor(pts, device="cuda")
    c = bem.Context(mesh, timing=1)
    res = {}

    def mk(prec, key):
        def f():
            u, it, rel = c.solve(prec, tol=TOL)
            c.surface_field(u[0], prec)
            phi, E = c.eval_field(u[0], pts_d, prec)
            res[key] = (u, it, rel, E)
        return f

    mk(bem.MIXED, "mixed")()
    c.reset_counters()
    t32 = events_ms(mk(bem.MIXED, "mixed"), stream, 5, flush)
    cnt = c.counters()
    pairs_step = sum(cnt["pairs"]) / 5
    c.reset_counters()
    t64 = events_ms(mk(bem.FP64, "fp64"), stream, 5, flush)
    cnt64 = c.counters()
    pairs64 = sum(cnt64["pairs"]) / 5
    u32, it32, rel32, E32 = res["mixed"]
    u64, it64, rel64, E64 = res["fp64"]
    c.close()
    # the mixed form with every refinement residual in FP64, or in double-FP32, instead
    # of the default (the first in double-FP32, the later ones updated)
    alt = {}
    for key, mode in (("mixed_with_fp64_residual", bem.RESIDUAL_FP64),
                      ("mixed_with_double_fp32_residual_every_step", bem.RESIDUAL_DF)):
        cf = bem.Context(mesh, residual=mode)
        resf = {}

        def stepf():
            u, it, rel = cf.solve(bem.MIXED, tol=TOL)
            cf.surface_field(u[0], bem.MIXED)
            phi, E = cf.eval_field(u[0], pts_d, bem.MIXED)
            resf.update(u=u, it=it, rel=rel, E=E)

        stepf()
        tf = events_ms(stepf, stream, 3, flush)
        cf.close()
        alt[key] = {
            "ms_per_step": float(np.median(tf)), "runs_ms": tf, "statistic": "median of 3",
            "gmres_iters": resf["it"], "relres": resf["rel"][0],
            "sigma_rel_l2_vs_fp64": (torch.linalg.norm(resf["u"][0] - u64[0]) / torch.linalg.norm(u64[0])).item(),
            "E_rel_vs_fp64": ((resf["E"] - E64).abs().max() / E64.abs().max()).item(),
            "sigma_rel_l2_vs_default_residual":
                (torch.linalg.norm(resf["u"][0] - u32[0]) / torch.linalg.norm(u32[0])).item()}
    m32, m64 = float(np.median(t32)), float(np.median(t64))
    out = {"workload": workload_name(mesh), "triangles": int(mesh.np_), "eval_points": len(pts),
           "statistic": "median of 5 runs (CUDA events), L2 flushed before each",
           "mixed": {"ms_per_step": m32, "runs_ms": t32, "gmres_iters": it32, "relres": rel32[0],
                     "residual": "first in double-FP32, later ones updated with the correction's mixed product",
                     "value": pairs_step / (m32 * 1e-3) / 1e9, "unit": UNIT},
           "fp64": {"ms_per_step": m64, "runs_ms": t64, "gmres_iters": it64, "relres": rel64[0],
                    "value": pairs64 / (m64 * 1e-3) / 1e9, "unit": UNIT},
           "mixed_speedup": m64 / m32,
           "sigma_rel_l2_mixed_vs_fp64": (torch.linalg.norm(u32[0] - u64[0]) / torch.linalg.norm(u64[0])).item(),
           "E_rel_mixed_vs_fp64": ((E32 - E64).abs().max() / E64.abs().max()).item()}
    out.update(alt)
    return out


def e2e_block(args, bem, mesh, pts, dev, flush, dist, world, pairs_step):
    """The step end to end through the C ABI with host buffers: bem_create from the
    host mesh, host-to-device copy of the points, solve, surface field, field,
    device-to-host copy of sigma, E+ and (phi, E)."""
    import torch
    M = len(pts)
    X_h = torch.tensor(pts).pin_memory()
    phi_h = torch.empty(M, dtype=torch.float64).pin_memory()
    E_h = torch.empty((M, 3), dtype=torch.float64).pin_memory()
    Es_h = torch.empty((mesh.np_, 3), dtype=torch.float64).pin_memory()
    u_h = torch.empty(mesh.n_unknowns, dtype=torch.float64).pin_memory()

    def e2e_step():
        c2 = bem.Context(mesh)           # host mesh -> device inside bem_create
        p_d = X_h.to(dev, non_blocking=True)
        u, it, rel = c2.solve(bem.MIXED, tol=TOL)
        Es = c2.surface_field(u[0], bem.MIXED)
        phi, E = c2.eval_field(u[0], p_d, bem.MIXED)
        u_h.copy_(u[0], non_blocking=True)
        Es_h.copy_(Es, non_blocking=True)
        phi_h.copy_(phi, non_blocking=True)
        E_h.copy_(E, non_blocking=True)
        torch.cuda.synchronize()
        c2.close()

    n_e2e = 2
    dist_barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        flush.add_(1.0)
        e2e_step()
    torch.cuda.synchronize()
    dist_barrier(dist)
    e2e_ms = dist_max(dist, (time.perf_counter() - t0) * 1e3 / n_e2e, dev)
    h2d = mesh.X.size * 8 + mesh.tri.size * 4 + mesh.region.size * 4 + pts.size * 8
    d2h = mesh.n_unknowns * 8 + mesh.np_ * 24 + M * 32
    return {"value": world * pairs_step / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "runs": n_e2e,
            "includes": "bem_create from host mesh, H2D points, solve, surface field, eval, D2H"}

# ------------------------------------------------------------------ batched family
def run_batch(args):
    """The uneven device family (seeded: triangle counts uniform in [n_min, n_max],
    2% vertex jitter) with nrhs Dirichlet right-hand sides each (V0 in 1, 0.5, -1, 2):
    the batched solve (persistent regular-pair launch in a graph-replayed Arnoldi
    iteration, FP64-accurate refinement to 1e-8) and the batched tracer on a sample
    of Fibonacci seeds per mesh.  One JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem
    from paper_2003_12663_gb300 import meshgen as mg

    meshes = mg.device_family(args.instances, n_min=args.n_min, n_max=args.n_max, seed=7)
    ctxs = [bem.Context(m) for m in meshes]
    nr = args.nrhs
    vals = [1.0, 0.5, -1.0, 2.0][:nr]
    V0 = []
    for m in meshes:
        V = np.zeros((nr, len(m.regions)))
        for r, v in enumerate(vals):
            V[r, 0] = v                     # region 0: the conductor sphere
        V0.append(torch.tensor(V, device="cuda"))
    B = bem.Batch(ctxs, nrhs=nr, timing=True)
    Q = ctxs[0].params.far_order ** 2
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(3)
    xs = [torch.tensor(rng.standard_normal((nr, c.nunk)), device=dev) for c in ctxs]

    # the persistent regular-pair kernel alone (event-timed inside the library)
    for _ in range(2):
        B.matvec(xs)
    B.reset_counters()
    n_mv = 5
    for _ in range(n_mv):
        flush.add_(1.0)
        B.matvec(xs)
    cm = B.counters()
    near = sum(c.near_pairs for c in ctxs)
    far_pairs = cm["pairs"] / max(cm["far_launches"], 1) - near
    flops = far_pairs * (FLOPS_PER_PAIR_OP * Q + 8 * nr)
    far_ms = cm["far_ms"] / max(cm["far_timed"], 1)
    props = torch.cuda.get_device_properties(dev)
    peak, peak_basis, _ = fp32_peak(bem, props.multi_processor_count)
    achieved = flops / (far_ms * 1e-3) / 1e12

    def solve():
        return B.solve(V0, tol=TOL, check=False)

    for _ in range(args.warmup):
        solve()
    for c in ctxs:
        c.reset_counters()
    B.reset_counters()
    clocks = ClockSampler(0)
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        us, iters, rel = solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    cb = B.counters()
    resid_pairs = sum(sum(c.counters()["pairs"]) for c in ctxs)
    ms = float(np.mean(times))
    value = (cb["rhs_pairs"] + resid_pairs) / args.steps / (ms * 1e-3) / 1e9

    # the field at box points of every mesh, one persistent launch per chunk of points
    Mb = args.batch_points
    bpts = [torch.tensor(mg.device_box_points(Mb, seed=100 + k), device=dev) for k in range(len(ctxs))]
    u_b = [u[0] for u in us]
    B.eval_field(u_b, bpts, bem.MIXED)       # warm-up
    B.reset_counters()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.eval_field(u_b, bpts, bem.MIXED)
    e1.record(stream)
    torch.cuda.synchronize()
    ev_ms = e0.elapsed_time(e1)
    ev_pairs = B.counters()["eval_pairs"]
    # field lines: seeds on a sphere of radius 1.05 around the conductor, mixed form
    L = args.seeds
    seeds = [mg.fibonacci_seeds(L, radius=1.05) for _ in ctxs]
    u1 = [u[0] for u in us]
    B.trace(u1, seeds, bem.MIXED)            # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    K, st, ns = B.trace(u1, seeds, bem.MIXED)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tms = e0.elapsed_time(e1)
    steps_total = int(sum(n.sum().item() for n in ns))
    st_all = torch.cat(st).cpu().numpy()
    tri = [c.np for c in ctxs]
    out = {"mode": "batch", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "dtype": "f32 regular pairs + f64",
           "data": "synthetic (seeded meshes)",
           "config": {"workload": f"device family: {args.instances} meshes, {min(tri)}-{max(tri)} triangles "
                                  f"(sum {sum(tri)}), {nr} Dirichlet right-hand sides each, tol {TOL}",
                      "instances": args.instances, "nrhs": nr, "triangles_total": sum(tri),
                      "sum_N_squared": int(sum(t * t for t in tri)), "l2": "flushed (256 MB write) between steps"},
           "solve": {"ms": ms, "arnoldi_steps_per_step": cb["arnoldi_steps"] / args.steps,
                     "graph_launches_per_step": cb["graph_launches"] / args.steps,
                     "kernel_launches_per_step": cb["kernel_launches"] / args.steps,
                     "batched_rhs_pairs_per_step": cb["rhs_pairs"] / args.steps,
                     "residual_pairs_per_step": resid_pairs / args.steps,
                     "relres_max": float(rel.max()), "iters_max": int(iters.max())},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": f"k_bfar<{Q},{nr}>: persistent batched FP32 regular pairs, phi+E, {nr} rhs",
                        "flops_per_launch": flops, "avg_launch_ms": far_ms, "peak_basis": peak_basis,
                        "flops_basis": f"far pairs x ({FLOPS_PER_PAIR_OP} x {Q} nodes + 8 x {nr} rhs)"},
           "eval": {"points_per_mesh": Mb, "ms": ev_ms, "pairs": ev_pairs,
                    "ginteractions_per_s": ev_pairs / (ev_ms * 1e-3) / 1e9,
                    "call": "bem_batch_eval_field (mixed): one persistent regular-pair launch for all meshes"},
           "trace": {"lines": int(L * len(ctxs)), "ms": tms, "lines_per_s": L * len(ctxs) / (tms * 1e-3),
                     "rk4_steps": steps_total,
                     "status_counts": {int(k): int(v) for k, v in zip(*np.unique(st_all, return_counts=True))},
                     "sample": f"{L} Fibonacci seeds per mesh (radius 1.05), h=1e-3, r_max=10"}}
    if clk:
        out["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    B.close()
    for c in ctxs:
        c.close()
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ field lines alone
def run_trace(args):
    """bem_trace_lines on the device workload (mixed form): --lines Fibonacci seeds on
    |x| = 1.05 around the conductor sphere, h = 1e-3, r_max = 10; one warm-up call on
    8 lines, then the timed call.  Reports lines/s and field-evaluation pair-ops/s."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem
    from paper_2003_12663_gb300 import meshgen as mg
    mesh = mg.device_mesh(args.scale if args.scale is not None else 1.0, seed=2)
    seeds = torch.tensor(mg.fibonacci_seeds(args.lines, radius=args.seed_radius))
    for ncl in [int(v) for v in str(args.trace_cluster).split(",")]:
        ctx = bem.Context(mesh, trace_cluster=ncl)
        u, _, _ = ctx.solve(bem.MIXED, tol=TOL)
        ctx.trace_lines(u[0], seeds[:8], bem.MIXED, max_steps=args.max_steps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        K, st, ns, xe = ctx.trace_lines(u[0], seeds, bem.MIXED, max_steps=args.max_steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        steps = int(ns.sum().item())
        Q = ctx.params.far_order ** 2
        print(json.dumps({"mode": "trace", "triangles": ctx.np, "lines": args.lines,
                          "seed_radius": args.seed_radius, "trace_cluster": ncl, "ms": ms,
                          "lines_per_s": args.lines / (ms * 1e-3), "rk4_steps": steps,
                          "field_pair_ops_per_s": steps * 4 * ctx.np * Q / (ms * 1e-3),
                          "K_sum": float(K.sum().item()), "max_steps_of_a_line": int(ns.max().item()),
                          "status_counts": {int(k): int(v) for k, v in
                                            zip(*np.unique(st.cpu().numpy(), return_counts=True))}}), flush=True)
        ctx.close()


# ------------------------------------------------------------------ per-configuration report
def K_sphere_closed(V0=1.0, c=1e-2, E0=0.5, d=0.1, rmax=10.0):
    """K along a radial line from the unit sphere at V0 (continuum field V0 x / |x|^3):
    int_1^rs c (V0/r^2 - E0)^2 dr - d (rmax - rs), rs = sqrt(V0/E0)."""
    rs = (V0 / E0) ** 0.5
    F = lambda r: c * (-V0 * V0 / (3 * r ** 3) + 2 * V0 * E0 / r + E0 * E0 * r)
    return F(rs) - F(1.0) - d * (rmax - rs)


def run_report(args):
    """One JSON line per configuration: set-up / solve / field / trace / adjoint times
    of the FP64 and mixed GPU forms (CUDA events), the oracle's time on a stated
    sample (host cores), and the errors against closed forms and the oracle."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem
    from paper_2003_12663_gb300 import meshgen as mg
    from oracle import oracle as O
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) * 1e3

    def emit(d):
        d["cores"] = os.cpu_count()
        print(json.dumps(d), flush=True)

    want = set(args.report_configs.split(","))
    if "c1" in want:
        mesh = mg.sphere_mesh(3)
        pts = mg.sphere_eval_points(1, 1000, 1000)
        pts_d = torch.tensor(pts, device="cuda")
        P = O.Problem(mesh, eta=4.0, g=3)
        A_o, t_asm = wall(lambda: P.assemble())
        u_o, t_lu = wall(lambda: np.linalg.solve(A_o, P.rhs()))
        (phi_o, E_o), t_fo = wall(lambda: P.field(u_o, pts))
        out = {"config": "c1 sphere, 1,280 triangles, V0=1, tol 1e-10, 2,000 points",
               "oracle_ms": {"assemble": t_asm, "lu_solve": t_lu, "field": t_fo}}
        for name, prec in (("fp64", bem.FP64), ("mixed", bem.MIXED)):
            ctx, t_set = wall(lambda: bem.Context(mesh))
            _, t_rows = timed(lambda: ctx.assemble_rows(precision=prec))
            (u, it, rel), t_sol = timed(lambda: ctx.solve(prec, tol=1e-10))
            (phi, E), t_ev = timed(lambda: ctx.eval_field(u[0], pts_d, prec))
            ug, phig, Eg = u[0].cpu().numpy(), phi.cpu().numpy(), E.cpu().numpy()
            inside = np.linalg.norm(pts, axis=1) < 1.0
            out[name] = {"setup_ms": t_set, "assemble_rows_ms": t_rows, "solve_ms": t_sol, "iters": it,
                         "eval_ms": t_ev, "relres": rel[0],
                         "sigma_rel_l2_vs_oracle": float(np.linalg.norm(ug - u_o) / np.linalg.norm(u_o)),
                         "sigma_rms_vs_exact_1": float(np.sqrt(np.mean((ug - 1.0) ** 2))),
                         "phi_inside_max_dev_from_1": float(np.abs(phig[inside] - 1.0).max()),
                         "E_inside_max": float(np.linalg.norm(Eg[inside], axis=1).max()),
                         "E_rel_vs_oracle": float(np.abs(Eg - E_o).max() / np.abs(E_o).max())}
            ctx.close()
        emit(out)
    if "c2" in want:
        mesh = mg.device_mesh(1.0, seed=2)
        pts = mg.device_box_points(100000, seed=5)
        pts_d = torch.tensor(pts, device="cuda")
        out = {"config": f"c2 device, {mesh.np_} triangles, tol 1e-8, 1e5 points"}
        res = {}
        for name, prec in (("fp64", bem.FP64), ("mixed", bem.MIXED)):
            ctx, t_set = wall(lambda: bem.Context(mesh))
            (u, it, rel), t_sol = timed(lambda: ctx.solve(prec, tol=TOL))
            Es, t_sf = timed(lambda: ctx.surface_field(u[0], prec))
            (phi, E), t_ev = timed(lambda: ctx.eval_field(u[0], pts_d, prec))
            res[name] = (u[0], E)
            out[name] = {"setup_ms": t_set, "solve_ms": t_sol, "iters": it, "relres": rel[0],
                         "surface_field_ms": t_sf, "eval_ms": t_ev}
            ctx.close()
        u64, E64 = res["fp64"]
        um, Em = res["mixed"]
        out["mixed"]["sigma_rel_l2_vs_fp64"] = (torch.linalg.norm(um - u64) / torch.linalg.norm(u64)).item()
        out["mixed"]["E_rel_vs_fp64"] = ((Em - E64).abs().max() / E64.abs().max()).item()
        # oracle: pair integrals of a seeded sample of rows, extrapolated to the N^2 pairs
        rate, rows, secs = cpu_oracle_rate(mesh, 8.0)
        out["oracle"] = {"pairs_per_s": rate, "sample": f"{rows} rows x {mesh.np_} triangles, {secs:.1f} s",
                         "one_product_s_extrapolated": mesh.np_ ** 2 / rate}
        sel = np.random.default_rng(9).choice(len(pts), 500, replace=False)
        P = O.Problem(mesh, eta=4.0, g=3)
        _, E_o = P.field(u64.cpu().numpy(), pts[sel])
        out["fp64"]["E_rel_vs_oracle_500pts"] = float(np.abs(E64.cpu().numpy()[sel] - E_o).max() / np.abs(E_o).max())
        out["mixed"]["E_rel_vs_oracle_500pts"] = float(np.abs(Em.cpu().numpy()[sel] - E_o).max() / np.abs(E_o).max())
        emit(out)
    if "c3" in want:
        mesh = mg.sphere_mesh(3)
        seeds = torch.tensor(mg.fibonacci_seeds(256))
        Kc = K_sphere_closed()
        dKc = (K_sphere_closed(1.0 + 1e-6) - K_sphere_closed(1.0 - 1e-6)) / 2e-6
        out = {"config": "c3 sphere 1,280 triangles, 256 Fibonacci lines, h=1e-3, r_max=10",
               "K_closed_per_line": Kc, "dK_dV0_closed_per_line": dKc}
        ctx = bem.Context(mesh)
        for name, prec in (("fp64", bem.FP64), ("mixed", bem.MIXED)):
            (u, it, rel), t_sol = timed(lambda: ctx.solve(prec, tol=1e-12 if prec == bem.FP64 else 1e-10))
            (K, st, ns, xe), t_tr = timed(lambda: ctx.trace_lines(u[0], seeds, prec))
            w = torch.ones(256, dtype=torch.float64, device="cuda")
            (Ka, gX, gV0, geps), t_adj = timed(lambda: ctx.adjoint(u[0], seeds, w, prec))
            Kn = K.cpu().numpy()
            out[name] = {"solve_ms": t_sol, "trace_ms": t_tr, "adjoint_ms": t_adj,
                         "rk4_steps": int(ns.sum().item()), "status_1": int((st == 1).sum().item()),
                         "K_sum": float(Kn.sum()), "K_mean_abs_err_vs_closed": float(np.abs(Kn - Kc).mean()),
                         "dK_dV0_per_line": gV0[0].item() / 256}
        # oracle tracer on 4 of the lines (FP64 field of the method), extrapolated to 256
        P = O.Problem(mesh, eta=4.0, g=3)
        u64, _, _ = ctx.solve(bem.FP64, tol=1e-12)
        (Ko, so, no, xo), t_o = wall(lambda: P.trace(u64[0].cpu().numpy(), mg.fibonacci_seeds(256)[:4]))
        out["oracle"] = {"trace_4_lines_ms": t_o, "trace_256_lines_s_extrapolated": t_o * 64 / 1e3}
        ctx.close()
        emit(out)
    if "bushing" in want:
        # thin floating sheets (Eq. sheets): rod at 1, four floating foils, grounded
        # outer foil; foil potentials and net charges at ~21k triangles
        mesh = mg.bushing_mesh(1.0)
        a_ = mesh.X[mesh.tri[:, 1]] - mesh.X[mesh.tri[:, 0]]
        b_ = mesh.X[mesh.tri[:, 2]] - mesh.X[mesh.tri[:, 0]]
        area = 0.5 * np.linalg.norm(np.cross(a_, b_), axis=1)
        out = {"config": f"bushing analogue, {mesh.np_} triangles (rod, 4 floating foils, grounded foil), "
                         f"tol {TOL}"}
        res = {}
        for name, prec in (("fp64", bem.FP64), ("mixed", bem.MIXED)):
            ctx, t_set = wall(lambda: bem.Context(mesh))
            (u, it, rel), t_sol = timed(lambda: ctx.solve(prec, tol=TOL))
            ug = u[0].cpu().numpy()
            q = ug[: mesh.np_] * area
            q_rod = float(np.sum(q[mesh.region == 0]))
            res[name] = ug
            out[name] = {"setup_ms": t_set, "solve_ms": t_sol, "iters": it, "relres": rel[0],
                         "foil_V": [float(v) for v in ug[mesh.np_:]],
                         "foil_net_charge_over_rod": [float(np.sum(q[mesh.region == f + 1]) / q_rod)
                                                      for f in range(4)]}
            ctx.close()
        out["mixed"]["sigma_rel_l2_vs_fp64"] = float(np.linalg.norm(res["mixed"] - res["fp64"]) /
                                                     np.linalg.norm(res["fp64"]))
        small = mg.bushing_mesh(0.25)
        Ps = O.Problem(small, eta=4.0, g=3)
        (u_o), t_o = wall(lambda: Ps.solve())
        ctx = bem.Context(small)
        u_s, _, _ = ctx.solve(bem.MIXED, tol=1e-10)
        ctx.close()
        rate, rows, secs = cpu_oracle_rate(mesh, 8.0)
        out["oracle"] = {"small_case": f"{small.np_} triangles: assemble + LU {t_o:.0f} ms",
                         "small_case_foil_V": [float(v) for v in u_o[small.np_:]],
                         "small_case_mixed_gpu_foil_V": [float(v) for v in u_s[0].cpu().numpy()[small.np_:]],
                         "pairs_per_s": rate, "sample": f"{rows} rows x {mesh.np_} triangles, {secs:.1f} s",
                         "one_product_s_extrapolated": mesh.np_ ** 2 / rate}
        emit(out)
    if "p1" in want:
        # the paper's own discretisation: curved six-node triangles, P1 at the vertices
        for level in (3, 4):
            nodes, tri6, nv = mg.quadratic_sphere(level)
            body = np.zeros(len(tri6), np.int32)
            regs = [{"kind": "conductor", "V0": 1.0}]
            ctx, t_set = wall(lambda: bem.P1Context(nodes, tri6, nv, body, regs))
            res = {}
            for name, prec in (("fp64", bem.FP64), ("mixed", bem.MIXED)):
                (u, it, rel), t_sol = timed(lambda: ctx.solve(prec, tol=1e-10))
                x = u[0]
                _, t_mv = timed(lambda: ctx.matvec(x, prec))
                res[name] = {"solve_ms": t_sol, "iters": it, "relres": rel[0], "matvec_ms": t_mv,
                             "max_abs_sigma_minus_1": float((u[0] - 1.0).abs().max().item())}
            emit({"config": f"curved sphere level {level}: {len(tri6)} six-node triangles, {nv} vertices, "
                            f"P1 collocation, V0=1, tol 1e-10",
                  "setup_ms": t_set, "near_pairs": ctx.near_pairs, **res})
            ctx.close()
        # a conductor inside a dielectric ball (Eq. Final3 rows): charges against Gauss's law
        for level in (2, 3):
            nodes, tri6, nv, body = mg.quadratic_bodies([mg.quadratic_sphere(level, 1.0),
                                                         mg.quadratic_sphere(level, 2.0)])
            body = np.asarray(body, np.int32)
            regs = [{"kind": "conductor", "V0": 1.0}, {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": 4.0}]
            ctx, t_set = wall(lambda: bem.P1Context(nodes, tri6, nv, body, regs))
            Qg = 4 * np.pi / (1.0 / 4.0 + 0.75 / 2.0)
            want = np.array([Qg / 4.0, Qg * 0.75])
            wts = p1_vertex_weights(nodes, tri6, nv, body, 2)   # int psi_v dS per body
            res = {}
            for name, prec in (("fp64", bem.FP64), ("mixed", bem.MIXED)):
                (u, it, rel), t_sol = timed(lambda: ctx.solve(prec, tol=1e-10))
                q = wts @ u[0].cpu().numpy()[:nv]
                res[name] = {"solve_ms": t_sol, "iters": it, "relres": rel[0],
                             "charge_rel_err_vs_gauss": [float(v) for v in np.abs(q - want) / want]}
            emit({"config": f"curved conductor sphere (a=1, V0=1) in a dielectric ball (b=2, eps 4), level {level}: "
                            f"{len(tri6)} six-node triangles, {nv} vertices, tol 1e-10",
                  "setup_ms": t_set, **res})
            ctx.close()
    if "c5" in want:
        scale = (200000 / 20068.0) ** 0.5
        mesh = mg.device_mesh(scale, seed=2)
        pts = mg.device_box_points(1000000, seed=5)
        pts_d = torch.tensor(pts, device="cuda")
        ctx, t_set = wall(lambda: bem.Context(mesh))
        (u, it, rel), t_sol = timed(lambda: ctx.solve(bem.MIXED, tol=TOL))
        (phi, E), t_ev = timed(lambda: ctx.eval_field(u[0], pts_d, bem.MIXED))
        x = u[0]
        _, t_mv32 = timed(lambda: ctx.matvec(x, bem.MIXED))
        _, t_mv64 = timed(lambda: ctx.matvec(x, bem.FP64))
        L = args.c5_lines
        seeds = torch.tensor(mg.fibonacci_seeds(L, radius=1.05))
        (K, st, ns, xe), t_tr = timed(lambda: ctx.trace_lines(u[0], seeds, bem.MIXED))
        sel = np.random.default_rng(5).choice(len(pts), 1000, replace=False)
        P = O.Problem(mesh, eta=4.0, g=3)
        (_, E_o), t_o = wall(lambda: P.field(u[0].cpu().numpy(), pts[sel]))
        emit({"config": f"c5 device at {mesh.np_} triangles, mixed to {TOL}, 1e6 box points, {L} lines (sample)",
              "mixed": {"setup_ms": t_set, "solve_ms": t_sol, "iters": it, "relres": rel[0], "eval_ms": t_ev,
                        "trace_ms": t_tr, "rk4_steps": int(ns.sum().item()),
                        "E_rel_vs_oracle_1000pts": float(np.abs(E.cpu().numpy()[sel] - E_o).max() / np.abs(E_o).max())},
              "matvec_ms": {"mixed": t_mv32, "fp64": t_mv64},
              "fp64_solve_s_extrapolated": it * t_mv64 / 1e3,
              "oracle": {"field_1000pts_ms": t_o, "field_1e6pts_s_extrapolated": t_o / 1e3 * 1000}})
        ctx.close()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores, timed
    on a bounded sample of the same workload.  Each step computes the oracle's pair
    integrals of 48 seeded collocation rows (the solve's products) and the field of
    48 seeded evaluation points (the field phase) against all triangles; the line's
    config names exactly that sample."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    mesh, pts = workload(args)
    from oracle import oracle as O
    P = O.Problem(mesh, eta=4.0, g=3)
    rng = np.random.default_rng(7)
    rows = 48
    ppts = 48

    def step():
        idx = np.sort(rng.choice(P.N, size=rows, replace=False))
        P.pair_block(P.centroids[idx], idx)            # collocation rows (solve)
        sel = rng.choice(len(pts), size=ppts, replace=False)
        P.field(np.ones(P.N), pts[sel])                # field evaluation
        return (rows + ppts) * P.N

    for _ in range(args.warmup):
        step()
    times, pairs = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pairs = step()
        times.append(time.perf_counter() - t0)
    ms = float(np.mean(times)) * 1e3
    value = pairs / (ms * 1e-3) / 1e9
    sample = (f"per step: oracle pair integrals of {rows} seeded collocation rows and {ppts} "
              f"evaluation points x {P.N} triangles (FP64, OpenMP)")
    cfg = {"workload": workload_name(mesh), "triangles": int(mesh.np_), "unknowns": int(mesh.n_unknowns),
           "counts_sphere_torus_cylinder": list(mesh.info["counts"]),
           "timed_per_step": f"{rows} collocation rows + {ppts} field points against all {P.N} triangles "
                             f"(no solve, no full field: a bounded sample of the step's pair integrals)",
           "far_rule": "3x3 Duffy/Gauss, eta=4", "parallelism": "host cores, rank 0 only"}
    print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f64", "data": "synthetic (seeded meshes and points)",
                      "config": cfg, "impl": "reference",
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                                       "kind": "oracle", "sample": sample, "cpu_model": cpu_model()},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "matvec":
        run_matvec(a)
    elif a.mode == "batch":
        run_batch(a)
    elif a.mode == "report":
        run_report(a)
    elif a.mode == "trace":
        run_trace(a)
    else:
        run_ours(a)
