#!/usr/bin/env python
"""Benchmark: numeric factorization GFLOP/s and solve time of the supernodal
right-looking Cholesky (RLB) on one GB300.

Workload: 3D 7-point variable-coefficient diffusion on a 48^3 grid
(n = 110,592; edge coefficients log-uniform[1e-2, 1e2]; diagonal = row sum + 1e-6),
geometric nested dissection, partition refinement, FP64 RLB factor, 4 right-hand
sides uniform[-1, 1]. Seeded synthetic input (stand-in for the paper's
SuiteSparse matrices).

One step = refactor (values already in HBM: value load, every level's POTRF,
TRSM and RLB updates) + solve of the 4 right-hand sides (forward and backward
sweeps, FP64 residual and backward error).
value = sum_j |L_{*,j}|^2 / factor time (GFLOP/s), over the timed steps.

--impl reference times the oracle (plain FP64 column Cholesky in C) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor GFLOP/s + solve time: FP64 vs FP32/TF32+IR at <=1e-14 backward error"
WORKLOAD = "diffusion3d_7pt_varcoef_48^3"
SAMPLE_SIDE = 32  # oracle sample: the same generator on a 32^3 grid


# DRAM bytes (read + write) of every launch of a kernel class in one
# factorization, measured with ncu on the current kernel code (recorded with
# its command in profiles/k_gemm_tiles_fp64_diffusion48.md). Key: (class,
# precision, workload, scale, merge). Classes without a capture of the current
# code report null.
TRAFFIC = {("gemm_simt", "fp64", 2, 1.0, 0.125): 2544617984}


def reduce_max_over_ranks(dist, values, device):
    """Max over ranks of per-rank timings (replicas: the job takes as long as
    its slowest rank). dist None: single process, values unchanged."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(world, flops, steps, max_ms):
    """GFLOP/s of the whole job: every rank factors its own copy (weak scaling),
    so the job does world x flops x steps in the slowest rank's time."""
    return world * flops * steps / (max_ms * 1e-3) / 1e9


def _time_factor_solve(num, dv, Bd, Xd, stream, reps, **solve_kw):
    """Best of reps (refactor, solve) pairs timed with CUDA events on the stream."""
    import torch
    num.solve(Bd, Xd, **solve_kw)
    best = None
    for _ in range(reps):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        num.refactor(dv)
        b.record(stream)
        _, si = num.solve(Bd, Xd, **solve_kw)
        c.record(stream)
        torch.cuda.synchronize()
        t = (a.elapsed_time(b), b.elapsed_time(c))
        if best is None or sum(t) < sum(best[0]):
            best = (t, si)
    return best


def _other_workloads(args, sc, inputs, torch, np, dev, stream):
    """The other workloads of the benchmark's configuration list, each measured
    once: the 64^2 Laplacian (RL vs RLB in FP64), the batch of 256 2D Laplacians
    (batched low-precision factor + refinement vs per-matrix FP64), the
    anisotropic 3D matrix (FP64 vs TF32x3 + preconditioned CG, PR on vs off) and
    the 48^3 matrix under the general-graph ordering."""
    out = {}
    # 64^2 2D Laplacian, FP64, RL (Alg. 4) and RLB (Alg. 5), fundamental supernodes
    A1, n1 = inputs.workload(1)
    dv1 = torch.tensor(A1.values, device=dev, dtype=torch.float64)
    B1 = torch.tensor(np.ascontiguousarray(inputs.rhs(A1.n, n1, inputs.SEED_BASE + 1).T), device=dev)
    r = {"workload": A1.name, "n": A1.n}
    for var in ("rl", "rlb"):
        sy = sc.Symbolic(A1, ordering="grid_nd", grid=A1.grid, variant=var, merge=args.merge)
        nm = sy.factor(dv1, precision="fp64")
        (fm, sm_), si = _time_factor_solve(nm, dv1, B1, torch.zeros_like(B1), stream, 5)
        fl = sy.view()["flops"]
        r[var] = {"factor_ms": fm, "factor_gflops": fl / (fm * 1e-3) / 1e9, "solve_ms": sm_, "eta_max": si["eta_max"]}
        nm.free()
    out["rl_vs_rlb_lap2d_64"] = r
    # 256 2D Laplacians: one batched factorization vs a loop of per-matrix FP64 factorizations
    mats, n4 = inputs.workload(4)
    syms = [sc.Symbolic(A, ordering="grid_nd", grid=A.grid, merge=args.merge) for A in mats]
    bsym = sc.Symbolic.batch(syms)
    vals = torch.tensor(np.concatenate([A.values for A in mats]), device=dev, dtype=torch.float64)
    ntot = sum(A.n for A in mats)
    Bb = torch.tensor(np.ascontiguousarray(inputs.rhs(ntot, n4, inputs.SEED_BASE + 4).T), device=dev)
    flb = sum(sy.view()["flops"] for sy in syms)
    r = {"matrices": len(mats), "n_total": ntot, "sum_cj2": flb}
    for prec in ("fp32", "tf32x3"):
        nm = bsym.factor(vals, precision=prec)
        (fm, sm_), si = _time_factor_solve(nm, vals, Bb, torch.zeros_like(Bb), stream, 3)
        r["batched_" + prec] = {"factor_ms": fm, "factor_gflops": flb / (fm * 1e-3) / 1e9, "solve_ms": sm_,
                                "total_ms": fm + sm_, "eta_max": si["eta_max"], "ir_iterations": si["iterations"],
                                "converged": si["converged"]}
        nm.free()
    nums, parts = [], []
    off = row = 0
    for A, sy in zip(mats, syms):
        v = vals[off:off + A.nnz]
        nums.append(sy.factor(v, precision="fp64"))
        parts.append((v, Bb[:, row:row + A.n].contiguous()))
        off += A.nnz
        row += A.n
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    worst = 0.0
    for nm, (v, Bi) in zip(nums, parts):
        nm.refactor(v)
        _, si = nm.solve(Bi, torch.zeros_like(Bi))
        worst = max(worst, si["eta_max"])
    b.record(stream)
    torch.cuda.synchronize()
    r["per_matrix_fp64"] = {"total_ms": a.elapsed_time(b), "eta_max": worst}
    for nm in nums:
        nm.free()
    r["speedup_total"] = r["per_matrix_fp64"]["total_ms"] / min(r["batched_fp32"]["total_ms"],
                                                             r["batched_tf32x3"]["total_ms"])
    out["batch_lap2d_256"] = r
    del vals, Bb
    # anisotropic 3D 7-point (1:1:100 x log-uniform, shift 1e-8): PR on vs off, FP64 vs TF32x3 + CG
    A5, n5 = inputs.workload(5, args.aniso_scale)
    dv5 = torch.tensor(A5.values, device=dev, dtype=torch.float64)
    B5 = torch.tensor(np.ascontiguousarray(inputs.rhs(A5.n, n5, inputs.SEED_BASE + 5).T), device=dev)
    r = {"workload": A5.name, "n": A5.n, "nrhs": n5}
    for pr in (True, False):
        sy = sc.Symbolic(A5, ordering="grid_nd", grid=A5.grid, pr=pr, merge=args.merge)
        vw = sy.view()
        key = "pr_on" if pr else "pr_off"
        r[key] = {"blocks": int(len(vw["blk_first"])), "sum_cj2": vw["flops"]}
        nm = sy.factor(dv5, precision="tf32x3")
        (fm, sm_), si = _time_factor_solve(nm, dv5, B5, torch.zeros_like(B5), stream, 2, method="cg",
                                           max_iterations=1000)
        r[key]["tf32x3_cg"] = {"factor_ms": fm, "factor_gflops": vw["flops"] / (fm * 1e-3) / 1e9,
                               "solve_ms": sm_, "total_ms": fm + sm_, "eta_max": si["eta_max"],
                               "iterations": si["iterations"], "converged": si["converged"]}
        nm.free()
        if pr:
            # FP64 at the full size runs for tens of seconds: one factorization, timed by the
            # library's CUDA events (the first call also captures the graph: < 0.5 % of it)
            nm = sy.factor(dv5, precision="fp64")
            fm = nm.info.factor_ms
            X5 = torch.zeros_like(B5)
            nm.solve(B5, X5)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, si = nm.solve(B5, X5)
            c.record(stream)
            torch.cuda.synchronize()
            sm_ = a.elapsed_time(c)
            r[key]["fp64"] = {"factor_ms": fm, "factor_gflops": vw["flops"] / (fm * 1e-3) / 1e9,
                              "solve_ms": sm_, "total_ms": fm + sm_, "eta_max": si["eta_max"]}
            nm.free()
            r["speedup_tf32x3_cg_vs_fp64"] = r[key]["fp64"]["total_ms"] / r[key]["tf32x3_cg"]["total_ms"]
    out["aniso_3d"] = r
    # the benchmark's 48^3 matrix given without grid coordinates, ordered by the
    # library's general-graph nested dissection (breadth-first level separators)
    try:
        out["graph_nd_diff7_48"] = _graph_nd_workload(args, sc, inputs, torch, np, dev, stream)
    except Exception as ex:  # reported, not fatal
        out["graph_nd_diff7_48"] = {"error": str(ex)}
    return out


def _graph_nd_workload(args, sc, inputs, torch, np, dev, stream):
    A2, n2 = inputs.workload(2)
    sy = sc.Symbolic(A2, ordering="graph_nd", pr=True, merge=args.merge)
    vw = sy.view()
    dv2 = torch.tensor(A2.values, device=dev, dtype=torch.float64)
    B2 = torch.tensor(np.ascontiguousarray(inputs.rhs(A2.n, n2, inputs.SEED_BASE + 2).T), device=dev)
    r = {"workload": A2.name + " (no coordinates)", "ordering": "graph ND (leaf 8) + PR", "n": A2.n,
         "nnz_L": int(vw["nnzL"]), "sum_cj2": vw["flops"], "nsuper": int(vw["nsuper"])}
    for prec, kw in (("fp64", {}), ("tf32x3", {"method": "cg", "max_iterations": 400})):
        nm = sy.factor(dv2, precision=prec)
        (fm, sm_), si = _time_factor_solve(nm, dv2, B2, torch.zeros_like(B2), stream, 3, **kw)
        r[prec] = {"factor_ms": fm, "factor_gflops": vw["flops"] / (fm * 1e-3) / 1e9, "solve_ms": sm_,
                   "total_ms": fm + sm_, "eta_max": si["eta_max"], "iterations": si["iterations"]}
        nm.free()
    return r


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "tf32x3"])
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--aniso-scale", type=float, default=1.0,
                    help="grid scale of the anisotropic 3D workload (1.0 = 128^3)")
    ap.add_argument("--merge", type=float, default=0.125, help="supernode merging budget (Sec. 3.1); 0 = off")
    ap.add_argument("--workload", type=int, default=2, choices=[2, 3],
                    help="2: the benchmark matrix (48^3 7-point); 3: 80^3 27-point (for profiling the TF32 path)")
    ap.add_argument("--scale", type=float, default=1.0, help="grid-side scale of the workload (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-plan autotuner's measurement")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the TF32+refinement vs FP64 comparison on the 80^3 27-point matrix")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_sample(steps: int):
    """Times the oracle (as it stands) on the same generator at 32^3: returns (GFLOP/s, sample text)."""
    import oracle
    from paper_2409_13090_gb300 import inputs
    A = inputs.diffusion_3d_7pt(SAMPLE_SIDE, SAMPLE_SIDE, SAMPLE_SIDE, inputs.SEED_BASE + 2)
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True)
    flops = o.symbolic().flops
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        info = o.factor()
        times.append(time.perf_counter() - t0)
        assert info == 0
    return flops, times, f"oracle Alg. 1 column Cholesky of the same generator on a {SAMPLE_SIDE}^3 grid " \
                         f"(n={A.n}, sum c_j^2={flops:.3e}), 1 thread"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    flops, times, sample = _cpu_sample(args.warmup + args.steps)
    t = times[args.warmup:]
    val = flops * len(t) / sum(t) / 1e9
    line = {"metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n": 110592, "nrhs": 4, "precision": "fp64",
                       "sample": sample, "parallelism": "none (host)"},
            "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = _args()
    import oracle  # noqa: F401  (only the cpu_baseline leg and --impl reference execute it)
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    import paper_2409_13090_gb300 as sc
    from paper_2409_13090_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sc.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    A, nrhs = inputs.workload(args.workload, args.scale)
    t0 = time.perf_counter()
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, nd_leaf=8, pr=True, variant="rlb", merge=args.merge)
    analyze_s = time.perf_counter() - t0
    view = sym.view()
    flops = view["flops"]
    dv = torch.tensor(A.values, device=dev, dtype=torch.float64)
    B = inputs.rhs(A.n, nrhs, inputs.SEED_BASE + 2)
    Bd = torch.tensor(np.ascontiguousarray(B.T), device=dev)  # (nrhs, n) = column-major n x nrhs
    Xd = torch.zeros_like(Bd)
    num = sym.factor(dv, precision=args.precision)
    assert num.rc == 0, num.rc
    for _ in range(max(3, args.warmup)):
        num.refactor(dv)
        _, sinfo = num.solve(Bd, Xd)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    etas = []
    iters = []
    for e0, e1, e2 in ev:
        e0.record(stream)
        finfo = num.refactor(dv)
        e1.record(stream)
        _, sinfo = num.solve(Bd, Xd)
        e2.record(stream)
        launches += finfo.kernel_launches + sinfo["kernel_launches"]
        etas.append(sinfo["eta_max"])
        iters.append(sinfo["iterations"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    fac_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    sol_ms = sum(b.elapsed_time(c) for _, b, c in ev)
    step_ms = sum(a.elapsed_time(c) for a, _, c in ev)
    fac_ms, sol_ms, step_ms = reduce_max_over_ranks(dist, [fac_ms, sol_ms, step_ms], dev)
    K = args.steps
    value = whole_job_rate(world, flops, K, fac_ms)

    # ---- end to end through host buffers (pinned): H2D values + factor + solve with H2D B / D2H X
    vals_h = torch.tensor(A.values, dtype=torch.float64).pin_memory()
    B_h = torch.tensor(np.ascontiguousarray(B.T)).pin_memory()
    X_h = torch.zeros_like(B_h).pin_memory()
    e2e_f, e2e_s = [], []
    for i in range(K + 1):
        torch.cuda.synchronize()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        num.refactor(vals_h)
        b.record(stream)
        num.solve(B_h, X_h)
        c.record(stream)
        torch.cuda.synchronize()
        if i:
            e2e_f.append(a.elapsed_time(b))
            e2e_s.append(b.elapsed_time(c))
    e2e = {"value": world * flops / (sum(e2e_f) / len(e2e_f) * 1e-3) / 1e9, "unit": "GFLOP/s",
           "h2d_bytes_per_step": int(A.nnz * 8 + A.n * nrhs * 8), "d2h_bytes_per_step": int(A.n * nrhs * 8 + 8),
           "factor_ms": sum(e2e_f) / len(e2e_f), "solve_ms": sum(e2e_s) / len(e2e_s)}

    # ---- per-kernel profile of the same factorization (CUDA events around every launch)
    prof = None
    for _ in range(3):
        p = num.profile(dv)
        if prof is None:
            prof = {k: dict(v) for k, v in p.items()}
        else:
            for k in p:
                prof[k]["ms"] += p[k]["ms"]
    for k in prof:
        prof[k]["ms"] /= 3
    peaks, peak_kind = _peaks()
    fp_peak = {}
    for kind, nm in ((0, "fp64"), (1, "fp32")):
        try:
            fp_peak[nm] = sc.sc_probe_fma_peak(kind) / 1e12
        except Exception:
            fp_peak[nm] = None
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
    if dom == "gemm_tc":
        peak = peaks["bf16_tflops_sustained"] * (1.1 / 2.25)
        bound, pk = "tensor", f"TF32 = {peak_kind} bf16 sustained x 1.1/2.25 (nominal tf32/bf16)"
    else:
        peak = fp_peak["fp64" if args.precision == "fp64" else "fp32"]
        bound, pk = "alu", "measured FMA-chain probe (sc_probe_fma_peak)"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if peak else None,
                "traffic": TRAFFIC.get((dom, args.precision, args.workload, args.scale, args.merge)),
                "traffic_scope": "DRAM bytes of all launches of the class in one factorization (ncu)",
                "kernel": dom,
                "kernel_launches": d["launches"], "peak_source": pk,
                "profile": {k: {"ms": round(v["ms"], 4), "gflop": round(v["flops"] / 1e9, 3),
                                "launches": v["launches"]} for k, v in prof.items()},
                "fma_peak_tflops": fp_peak}

    # ---- the solve against HBM: each sweep reads L once, the work vectors in and
    #      out, and glbind; the timed solve also forms the FP64 residual (CSR A)
    s_l = 8 if args.precision == "fp64" else 4
    sweeps = 2 * (1 + (sum(iters) / len(iters) if iters else 0))
    solve_bytes = sweeps * (int(view["nnzL"]) * s_l + 2 * A.n * nrhs * s_l + len(view["glbind"]) * 4)
    solve_ms_step = sol_ms / K
    solve_roofline = {"bound": "hbm", "achieved": solve_bytes / (solve_ms_step * 1e-3) / 1e9,
                      "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": solve_bytes / (solve_ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"],
                      "bytes_per_solve": int(solve_bytes), "peak_source": f"{peak_kind} HBM copy",
                      "note": "the sweeps are bound by the chain of dependent chunk steps, not by HBM"}

    # ---- the launch-plan autotuner (sc_tune) on the same matrix: the headline above
    #      uses the default plan; here the tuned plan's factor is timed the same way
    tune = None
    if not args.no_tune:
        try:
            sym_t = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, nd_leaf=8, pr=True, variant="rlb",
                                merge=args.merge)
            t0 = time.perf_counter()
            table = sym_t.tune(dv, precision=args.precision, reps=3)
            tune_s = time.perf_counter() - t0
            num_t = sym_t.factor(dv, precision=args.precision)
            for _ in range(3):
                num_t.refactor(dv)

            def _factor_ms(h):
                evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(K)]
                torch.cuda.synchronize()
                for a, b in evs:
                    a.record(stream)
                    h.refactor(dv)
                    b.record(stream)
                torch.cuda.synchronize()
                return sum(a.elapsed_time(b) for a, b in evs) / K

            ms_tuned, ms_default = _factor_ms(num_t), _factor_ms(num)
            tune = {"table": {k: table[k] for k in sc.TUNE_FIELDS}, "settings_timed": table["tried"],
                    "tune_s": tune_s, "factor_ms_default": ms_default, "factor_ms_tuned": ms_tuned,
                    "gflops_default": flops / (ms_default * 1e-3) / 1e9,
                    "gflops_tuned": flops / (ms_tuned * 1e-3) / 1e9,
                    "note": "0 = library default; the headline value uses the default plan"}
            num_t.free()
        except Exception as ex:  # reported, not fatal: the headline is already measured
            tune = {"error": str(ex)}

    # ---- the low-precision form on the same matrix (factor GFLOP/s, refinement outcome)
    mixed = None
    if not args.no_mixed and args.precision == "fp64":
        mixed = {}
        for prec in ("fp32", "tf32", "tf32x3"):
            nm = sym.factor(dv, precision=prec)
            for _ in range(2):
                nm.refactor(dv)
            fts = []
            for _ in range(3):
                fi = nm.refactor(dv)
                fts.append(fi.factor_ms)
            _, si = nm.solve(Bd, torch.zeros_like(Bd))
            mixed[prec] = {"factor_gflops": flops / (min(fts) * 1e-3) / 1e9, "factor_ms": min(fts),
                           "ir_iterations": si["iterations"], "eta_max": si["eta_max"], "converged": si["converged"],
                           "solve_ms": si["solve_ms"], "pivot_fallbacks": fi.pivot_fallbacks}
            # conjugate gradients preconditioned by the same factor (classical refinement cannot
            # converge here: kappa x unit roundoff of the factor exceeds 1)
            nm.solve(Bd, torch.zeros_like(Bd), method="cg", max_iterations=400)
            _, sc_ = nm.solve(Bd, torch.zeros_like(Bd), method="cg", max_iterations=400)
            mixed[prec]["cg"] = {"iterations": sc_["iterations"], "eta_max": sc_["eta_max"],
                                 "converged": sc_["converged"], "solve_ms": sc_["solve_ms"],
                                 "total_ms": min(fts) + sc_["solve_ms"]}
            nm.free()

    # ---- the chosen form vs the plain form where refinement converges: 80^3 27-point stencil
    #      (kappa ~ 1e2), 16 right-hand sides, TF32 factor + FP64 refinement vs FP64 factor + solve
    compare = None
    if not args.no_compare and args.workload == 2 and args.scale == 1.0:
        A3, nrhs3 = inputs.workload(3)
        sym3 = sc.Symbolic(A3, ordering="grid_nd", grid=A3.grid, nd_leaf=8, pr=True, variant="rlb", merge=args.merge)
        f3 = sym3.view()["flops"]
        dv3 = torch.tensor(A3.values, device=dev, dtype=torch.float64)
        B3 = inputs.rhs(A3.n, nrhs3, inputs.SEED_BASE + 3)
        B3d = torch.tensor(np.ascontiguousarray(B3.T), device=dev)
        X3d = torch.zeros_like(B3d)
        compare = {"workload": A3.name, "n": A3.n, "sum_cj2": f3, "nrhs": nrhs3}
        for prec, reps in (("tf32", 3), ("tf32x3", 3), ("fp64", 2)):
            nm = sym3.factor(dv3, precision=prec)
            nm.solve(B3d, X3d)
            best = None
            for _ in range(reps):
                a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(stream)
                nm.refactor(dv3)
                b.record(stream)
                _, si = nm.solve(B3d, X3d)
                c.record(stream)
                torch.cuda.synchronize()
                t = (a.elapsed_time(b), b.elapsed_time(c))
                if best is None or sum(t) < sum(best[0]):
                    best = (t, si)
            (fm, sm_), si = best
            compare[prec] = {"factor_ms": fm, "factor_gflops": f3 / (fm * 1e-3) / 1e9, "solve_ms": sm_,
                             "total_ms": fm + sm_, "eta_max": si["eta_max"], "ir_iterations": si["iterations"],
                             "converged": si["converged"]}
            nm.free()
        compare["speedup_total"] = compare["fp64"]["total_ms"] / min(compare["tf32"]["total_ms"],
                                                                     compare["tf32x3"]["total_ms"])
        del dv3, B3d, X3d

    others = None
    if not args.no_others and args.workload == 2 and args.scale == 1.0 and rank == 0:
        others = _other_workloads(args, sc, inputs, torch, np, dev, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cflops, ctimes, sample = _cpu_sample(2)
        cpu = {"value": cflops / min(ctimes) / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
               "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": step_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD if (args.workload == 2 and args.scale == 1.0) else A.name, "n": A.n, "nnz_A_lower": A.nnz, "nnz_L": int(view["nnzL"]),
                           "sum_cj2": flops, "nsuper": int(view["nsuper"]), "nrhs": nrhs,
                           "precision": args.precision, "variant": "rlb", "ordering": "grid ND (leaf 8) + PR",
                           "merge_frac": args.merge,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (factor storage rewritten every step)",
                           "analyze_s": analyze_s},
                "factor_ms": fac_ms / K, "solve_ms": sol_ms / K, "eta_max": max(etas),
                "ir_iterations": max(iters), "gpu_launches": launches, "clocks": clk, "e2e": e2e,
                "roofline": roofline, "solve_roofline": solve_roofline, "tune": tune, "cpu_baseline": cpu,
                "mixed": mixed,
                "tf32_ir_vs_fp64_stencil27_80": compare,
                "other_workloads": others}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
