#!/usr/bin/env python
"""Benchmark: numeric factorization GFLOP/s and solve time of the supernodal
right-looking Cholesky (RLB, Alg. 5) on one GB300, FP64 against the
TF32x3 + refinement form, at <= 1e-14 backward error.

Headline workload (the largest configuration): 3D 7-point anisotropic diffusion
on a 128^3 grid (n = 2,097,152; coefficients 1:1:100 along x:y:z times
log-uniform[0.1, 10] noise; diagonal shift 1e-8), geometric nested dissection,
partition refinement, supernode merging 12.5 %, 64 right-hand sides
uniform[-1, 1]. Seeded synthetic input (stand-in for the paper's SuiteSparse
matrices).

One step = refactor in FP64 (values already in HBM: value load, every level's
POTRF, TRSM and RLB updates) + solve of the 64 right-hand sides (forward and
backward sweeps, FP64 residual and backward error).
value = sum_j |L_{*,j}|^2 / factor time (GFLOP/s) over the timed steps.
The same line carries the chosen form on the same matrix (TF32x3 factor +
conjugate gradients preconditioned by it, to eta <= 1e-14), the end-to-end
numbers through host buffers, per-kernel-class rooflines, the other
workloads, and the oracle timed on the host cores.

--impl reference times the oracle (plain FP64 column Cholesky in C) on the
host cores on a bounded sample of the headline matrix: the leading principal
block of P A P^T that one subtree of the nested dissection spans.
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
WORKLOADS = {2: "diffusion3d_7pt_varcoef_48^3", 3: "stencil3d_27pt_80^3", 5: "aniso3d_7pt_128^3"}
SAMPLE_VOLUME = 32768  # oracle sample: a nested-dissection subtree of about this many unknowns

# DRAM bytes (read + write) of every launch of a kernel class in one
# factorization, measured with ncu on the current kernel code (each recorded
# with its command under profiles/). Key: (class, precision, workload, scale,
# merge). Classes without a capture of the current code report null.
TRAFFIC = {}


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


def _timed_steps(num, dv, Bd, Xd, stream, steps, **solve_kw):
    """steps (refactor, solve) pairs, each bracketed by CUDA events on the
    launching stream; returns per-step factor and solve ms, launches, eta,
    iterations."""
    import torch
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(steps)]
    launches, etas, iters, conv = 0, [], [], []
    for e0, e1, e2 in ev:
        e0.record(stream)
        finfo = num.refactor(dv)
        e1.record(stream)
        _, si = num.solve(Bd, Xd, **solve_kw)
        e2.record(stream)
        launches += finfo.kernel_launches + si["kernel_launches"]
        etas.append(si["eta_max"])
        iters.append(si["iterations"])
        conv.append(si["converged"] or si["rc"] == 0)
    torch.cuda.synchronize()
    return ([a.elapsed_time(b) for a, b, _ in ev], [b.elapsed_time(c) for _, b, c in ev], launches, etas, iters,
            conv)


def _e2e(num, A, B, stream, steps, **solve_kw):
    """End to end through the public API with pinned host buffers: every step
    copies the values and B host -> device and X device -> host inside the
    timed region (refactor + solve)."""
    import numpy as np
    import torch
    vals_h = torch.tensor(A.values, dtype=torch.float64).pin_memory()
    B_h = torch.tensor(np.ascontiguousarray(B.T)).pin_memory()
    X_h = torch.zeros_like(B_h).pin_memory()
    f, s, lib, its, cin, cout = [], [], [], [], [], []
    for i in range(steps + 1):
        torch.cuda.synchronize()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        num.refactor(vals_h)
        b.record(stream)
        _, si = num.solve(B_h, X_h, **solve_kw)
        c.record(stream)
        torch.cuda.synchronize()
        if i:  # the first pair is a warm-up of the host-buffer path
            f.append(a.elapsed_time(b))
            s.append(b.elapsed_time(c))
            lib.append(si["solve_ms"])
            its.append(si["iterations"])
            cin.append(si["copy_in_ms"])
            cout.append(si["copy_out_ms"])
    # the copy rates of these pinned buffers on their own (B in, X out)
    Bt = torch.empty(B_h.shape, dtype=B_h.dtype, device="cuda")
    rates = {}
    for key, dst, src in (("h2d_gbs", Bt, B_h), ("d2h_gbs", X_h, Bt)):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dst.copy_(src, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        rates[key] = B_h.numel() * 8 / (a.elapsed_time(b) * 1e6)
    del Bt
    return sum(f) / len(f), sum(s) / len(s), {"lib_solve_ms": sum(lib) / len(lib), "iterations": max(its),
                                               "lib_copy_in_ms": sum(cin) / len(cin),
                                               "lib_copy_out_ms": sum(cout) / len(cout), **rates}


def _class_rooflines(prof, peaks, fp_peak, precision, workload, scale, merge):
    """Per kernel class of one factorization: algorithmic flops / summed launch
    time against the class's peak (SIMT classes: the measured FMA rate of the
    storage precision; tensor-core tiles: the TF32 peak)."""
    out = {}
    tf32 = peaks["bf16_tflops_sustained"] * (1.1 / 2.25)
    for k, v in prof.items():
        if not v["launches"]:
            continue
        ach = v["flops"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] > 0 else 0.0
        if k == "gemm_tc":
            pk, bound = tf32, "tensor"
        else:
            pk, bound = fp_peak["fp64" if precision == "fp64" else "fp32"], "alu"
        out[k] = {"bound": bound, "launches": v["launches"], "ms": round(v["ms"], 4),
                  "gflop": round(v["flops"] / 1e9, 3), "achieved_tflops": ach, "peak_tflops": pk,
                  "frac": ach / pk if pk else None,
                  "traffic_bytes": TRAFFIC.get((k, precision, workload, scale, merge))}
        if k == "gemm_tc" and precision == "tf32x3":
            # each algorithmic product is three tensor-core products (hi*hi, hi*lo, lo*hi)
            out[k]["tensor_pipe_tflops"] = 3 * ach
            out[k]["tensor_pipe_frac"] = 3 * ach / pk if pk else None
    return out


def _solve_roofline(view, n, nrhs, s_l, ms, sweeps, peaks, peak_kind, fma_peak):
    """A triangular solve against both of its limits: HBM (per sweep nnz(L) x
    entry size + 2 n nrhs x entry size + |glbind| x 4 bytes) and the FMA rate of
    the storage precision (2 nnz(L) nrhs flops per sweep); the larger of the
    two floors is the bound."""
    nnz_l, gl = int(view["nnzL"]), len(view["glbind"])
    byts = sweeps * (nnz_l * s_l + 2 * n * nrhs * s_l + gl * 4)
    flops = sweeps * 2.0 * nnz_l * nrhs
    t_hbm = byts / (peaks["hbm_gbs"] * 1e9)
    t_alu = flops / (fma_peak * 1e12) if fma_peak else 0.0
    bound = "alu" if t_alu > t_hbm else "hbm"
    floor_ms = 1e3 * max(t_hbm, t_alu)
    return {"bound": bound, "ms": ms, "floor_ms": floor_ms, "frac": floor_ms / ms if ms else None,
            "achieved_gbs": byts / (ms * 1e-3) / 1e9, "peak_gbs": peaks["hbm_gbs"],
            "achieved_tflops": flops / (ms * 1e-3) / 1e12, "peak_tflops": fma_peak,
            "bytes": int(byts), "flops": flops, "sweeps": sweeps,
            "peak_source": f"{peak_kind} HBM copy; measured FMA-tile probe",
            "definition": "per sweep: nnz(L) x entry size + 2 n nrhs x entry size + |glbind| x 4 bytes and "
                          "2 nnz(L) nrhs flops; frac = the larger floor / the measured time"}


def _other_workloads(args, sc, inputs, torch, np, dev, stream, sym5, A5, dv5, B5d, flops5):
    """The other workloads of the benchmark's configuration list, each measured
    once: the 64^2 Laplacian (RL vs RLB in FP64), the batch of 256 2D Laplacians
    (batched low-precision factor + refinement vs per-matrix FP64), the 48^3
    variable-coefficient matrix (FP64 and the low-precision forms with classical
    refinement and CG), the 80^3 27-point stencil (TF32 / TF32x3 + refinement vs
    FP64), the 128^3 anisotropic matrix without partition refinement, and the
    48^3 matrix under the general-graph ordering."""
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
    # 48^3 variable-coefficient 7-point matrix: FP64, and the low-precision forms
    out["diffusion_48"] = _workload_48(args, sc, inputs, torch, np, dev, stream)
    # 80^3 27-point stencil (kappa ~ 1e2): TF32 / TF32x3 + classical refinement vs FP64
    out["stencil27_80"] = _workload_80(args, sc, inputs, torch, np, dev, stream)
    # the headline matrix without partition refinement (more, smaller blocks), TF32x3 + CG
    sy = sc.Symbolic(A5, ordering="grid_nd", grid=A5.grid, pr=False, merge=args.merge)
    vw = sy.view()
    nm = sy.factor(dv5, precision="tf32x3")
    (fm, sm_), si = _time_factor_solve(nm, dv5, B5d, torch.zeros_like(B5d), stream, 2, method="cg",
                                       max_iterations=1000)
    out["aniso_128_pr_off"] = {"blocks": int(len(vw["blk_first"])), "blocks_pr_on": int(len(sym5.view()["blk_first"])),
                               "tf32x3_cg": {"factor_ms": fm, "factor_gflops": flops5 / (fm * 1e-3) / 1e9,
                                             "solve_ms": sm_, "total_ms": fm + sm_, "eta_max": si["eta_max"],
                                             "iterations": si["iterations"], "converged": si["converged"]}}
    nm.free()
    del sy
    try:
        out["graph_nd_diff7_48"] = _graph_nd_workload(args, sc, inputs, torch, np, dev, stream)
    except Exception as ex:  # reported, not fatal
        out["graph_nd_diff7_48"] = {"error": str(ex)}
    return out


def _workload_48(args, sc, inputs, torch, np, dev, stream):
    """The 48^3 matrix (kappa ~ 1e9): FP64 factor + solve, and the FP32 / TF32 /
    TF32x3 factors with classical refinement (which stalls: kappa x the factor's
    unit roundoff exceeds 1) and with CG preconditioned by them. Keeps each
    form's solution for the comparison with the oracle."""
    A, nrhs = inputs.workload(2)
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, nd_leaf=8, pr=True, variant="rlb", merge=args.merge)
    fl = sym.view()["flops"]
    dv = torch.tensor(A.values, device=dev, dtype=torch.float64)
    B = inputs.rhs(A.n, nrhs, inputs.SEED_BASE + 2)
    Bd = torch.tensor(np.ascontiguousarray(B.T), device=dev)
    r = {"workload": A.name, "n": A.n, "nrhs": nrhs, "sum_cj2": fl}
    sols = {}
    for prec in ("fp64", "fp32", "tf32", "tf32x3"):
        nm = sym.factor(dv, precision=prec)
        Xd = torch.zeros_like(Bd)
        (fm, sm_), si = _time_factor_solve(nm, dv, Bd, Xd, stream, 3)
        r[prec] = {"factor_ms": fm, "factor_gflops": fl / (fm * 1e-3) / 1e9, "solve_ms": sm_,
                   "total_ms": fm + sm_, "ir_iterations": si["iterations"], "eta_max": si["eta_max"],
                   "converged": si["converged"], "pivot_fallbacks": nm.info.pivot_fallbacks}
        sols[prec + ("" if prec == "fp64" else "_ir")] = Xd.cpu().numpy().T.copy()
        if prec == "fp64":
            sols["L_fp64"] = nm.export_L()
        else:
            Xc = torch.zeros_like(Bd)
            (fm2, sm2), sc_ = _time_factor_solve(nm, dv, Bd, Xc, stream, 2, method="cg", max_iterations=400)
            r[prec]["cg"] = {"iterations": sc_["iterations"], "eta_max": sc_["eta_max"],
                             "converged": sc_["converged"], "solve_ms": sm2, "total_ms": fm2 + sm2}
            sols[prec + "_cg"] = Xc.cpu().numpy().T.copy()
        nm.free()
    r["_solutions"] = sols
    r["_B"] = B
    r["_A"] = A
    return r


def _workload_80(args, sc, inputs, torch, np, dev, stream):
    A3, nrhs3 = inputs.workload(3)
    sym3 = sc.Symbolic(A3, ordering="grid_nd", grid=A3.grid, nd_leaf=8, pr=True, variant="rlb", merge=args.merge)
    f3 = sym3.view()["flops"]
    dv3 = torch.tensor(A3.values, device=dev, dtype=torch.float64)
    B3d = torch.tensor(np.ascontiguousarray(inputs.rhs(A3.n, nrhs3, inputs.SEED_BASE + 3).T), device=dev)
    r = {"workload": A3.name, "n": A3.n, "sum_cj2": f3, "nrhs": nrhs3}
    for prec, reps in (("tf32", 3), ("tf32x3", 3), ("fp64", 2)):
        nm = sym3.factor(dv3, precision=prec)
        (fm, sm_), si = _time_factor_solve(nm, dv3, B3d, torch.zeros_like(B3d), stream, reps)
        r[prec] = {"factor_ms": fm, "factor_gflops": f3 / (fm * 1e-3) / 1e9, "solve_ms": sm_, "total_ms": fm + sm_,
                   "eta_max": si["eta_max"], "ir_iterations": si["iterations"], "converged": si["converged"]}
        nm.free()
    r["speedup_total"] = r["fp64"]["total_ms"] / min(r["tf32"]["total_ms"], r["tf32x3"]["total_ms"])
    return r


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
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "tf32x3"],
                    help="precision of the timed steps (the headline is FP64)")
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--merge", type=float, default=0.125, help="supernode merging budget (Sec. 3.1); 0 = off")
    ap.add_argument("--workload", type=int, default=5, choices=[2, 3, 5],
                    help="5: the headline (128^3 anisotropic); 2: 48^3 7-point; 3: 80^3 27-point (profiling)")
    ap.add_argument("--scale", type=float, default=1.0, help="grid-side scale of the workload (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-chosen", action="store_true", help="skip the TF32x3 + CG form on the same matrix")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-plan autotuner's measurement")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel-class profile")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during a timed region."""

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


# ---------------------------------------------------------------- CPU baseline (oracle)
def _nd_boxes(dims, leaf, target):
    """Boxes of the geometric nested dissection (split the longest axis, ties
    x, y, z, at lo + len // 2; order: left box, right box, separator plane) that
    hold at most `target` points, with the position of their first point in the
    ordering. Integer bookkeeping of the ordering only (which positions one
    subtree spans); it computes nothing of the factorization."""
    out = []

    def rec(lo, hi, pos):
        size = [hi[a] - lo[a] for a in range(3)]
        vol = size[0] * size[1] * size[2]
        if vol <= target or vol <= leaf:
            out.append((pos, vol, tuple(lo), tuple(hi)))
            return
        ax = max(range(3), key=lambda a: (size[a], -a))
        m = lo[ax] + size[ax] // 2
        lhi = list(hi)
        lhi[ax] = m
        rlo = list(lo)
        rlo[ax] = m + 1
        lvol = vol // size[ax] * (m - lo[ax])
        rec(list(lo), lhi, pos)
        rec(rlo, list(hi), pos + lvol)

    rec([0, 0, 0], list(dims), 0)
    return out


def _principal_block(A, perm, start, count):
    """Lower triangle (CSC) of the leading principal block of P A P^T that the
    positions start .. start + count - 1 of the ordering span, in that order."""
    import numpy as np
    import scipy.sparse as sp

    from paper_2409_13090_gb300.inputs import SparseSym
    lower = sp.csc_matrix((A.values, A.rowind, A.colptr), shape=(A.n, A.n))
    full = (lower + lower.T - sp.diags(lower.diagonal())).tocsc()
    idx = perm[start:start + count]
    sub = sp.tril(full[idx][:, idx]).tocsc()
    sub.sort_indices()
    return SparseSym(count, sub.indptr.astype(np.int64), sub.indices.astype(np.int32), sub.data.astype(np.float64),
                     (0, 0, 0), f"{A.name} principal block [{start}, {start + count})")


def _oracle_time(Asub, reps):
    """Oracle Alg. 1 column Cholesky of a sample in the order given (natural):
    (sum c_j^2, seconds of each factorization)."""
    import oracle
    o = oracle.Oracle(Asub, None, pr=True)
    flops = o.symbolic().flops
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        info = o.factor()
        times.append(time.perf_counter() - t0)
        assert info == 0, info
    return flops, times


def _oracle_worker(Asub):
    f, t = _oracle_time(Asub, 1)
    return f, t[0]


def _oracle_warm(_):
    import oracle
    oracle.lib()
    return os.getpid()


def _cpu_sample_matrix(A):
    """The headline matrix's sample for the oracle: the leading subtree of the
    nested dissection with at most SAMPLE_VOLUME points, as its principal block."""
    import oracle
    perm = oracle.nd_grid(*A.grid, 8)
    boxes = _nd_boxes(A.grid, 8, SAMPLE_VOLUME)
    pos, vol, lo, hi = boxes[0]
    return perm, boxes, _principal_block(A, perm, pos, vol), (lo, hi)


def _cpu_baseline(A, reps, all_cores=True):
    """The oracle as it stands, on the host cores: one core on the leading
    subtree block of the headline matrix, and (all_cores) one process per core
    on as many disjoint subtree blocks at once (whole-job GFLOP/s)."""
    import multiprocessing as mp

    import numpy as np
    perm, boxes, Asub, (lo, hi) = _cpu_sample_matrix(A)
    flops, times = _oracle_time(Asub, reps)
    one = flops / min(times) / 1e9
    sample = (f"oracle Alg. 1 column Cholesky (FP64, gcc -O2, 1 thread) of the leading principal block of "
              f"P A P^T of the headline matrix ({A.name}) spanned by one nested-dissection subtree: grid box "
              f"{lo}-{hi}, n = {Asub.n}, sum c_j^2 = {flops:.4e}")
    out = {"value": one, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample,
           "sample_n": Asub.n, "sample_sum_cj2": flops, "sample_seconds": min(times)}
    if all_cores:
        cores = len(os.sched_getaffinity(0))
        subs = [_principal_block(A, perm, p, v) for p, v, _, _ in boxes[:cores]]
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_warm, range(4 * cores))  # workers started, oracle loaded
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, subs, chunksize=1)
            wall = time.perf_counter() - t0
        tot = float(np.sum([f for f, _ in res]))
        out["all_cores"] = {"value": tot / wall / 1e9, "unit": "GFLOP/s", "cores": cores, "blocks": len(subs),
                            "sum_cj2": tot, "wall_s": wall,
                            "sample": f"{len(subs)} disjoint nested-dissection subtree blocks of the same matrix "
                                      f"(about {SAMPLE_VOLUME} unknowns each), one process per core (spawn pool started "
                                      f"before the timed region), wall time of the whole map"}
    return out


def _oracle_errors_48(r48):
    """The oracle factors and solves the 48^3 matrix (timed: part of the CPU
    baseline); the GPU results of every form are compared with it."""
    import numpy as np

    import oracle
    A, B, sols = r48["_A"], r48["_B"], r48["_solutions"]
    o = oracle.Oracle(A, oracle.nd_grid(*A.grid, 8), pr=True, merge=0.125)
    t0 = time.perf_counter()
    assert o.factor() == 0
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    Xo = o.solve(B)
    ts = time.perf_counter() - t0
    Lo = o.L_supernodal()
    fl = o.symbolic().flops
    out = {"oracle": {"factor_s": tf, "factor_gflops": fl / tf / 1e9, "solve_s": ts, "cores": 1,
                      "eta_max": float(oracle.backward_error(A, B, Xo).max())}}
    scale = np.abs(Xo).max(axis=0)
    for k, X in sols.items():
        if k == "L_fp64":
            out["L_fp64_rel_max"] = float(np.abs(X - Lo).max() / np.abs(Lo).max())
            out["L_fp64_rel_fro"] = float(np.linalg.norm(X - Lo) / np.linalg.norm(Lo))
            continue
        out["x_" + k] = float((np.abs(X - Xo).max(axis=0) / scale).max())
    out["note"] = ("x: max over right-hand sides of ||x - x_oracle||_inf / ||x_oracle||_inf (kappa ~ 1e9, so FP64 "
                   "solutions of eta ~ 1e-16 may differ by ~1e-7 relative); L: FP64 factor against the oracle's")
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2409_13090_gb300 import inputs
    A, nrhs = inputs.workload(args.workload, args.scale)
    _, _, Asub, (lo, hi) = _cpu_sample_matrix(A)
    flops, times = _oracle_time(Asub, args.warmup + args.steps)
    t = times[args.warmup:]
    val = flops * len(t) / sum(t) / 1e9
    sample = (f"oracle Alg. 1 column Cholesky (FP64, 1 thread) of the leading principal block of P A P^T spanned by "
              f"one nested-dissection subtree (grid box {lo}-{hi}, n = {Asub.n}, sum c_j^2 = {flops:.4e}); "
              f"one factorization per step")
    line = {"metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload] if args.scale == 1.0 else A.name, "n": A.n,
                       "nrhs": nrhs, "precision": "fp64", "sample": sample, "parallelism": "none (host)"},
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
    K, W = args.steps, max(3, args.warmup)
    headline = args.workload == 5 and args.scale == 1.0

    A, nrhs = inputs.workload(args.workload, args.scale)
    t0 = time.perf_counter()
    sym = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, nd_leaf=8, pr=True, variant="rlb", merge=args.merge)
    analyze_s = time.perf_counter() - t0
    view = sym.view()
    flops = view["flops"]
    dv = torch.tensor(A.values, device=dev, dtype=torch.float64)
    B = inputs.rhs(A.n, nrhs, inputs.SEED_BASE + args.workload)
    Bd = torch.tensor(np.ascontiguousarray(B.T), device=dev)  # (nrhs, n) = column-major n x nrhs
    Xd = torch.zeros_like(Bd)
    num = sym.factor(dv, precision=args.precision)
    assert num.rc == 0, num.rc
    for _ in range(W - 1):  # the factor call above was the first warm-up step's factorization
        num.refactor(dv)
    for _ in range(W):
        num.solve(Bd, Xd)
    torch.cuda.synchronize()

    # ---- the timed steps (FP64 by default): refactor + solve, CUDA events on the stream
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    fms, sms, launches, etas, iters, _ = _timed_steps(num, dv, Bd, Xd, stream, K)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    fac_ms, sol_ms = sum(fms), sum(sms)
    fac_ms, sol_ms = reduce_max_over_ranks(dist, [fac_ms, sol_ms], dev)
    value = whole_job_rate(world, flops, K, fac_ms)

    # ---- end to end through host buffers (pinned): H2D values and B, factor, solve, D2H X
    ne2e = max(1, min(K, 3))
    e2e_f, e2e_s, e2e_x = _e2e(num, A, B, stream, ne2e)
    e2e = {"value": world * flops / ((e2e_f + e2e_s) * 1e-3) / 1e9, "unit": "GFLOP/s",
           "definition": "sum c_j^2 / (refactor + solve) with every step's values and B copied host -> device "
                         "and X device -> host inside the timed region",
           "h2d_bytes_per_step": int(A.nnz * 8 + A.n * nrhs * 8), "d2h_bytes_per_step": int(A.n * nrhs * 8),
           "factor_ms": e2e_f, "solve_ms": e2e_s, "steps": ne2e, **e2e_x}

    peaks, peak_kind = _peaks()
    # ---- measured FMA peaks (the SIMT roofline denominators), clocks sampled meanwhile
    pclk = Clocks(local)
    pclk.start()
    time.sleep(0.2)
    fp_peak = {}
    for kind, nm in ((0, "fp64"), (1, "fp32")):
        try:
            fp_peak[nm] = sc.sc_probe_fma_peak(kind) / 1e12
        except Exception:
            fp_peak[nm] = None
    probe_clk = pclk.stop()

    # ---- per-kernel-class profile of the timed precision (CUDA events around every launch)
    rooflines, roofline = {}, None
    if not args.no_profile:
        prof = num.profile(dv)
        rooflines[args.precision] = _class_rooflines(prof, peaks, fp_peak, args.precision, args.workload,
                                                     args.scale, args.merge)
        dom = max(prof, key=lambda k: prof[k]["ms"])
        d = rooflines[args.precision][dom]
        best_seen = max(value / 1e3, d["achieved_tflops"]) if dom != "gemm_tc" else 0.0
        peak = d["peak_tflops"]
        peak_src = (f"TF32 = {peak_kind} bf16 sustained x 1.1/2.25 (nominal tf32/bf16)" if dom == "gemm_tc" else
                    "measured FMA-tile probe (sc_probe_fma_peak)")
        if dom != "gemm_tc" and peak is not None and best_seen > peak:
            peak, peak_src = best_seen, "best rate observed in this run (above the probe)"
        roofline = {"bound": d["bound"], "achieved": d["achieved_tflops"], "peak": peak, "unit": "TFLOP/s",
                    "frac": d["achieved_tflops"] / peak if peak else None, "traffic": d["traffic_bytes"],
                    "kernel": dom, "kernel_launches": d["launches"], "peak_source": peak_src,
                    "achieved_definition": "algorithmic flops of the class in one factorization / summed CUDA-event "
                                           "time of its launches (launches serialised, outside the graph)",
                    "whole_factor_frac": (value / 1e3) / peak if peak else None}

    # ---- the solve against its limits (HBM and FMA rate); the timed solve also forms the
    #      FP64 residual (CSR A)
    s_l = 8 if args.precision == "fp64" else 4
    sweeps = 2 * (1 + (sum(iters) / len(iters) if iters else 0))
    rooflines["solve_" + args.precision] = _solve_roofline(
        view, A.n, nrhs, s_l, sol_ms / K, sweeps, peaks, peak_kind, fp_peak["fp64" if args.precision == "fp64"
                                                                          else "fp32"])

    # ---- the chosen form on the same matrix: TF32x3 factor + CG preconditioned by it to eta <= 1e-14
    chosen = None
    if not args.no_chosen and args.precision == "fp64":
        numc = sym.factor(dv, precision="tf32x3")
        assert numc.rc == 0, numc.rc
        ckw = {"method": "cg", "max_iterations": 1000}
        Xc = torch.zeros_like(Bd)
        for _ in range(2):
            numc.refactor(dv)
            numc.solve(Bd, Xc, **ckw)
        kc = max(3, min(K, 10))
        cf, cs, cl, ce, ci, cc = _timed_steps(numc, dv, Bd, Xc, stream, kc, **ckw)
        cfm, csm = sum(cf) / kc, sum(cs) / kc
        ce2e_f, ce2e_s, ce2e_x = _e2e(numc, A, B, stream, ne2e, **ckw)
        chosen = {"precision": "tf32x3", "solve": "conjugate gradients preconditioned by the factor (FP64 vectors)",
                  "steps": kc, "factor_ms": cfm, "solve_ms": csm, "total_ms": cfm + csm,
                  "factor_gflops": flops / (cfm * 1e-3) / 1e9, "iterations": max(ci), "eta_max": max(ce),
                  "converged": all(cc), "gpu_launches": cl,
                  "speedup_total_vs_fp64": (fac_ms + sol_ms) / K / (cfm + csm),
                  "e2e": {"factor_ms": ce2e_f, "solve_ms": ce2e_s, "total_ms": ce2e_f + ce2e_s,
                          "speedup_vs_fp64_e2e": (e2e_f + e2e_s) / (ce2e_f + ce2e_s), **ce2e_x}}
        if not args.no_profile:
            profc = numc.profile(dv)
            for _ in range(2):
                p = numc.profile(dv)
                for k in p:
                    profc[k]["ms"] += p[k]["ms"]
            for k in profc:
                profc[k]["ms"] /= 3
            rooflines["tf32x3"] = _class_rooflines(profc, peaks, fp_peak, "tf32x3", args.workload, args.scale,
                                                   args.merge)
            rooflines["solve_tf32x3_cg"] = _solve_roofline(view, A.n, nrhs, 4, csm, 2 * (1 + max(ci)), peaks,
                                                           peak_kind, fp_peak["fp32"])
            rooflines["solve_tf32x3_cg"]["note"] = ("(1 + CG iterations) triangular solves over the FP32 factor; "
                                                    "the FP64 SpMV and vector updates are in the time, not in the floor")
        # ---- the launch-plan autotuner (sc_tune) on the chosen form of the same matrix
        if not args.no_tune:
            try:
                sym_t = sc.Symbolic(A, ordering="grid_nd", grid=A.grid, nd_leaf=8, pr=True, variant="rlb",
                                    merge=args.merge)
                t0 = time.perf_counter()
                table = sym_t.tune(dv, precision="tf32x3", reps=3)
                tune_s = time.perf_counter() - t0
                num_t = sym_t.factor(dv, precision="tf32x3")

                def _factor_ms(h, reps=5):
                    for _ in range(2):
                        h.refactor(dv)
                    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                           for _ in range(reps)]
                    torch.cuda.synchronize()
                    for a, b in evs:
                        a.record(stream)
                        h.refactor(dv)
                        b.record(stream)
                    torch.cuda.synchronize()
                    return sum(a.elapsed_time(b) for a, b in evs) / reps

                ms_tuned, ms_default = _factor_ms(num_t), _factor_ms(numc)
                chosen["tune"] = {"table": {k: table[k] for k in sc.TUNE_FIELDS}, "settings_timed": table["tried"],
                                  "tune_s": tune_s, "factor_ms_default": ms_default, "factor_ms_tuned": ms_tuned,
                                  "note": "0 = library default; the timed steps use the default plan"}
                num_t.free()
                del sym_t
            except Exception as ex:  # reported, not fatal: the headline is already measured
                chosen["tune"] = {"error": str(ex)}
        numc.free()

    others = None
    if not args.no_others and headline and rank == 0:
        others = _other_workloads(args, sc, inputs, torch, np, dev, stream, sym, A, dv, Bd, flops)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(A, 2)
        if others and "diffusion_48" in others:
            try:
                others["errors_vs_oracle_diffusion_48"] = _oracle_errors_48(others["diffusion_48"])
            except Exception as ex:
                others["errors_vs_oracle_diffusion_48"] = {"error": str(ex)}
    if others and "diffusion_48" in others:
        for k in ("_solutions", "_B", "_A"):
            others["diffusion_48"].pop(k, None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": (fac_ms + sol_ms) / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOADS[args.workload] if args.scale == 1.0 else A.name, "n": A.n,
                           "nnz_A_lower": A.nnz, "nnz_L": int(view["nnzL"]), "sum_cj2": flops,
                           "nsuper": int(view["nsuper"]), "blocks": int(len(view["blk_first"])), "nrhs": nrhs,
                           "precision": args.precision, "variant": "rlb", "ordering": "grid ND (leaf 8) + PR",
                           "merge_frac": args.merge,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (factor storage rewritten every step)",
                           "analyze_s": analyze_s},
                "factor_ms": fac_ms / K, "solve_ms": sol_ms / K, "eta_max": max(etas),
                "ir_iterations": max(iters), "gpu_launches": launches, "clocks": clk, "e2e": e2e,
                "roofline": roofline, "rooflines": rooflines,
                "fma_peak_tflops": dict(fp_peak, clocks=probe_clk), "chosen_form": chosen, "cpu_baseline": cpu,
                "other_workloads": others}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
