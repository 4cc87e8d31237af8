#!/usr/bin/env python3
"""Benchmark of the HEOM hot path on GB300.

Workload (the batched-spectra configuration, the largest that fits one GPU): 64 single-
impurity Anderson models (d = 4, eps = -5, Gamma = 2, W = 10, Pade with 2 poles: 24 fermionic
exponents), parameters drawn with seed 7522: U ~ U[0,12], bias mu ~ U[0,3], kT ~ U[0.2,1]
outside [0.68, 0.87], tier ~ {2,3,4} (301 / 2,325 / 12,951 ADOs). All 64 sets live in one
hierarchy of the tier-4 structure, each truncated at its own tier (deepest sets first). One
step = the stationary states of all 64 sets (one batched mixed-precision solve: FP32
BiCGStab inside FP64 refinement) plus the density of states of every set at 4,096
frequencies on [-20, 20] (524,288 shifted solves; one shift-invariant Arnoldi process per set
and sign, all 128 in one batched solve), every residual at 1e-8. Inputs are synthetic (the
paper's parameters; no data).

Reported: ADO-applies/s of the whole step (value; an ADO-apply is one output d x d block of
one column of M x, for the ADOs each set keeps), spectrum points/s, the roofline of the
dominant kernel class measured live with CUDA events, the end-to-end rate through the public
API from host parameters (e2e), and as extras: the tiled apply on an L2-exceeding batch and at
the paper's Example 1 scale, the previous single-model step (stationary state + DOS at 1,000
frequencies), stationary solves/s of 256 parameter sets with each factor of the chosen form
separately (plain FP64, batching, mixed precision), the charge-cavity model (d = 24), dense
operators at d = 16, 24, 32, a measured FP64 peak, and the CPU oracle on a bounded sample
(cpu_baseline).

``--impl reference`` times the CPU oracle (the only reference this project has) on a sample
of the same workload in the same unit; under torchrun only rank 0 runs it.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADO-applies/s (% HBM roofline); steady solves/s at 1e-8 res, chosen vs plain"
UNIT = "ADO-applies/s"
TOL = 1e-8
N_SETS = 64        # batched-spectra parameter sets
N_OMEGA_C3 = 4096  # frequencies per set
N_OMEGA = 1000     # frequencies of the single-model step (extra)
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _workload(rank: int = 0):
    """The single-model workload (SIAM tier 3, 1,000 frequencies): the extra C2 step."""
    import numpy as np

    import workloads as W
    model = W.siam_model(tier=3)
    om = W.omega_grid(N_OMEGA) + 1e-3 * rank  # each replica its own grid (weak scaling)
    return model, np.asarray(om)


def c3_draws():
    """The 64 drawn SIAM parameter sets, deepest tier first (each ADO is then kept by a
    leading run of sets, which the Gram-Schmidt kernels use to skip zero columns)."""
    import workloads as W
    return sorted(W.draw_siam_sets(N_SETS), key=lambda d: -d["tier"])


def c3_models(draws):
    import workloads as W
    return [W.siam_model(U=d["U"], mu=d["mu"], kT=d["kT"], tier=4) for d in draws]


def c3_build(heom, draws, models):
    """Even and odd hierarchies of the tier-4 structure holding every set, each truncated at
    its own tier: the public-API construction of the batched-spectra workload."""
    tiers = [d["tier"] for d in draws]
    out = []
    for parity in (1, -1):
        g = heom.build_hierarchy(heom.problem_from_model(models[0], parity))
        heom.set_params_from_models(g, models, parity)
        heom.set_truncation(g, [0] * len(draws), tiers)
        out.append(g)
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        with open(self.file.name) as f:
            rows = [[c.strip() for c in line.split(",")] for line in f if line.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for name, flag in zip(names, r[5:9]):
                if flag.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def _traffic_record(kernel_class: str):
    """ncu DRAM bytes per launch recorded under profiles/, valid only while the source files
    that define the measured kernels (the record's "sources", in csrc/) are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    entry = rec.get(kernel_class)
    if not entry or not entry.get("sources"):
        return None
    src = os.path.join(ROOT, "paper_2306_07522_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(entry["sources"]):
        with open(os.path.join(src, name), "rb") as f:
            h.update(f.read())
    if entry.get("sources_sha256") != h.hexdigest():
        return None
    return entry.get("dram_bytes_per_launch")


def reduce_over_ranks(seconds: float, units: float, world_size: int):
    """Whole-job numbers of a replicated run: the slowest rank's time and the units all ranks
    processed (weak scaling: every rank solves its own copy of the workload)."""
    if world_size <= 1:
        return seconds, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2306_07522_gb300 as heom
    import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("gloo")
    draws = c3_draws()
    models = c3_models(draws)
    om = np.asarray(W.omega_grid(N_OMEGA_C3)) + 1e-3 * rank  # each replica its own grid
    dop = models[0].fermion_baths[0][0]

    # setup (untimed): exponents, hierarchies, truncation, buffers
    even, odd = c3_build(heom, draws, models)
    N = even.n_ado
    x_ss = torch.zeros((N, 4, 4, N_SETS), dtype=torch.complex128, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # chosen form: all 64 stationary states in one batched mixed-precision solve (FP32
    # BiCGStab inside FP64 refinement), then every set's DOS from shift-invariant Arnoldi
    # processes (one per set and sign, all in one batched solve; float-float Gram-Schmidt)
    def step():
        st1, s1 = heom.steady(even, x_ss, tol=TOL, max_iter=4000, prec=heom.MIXED)
        A, st2, s2 = heom.spectrum(odd, x_ss, dop, om, tol=TOL, max_iter=2000, prec=heom.SHIFTED)
        return A, s1, s2

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, no launch accounting (its CUDA events between kernels
    # would add to the step time)
    sampler = ClockSampler(local)
    s = torch.cuda.current_stream()

    def timed(n):
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        t0 = time.perf_counter()
        out = []
        for k in range(n):
            flush.zero_()  # L2 flush between timed steps (outside the step's events)
            ev[k][0].record(s)
            A, s1, s2 = step()
            ev[k][1].record(s)
            out.append((s1, s2))
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        return sum(a.elapsed_time(b) for a, b in ev), time.perf_counter() - t0, out

    step_ms, wall, stats = timed(args.steps)
    clocks = sampler.stop()
    # ---- the same K steps again with the library's launch accounting on: per-class device
    # time (events around every launch, on the launching stream), units and bytes
    heom.profile_enable(True)
    prof_step_ms, _, _ = timed(args.steps)
    prof = heom.profile_read()
    heom.profile_enable(False)

    applies = sum(prof[c]["units"] for c in heom.APPLY_CLASSES)
    launches = sum(v["launches"] for v in prof.values())
    t, applies = reduce_over_ranks(step_ms / 1e3, applies, ws)
    value = applies / t
    points = ws * args.steps * N_SETS * len(om)

    # roofline of the dominant kernel class (largest device time in the timed region)
    dom = max(prof, key=lambda c: prof[c]["ms"])
    pk, pk_kind = _peaks()
    achieved = prof[dom]["bytes"] / (prof[dom]["ms"] / 1e3) / 1e9 if prof[dom]["ms"] > 0 else 0.0
    roofline = {"bound": "hbm", "kernel_class": dom, "achieved": round(achieved, 1),
                "peak": pk, "unit": "GB/s", "frac": round(achieved / pk, 4),
                "peak_source": f"{pk_kind} hbm_gbs",
                "traffic": _traffic_record(dom), "launches": prof[dom]["launches"],
                "avg_launch_us": round(1e3 * prof[dom]["ms"] / max(prof[dom]["launches"], 1), 2),
                "algorithmic_bytes_per_launch": prof[dom]["bytes"] / max(prof[dom]["launches"], 1),
                "share_of_step": round(prof[dom]["ms"] / prof_step_ms, 4),
                "measured_in": "a second pass of the K timed steps with per-launch CUDA events"}
    classes = {c: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None}
               for c, v in prof.items() if v["launches"]}

    s1, s2 = stats[-1]
    out_extra = {}
    # the hierarchies' workspaces go to the library's cache, which the end-to-end steps reuse
    del even, odd, x_ss, flush
    if rank == 0 and not args.quick:
        out_extra["e2e"] = _e2e(heom, torch, draws, models, om, dop, min(args.steps, 2))
        heom.release_workspace_cache()
        torch.cuda.empty_cache()
        out_extra["extras"] = _extras(heom, torch, dev, args)
        out_extra["cpu_baseline"] = _cpu_baseline(draws)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    tiers = [d["tier"] for d in draws]
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+c128",
        "data": "synthetic (paper parameters; no dataset)",
        "config": {"workload": "batched SIAM spectra: 64 parameter sets (seed 7522; tiers 2/3/4 "
                               "-> 301/2,325/12,951 ADOs) x 4,096 omega in [-20,20], stationary "
                               "states + DOS, residual 1e-8",
                   "sets_per_tier": {t: tiers.count(t) for t in (2, 3, 4)},
                   "n_ado_structure": N, "n_omega": len(om), "shifted_systems": 2 * N_SETS * len(om),
                   "solver": "stationary: one batched solve of all sets, FP32 BiCGStab inside FP64 "
                             "refinement; DOS: shift-invariant Arnoldi, one process per set and "
                             "sign (128 columns in one batched solve), FP64 apply, float-float "
                             "Gram-Schmidt, FP64 Hessenberg/rotations; sets truncated at their "
                             "own tiers inside the tier-4 structure",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed (256 MB write) before every timed step"},
        "roofline": roofline,
        "kernel_classes": classes,
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed": round(wall, 3),
        "ms_per_step_with_launch_events": round(prof_step_ms / args.steps, 3),
        "spectrum_points_per_s": round(points / t, 1),
        "steady_solves_per_s": round(ws * args.steps * N_SETS / t, 1),
        "worst_residual": {"stationary": max(x["residual"] for x in s1),
                           "dos": max(x["residual"] for x in s2)},
        "arnoldi_steps": s2[0]["iterations"],
    }
    line.update(out_extra)
    if "e2e" not in line:
        line["e2e"] = None
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def _time_apply(heom, torch, g, d, B, dt, reps=5):
    """Average device time (us) of heom_apply on random columns, after 3 warm-up launches."""
    shape = (g.n_ado, d, d) + ((B,) if B > 1 else ())
    gen = torch.Generator(device="cuda").manual_seed(2306)
    x = torch.randn(shape, dtype=dt, device="cuda", generator=gen)
    y = torch.empty_like(x)
    for _ in range(3):
        heom.apply(g, x, y)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        heom.apply(g, x, y)
    b.record()
    torch.cuda.synchronize()
    return 1e3 * a.elapsed_time(b) / reps


def _fp64_peak(torch):
    """Measured FP64 rate (TFLOP/s): best of 3 cuBLAS DGEMMs of 4096^3 (clocks untouched);
    the denominator of the FP64 apply's FP64 roofline."""
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return 2 * 4096 ** 3 / (best * 1e-3) / 1e12


def _sparse_terms(heom, prob, g):
    """Complex multiply-adds of one column of M x as the term programs hold them: per neighbour
    entry d nnz(O) for the left and d nnz(O) for the right product, per ADO the d^2 damping
    terms and the commutator's terms (for a diagonal H one per off-diagonal element)."""
    import numpy as np
    d = int(prob["d"])
    nnz_of_k = []
    for b in prob["baths"]:
        nnz_of_k += [int(np.count_nonzero(np.asarray(b["op"])))] * len(b["coef"])
    t = heom.export_tables(g)
    ent = 2 * d * np.asarray(nnz_of_k)[t["k"]]
    H = np.asarray(prob["H"])
    sys_terms = d * d - d if np.count_nonzero(H - np.diag(np.diag(H))) == 0 else (2 * d - 1) * d * d
    return int(ent.sum()) + g.n_ado * (d * d + sys_terms)


def _macs_per_column(heom, g, d):
    """Complex multiply-adds of one column of M x when every operator is dense: per output
    element the damping term, 2d - 1 commutator terms and 2d per neighbour entry."""
    import numpy as np
    t = heom.export_tables(g)
    E = np.diff(t["row_ptr"]).astype(np.float64)
    return float(np.sum(d * d * (1 + (2 * d - 1) + 2 * d * E)))


def _extras(heom, torch, dev, args):
    import numpy as np

    import workloads as W
    pk, pk_kind = _peaks()
    fp64_tf = _fp64_peak(torch)
    out = {"fp64_peak_tflops_measured": round(fp64_tf, 2)}
    model, om = _workload(0)
    # (1) the apply alone on an L2-exceeding batch: SIAM tier 3 x 1,024 columns (305 MB per
    # FP32 vector), autotuned; FP64 at the same shape against the FP64 roofline
    g = heom.build_hierarchy(heom.problem_from_model(model, 1))
    tune = heom.autotune(g, 1024, heom.FP32)
    us32 = _time_apply(heom, torch, g, 4, 1024, torch.complex64)
    heom.autotune(g, 1024, heom.FP64)
    us64 = _time_apply(heom, torch, g, 4, 1024, torch.complex128, reps=3)
    terms = _sparse_terms(heom, heom.problem_from_model(model, 1), g)
    b32 = 2.0 * g.n_ado * 16 * 8 * 1024
    fl64 = 8.0 * terms * 1024 / (us64 * 1e-6) / 1e12
    out["apply_L2_exceeding"] = {
        "workload": "SIAM tier 3 (2,325 ADOs) x 1,024 columns", "autotune": tune,
        "fp32_us": round(us32, 1), "fp32_GBps": round(b32 / (us32 * 1e-6) / 1e9, 1),
        "fp32_frac_hbm": round(b32 / (us32 * 1e-6) / 1e9 / pk, 4), "peak_GBps": pk,
        "peak_source": f"{pk_kind} hbm_gbs",
        "fp64_us": round(us64, 1), "fp64_GBps": round(2 * b32 / (us64 * 1e-6) / 1e9, 1),
        "terms_per_column": terms, "fp64_tflops": round(fl64, 3),
        "fp64_frac_of_measured_fp64_peak": round(fl64 / fp64_tf, 3),
        "ado_applies_per_s_fp32": round(g.n_ado * 1024 / (us32 * 1e-6), 1)}
    del g
    # (2) the paper's Example 1 scale (K_f = 56, n_max = 4 and 5), one column
    ps = {}
    for nmax in (4, 5):
        t0 = time.perf_counter()
        gp = heom.build_hierarchy(heom.problem_from_model(W.siam_model(tier=nmax, Gamma=1.0, n_poles=6)))
        r = {"n_ado": gp.n_ado, "build_s": round(time.perf_counter() - t0, 1),
             "terms_per_element": round(float(np.mean(np.diff(heom.export_tables(gp)["row_ptr"]))), 1)}
        for name, dt, sz in (("fp32", torch.complex64, 8), ("fp64", torch.complex128, 16)):
            us = _time_apply(heom, torch, gp, 4, 1, dt)
            gbps = 2 * gp.n_ado * 16 * sz / (us * 1e-6) / 1e9
            r[name] = {"us": round(us, 1), "GBps": round(gbps, 1), "frac_hbm": round(gbps / pk, 4),
                       "ado_applies_per_s": round(gp.n_ado / (us * 1e-6), 1)}
        ps[f"n_max_{nmax}"] = r
        del gp
    out["apply_paper_scale_batch1"] = ps
    # (3) the single-model step: stationary state (FP64, one cooperative launch) + DOS at
    # 1,000 frequencies (shift-invariant)
    even = heom.build_hierarchy(heom.problem_from_model(model, 1))
    odd = heom.build_hierarchy(heom.problem_from_model(model, -1))
    x = torch.zeros((even.n_ado, 4, 4), dtype=torch.complex128, device=dev)
    dop = model.fermion_baths[0][0]
    for k in range(4):
        if k == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        heom.steady(even, x, tol=TOL, max_iter=4000, prec=heom.FP64)
        heom.spectrum(odd, x, dop, om, tol=TOL, max_iter=4000, prec=heom.SHIFTED)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0) / 3
    out["single_model_step"] = {"workload": "SIAM tier 3: stationary state + DOS at 1,000 omega",
                                "ms": round(ms, 2), "spectrum_points_per_s": round(1000 / (ms * 1e-3), 1)}
    del even, odd, x
    out["steady_factors"] = _steady_factors(heom, torch, dev, model)
    out["charge_cavity"] = _charge_cavity(heom, torch, dev)
    out["dense_operators"] = _dense_ops(heom, torch)
    return out


def _steady_factors(heom, torch, dev, model, n_sets=256, n_single=8):
    """Stationary solves/s of 256 warm-start-shaped SIAM sets (tier 3) at 1e-8, each factor of
    the chosen form on its own: plain FP64 one set per call (FP64 applies everywhere), FP64
    with the sets batched, mixed precision batched. Parameters are uploaded before the timed
    region."""
    import numpy as np

    import workloads as W
    draws = W.draw_warmstart_samples(n_sets, seed=7522)
    models = [W.siam_model(eps=e, U=U, Gamma=G, kT=kT, mu=mu, tier=3) for U, e, G, kT, mu in draws]
    res = {}
    # plain: one set per hierarchy and call (sample of n_single sets, parameters set up front)
    singles = []
    for m in models[:n_single]:
        singles.append(heom.build_hierarchy(heom.problem_from_model(m, 1)))
    x1 = torch.zeros((singles[0].n_ado, 4, 4), dtype=torch.complex128, device=dev)
    worst = 0.0
    for prec, key in ((heom.FP64_STRICT, "fp64_strict_single"), (heom.FP64, "fp64_single_persistent")):
        heom.steady(singles[0], x1, tol=TOL, max_iter=4000, prec=prec, raise_on_error=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in singles:
            _, st = heom.steady(g, x1, tol=TOL, max_iter=4000, prec=prec, raise_on_error=False)
            worst = max(worst, st[0]["residual"])
        torch.cuda.synchronize()
        res[key] = round(n_single / (time.perf_counter() - t0), 1)
    del singles
    batch = heom.build_hierarchy(heom.problem_from_model(models[0], 1))
    heom.set_params_from_models(batch, models, 1)
    xb = torch.zeros((batch.n_ado, 4, 4, n_sets), dtype=torch.complex128, device=dev)
    for prec, key in ((heom.FP64, "fp64_batched"), (heom.MIXED, "mixed_batched")):
        heom.steady(batch, xb, tol=TOL, max_iter=4000, prec=prec, raise_on_error=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, sb = heom.steady(batch, xb, tol=TOL, max_iter=4000, prec=prec, raise_on_error=False)
        torch.cuda.synchronize()
        res[key] = round(n_sets / (time.perf_counter() - t0), 1)
        res[key + "_all_converged"] = all(x["status"] == 0 for x in sb)
        worst = max(worst, max(x["residual"] for x in sb))
    res["worst_residual"] = worst
    res["chosen_over_plain"] = round(res["mixed_batched"] / res["fp64_strict_single"], 2)
    res["note"] = (f"{n_sets} sets (seed 7522; U, eps, Gamma, kT, bias drawn), tier 3; single-set "
                   f"rates from the first {n_single} sets")
    return res


def _charge_cavity(heom, torch, dev):
    """The charge-cavity model (d = 24, 790 ADOs): apply throughput, RK4 to t = 50
    (dt = 0.01, 5,000 steps), stationary state."""
    import workloads as W
    m = W.charge_cavity_model()
    g = heom.build_hierarchy(heom.problem_from_model(m))
    r = {"n_ado": g.n_ado, "d": 24}
    for B in (1, 64):
        for name, dt in (("fp32", torch.complex64), ("fp64", torch.complex128)):
            us = _time_apply(heom, torch, g, 24, B, dt)
            r[f"apply_{name}_B{B}_us"] = round(us, 1)
            r[f"apply_{name}_B{B}_ado_applies_per_s"] = round(g.n_ado * B / (us * 1e-6), 1)
    for name, dt in (("fp32", torch.complex64), ("fp64", torch.complex128)):
        x = torch.zeros((g.n_ado, 24, 24), dtype=dt, device=dev)
        x[0] = torch.from_numpy(m.rho0).to(dev, dt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        heom.evolve(g, x, 0.01, 5000)
        torch.cuda.synchronize()
        r[f"rk4_t50_{name}_s"] = round(time.perf_counter() - t0, 2)
    x = torch.zeros((g.n_ado, 24, 24), dtype=torch.complex128, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = heom.steady(g, x, tol=TOL, max_iter=6000, prec=heom.MIXED, raise_on_error=False)
    torch.cuda.synchronize()
    r["steady_mixed_s"] = round(time.perf_counter() - t0, 3)
    r["steady_residual"] = st[0]["residual"]
    return r


def _dense_ops(heom, torch):
    """Dense random H, V and d at d = 16, 24, 32 (the C ABI accepts any operators): the term
    programs do d multiply-adds per element and operator product; achieved FP32 rate against
    the CUDA-core FP32 peak (152 SMs x 128 lanes x 2 flops x clock)."""
    import workloads as W
    peak32 = 152 * 128 * 2 * 2.07e9 / 1e12
    out = {"fp32_cuda_core_peak_tflops_nominal": round(peak32, 1)}
    for d in (16, 24, 32):
        prob = W.random_raw_problem(d, [("RI", 2)], [8], 2, 2, seed=60 + d)
        g = heom.build_hierarchy(prob)
        macs = _macs_per_column(heom, g, d)
        us = _time_apply(heom, torch, g, d, 64, torch.complex64)
        tf = 8 * macs * 64 / (us * 1e-6) / 1e12
        out[f"d{d}"] = {"n_ado": g.n_ado, "batch": 64, "fp32_us": round(us, 1),
                        "fp32_tflops": round(tf, 2), "frac_fp32_peak": round(tf / peak32, 3)}
    return out


def _e2e(heom, torch, draws, models, om, dop, n_steps):
    """Same metric through the public API from host parameters: exponents and both
    hierarchies built from the physical parameters of the 64 sets (tables copied to the
    device), truncation, the stationary solve, the spectrum, A(w) back on the host,
    hierarchies destroyed -- every step."""
    heom.profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_steps):
        even, odd = c3_build(heom, draws, models)
        x = torch.zeros((even.n_ado, 4, 4, N_SETS), dtype=torch.complex128, device="cuda")
        heom.steady(even, x, tol=TOL, max_iter=4000, prec=heom.MIXED)
        A, _, _ = heom.spectrum(odd, x, dop, om, tol=TOL, max_iter=2000, prec=heom.SHIFTED)
        del even, odd, x
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    prof = heom.profile_read()
    h2d, d2h = heom.profile_copies()
    heom.profile_enable(False)
    applies = sum(prof[c]["units"] for c in heom.APPLY_CLASSES)
    return {"value": round(applies / dt, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d / n_steps), "d2h_bytes_per_step": int(d2h / n_steps),
            "steps": n_steps, "ms_per_step": round(1e3 * dt / n_steps, 2),
            "spectrum_points_per_s": round(n_steps * N_SETS * len(om) / dt, 1)}


def _oracle_apply_rate(M, n_ado, d, reps, cols=32, seed=2306):
    """The oracle's apply (CSR sparse matrix times a block of ADO vectors), timed."""
    import numpy as np
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((n_ado * d * d, cols)) + 1j * rng.standard_normal((n_ado * d * d, cols))
    t0 = time.perf_counter()
    for _ in range(reps):
        M @ V
    dt = time.perf_counter() - t0
    return reps * cols * n_ado, dt


def _oracle_sample(draws):
    """The oracle's matrices of two drawn sets (the first of tier 2 and of tier 3): the bounded
    sample of the workload the CPU baseline and the reference arm time."""
    from oracle import hierarchy as hy
    from oracle import liouvillian as lv
    import workloads as W
    out = []
    for tier in (2, 3):
        dr = next(x for x in draws if x["tier"] == tier)
        m = W.siam_model(U=dr["U"], mu=dr["mu"], kT=dr["kT"], tier=tier)
        pe = hy.model_to_problem(m, 1)
        h = hy.problem_hierarchy(pe)
        t0 = time.perf_counter()
        Me = lv.build_matrix(pe, h)
        Mo = lv.build_matrix(hy.model_to_problem(m, -1), h)
        out.append(dict(tier=tier, model=m, n_ado=h.n_ado, Me=Me, Mo=Mo,
                        build_s=time.perf_counter() - t0))
    return out


def _cpu_baseline(draws):
    """The CPU oracle, as it stands, on a bounded sample of the batched-spectra workload: two
    sets (tier 2 and tier 3): its apply (scipy CSR SpMV, single-threaded) in the metric's
    unit; its stationary state and DOS at two frequencies per set (GMRES path; the tier-3
    sparse LU fills in for minutes), as spectrum points/s of the sample."""
    import numpy as np

    from oracle import solvers as so
    sample = _oracle_sample(draws)
    applies, dt = 0, 0.0
    for smp in sample:
        a_, t_ = _oracle_apply_rate(smp["Me"], smp["n_ado"], 4, reps=5)
        applies += a_
        dt += t_
    t0 = time.perf_counter()
    npts = 0
    for smp in sample:
        X = so.steady_state_iterative(smp["Me"], 4, tol=1e-10)
        so.dos_iterative(smp["Mo"], X, smp["model"].fermion_baths[0][0], np.array([-3.0, 4.5]), tol=1e-10)
        npts += 2
    t_sol = time.perf_counter() - t0
    return {"value": round(applies / dt, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"two of the 64 sets (tier 2: {sample[0]['n_ado']} ADOs, tier 3: "
                       f"{sample[1]['n_ado']} ADOs): 5 CSR SpMVs of 32 ADO vectors each, then "
                       f"each set's stationary state and DOS at 2 omega (GMRES); matrices "
                       f"assembled in {sum(x['build_s'] for x in sample):.1f} s; tier-4 sets "
                       f"not sampled; host cores {os.cpu_count()}, scipy single-threaded"),
            "spectrum_points_per_s_sample": round(npts / t_sol, 4)}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    draws = c3_draws()
    sample = _oracle_sample(draws)
    for _ in range(args.warmup):
        for smp in sample:
            _oracle_apply_rate(smp["Me"], smp["n_ado"], 4, reps=1)
    tot_a, tot_t = 0, 0.0
    for _ in range(args.steps):
        for smp in sample:
            a_, t_ = _oracle_apply_rate(smp["Me"], smp["n_ado"], 4, reps=3)
            tot_a += a_
            tot_t += t_
    value = tot_a / tot_t
    sample_txt = (f"each step: 3 CSR SpMVs (scipy, single-threaded) of 32 ADO vectors on the "
                  f"oracle's matrices of a tier-2 and a tier-3 set of the 64 ({sample[0]['n_ado']} "
                  f"and {sample[1]['n_ado']} ADOs); host cores {os.cpu_count()}")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot_t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic (paper parameters; no dataset)",
        "config": {"workload": "batched SIAM spectra: 64 parameter sets (seed 7522; tiers 2/3/4 "
                               "-> 301/2,325/12,951 ADOs) x 4,096 omega in [-20,20], stationary "
                               "states + DOS, residual 1e-8"},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample_txt},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_apply_only(args):
    """Kernel micro-benchmark for profiling: heom_apply on the workload's hierarchy with
    ``--batch`` random columns, ``--warmup`` untimed then ``--steps`` timed launches."""
    import torch

    import paper_2306_07522_gb300 as heom
    model, _ = _workload(0)
    g = heom.build_hierarchy(heom.problem_from_model(model, 1))
    dt = torch.complex64 if args.prec == "fp32" else torch.complex128
    tune = heom.autotune(g, args.batch, heom.FP32 if args.prec == "fp32" else heom.FP64)
    gen = torch.Generator(device="cuda").manual_seed(2306)
    x = torch.randn((g.n_ado, model.d, model.d, args.batch), dtype=dt, device="cuda", generator=gen)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        heom.apply(g, x, y)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        heom.apply(g, x, y)
    b.record()
    torch.cuda.synchronize()
    us = 1e3 * a.elapsed_time(b) / max(args.steps, 1)
    s = 8 if args.prec == "fp32" else 16
    byts = 2.0 * g.n_ado * model.d ** 2 * s * args.batch
    pk, kind = _peaks()
    print(json.dumps({"kernel": "heom_apply", "prec": args.prec, "n_ado": g.n_ado,
                      "batch": args.batch, "us_per_launch": round(us, 2),
                      "ado_applies_per_s": round(g.n_ado * args.batch / (us * 1e-6), 1),
                      "algorithmic_GBps": round(byts / (us * 1e-6) / 1e9, 1),
                      "frac_hbm": round(byts / (us * 1e-6) / 1e9 / pk, 4), "peak": kind,
                      "autotune": tune}))


def run_spectra_only(args):
    """Profiling case of the batched-spectra step: the first --sets of the 64 drawn sets (deepest
    first), --n-omega frequencies, at most --max-iter Arnoldi steps; --steps steps after
    --warmup, timed with CUDA events."""
    import numpy as np
    import torch

    import paper_2306_07522_gb300 as heom
    import workloads as W
    draws = c3_draws()
    # the first sets of each tier, deepest first, so every tier is present
    pick = sorted([d for t in (4, 3, 2) for d in [x for x in draws if x["tier"] == t][:max(1, args.sets // 3)]],
                  key=lambda d: -d["tier"])[:args.sets]
    models = c3_models(pick)
    even, odd = c3_build(heom, pick, models)
    om = np.asarray(W.omega_grid(args.n_omega))
    dop = models[0].fermion_baths[0][0]
    x = torch.zeros((even.n_ado, 4, 4, len(pick)), dtype=torch.complex128, device="cuda")

    def step():
        heom.steady(even, x, tol=TOL, max_iter=4000, prec=heom.MIXED, raise_on_error=False)
        return heom.spectrum(odd, x, dop, om, tol=TOL, max_iter=args.max_iter, prec=heom.SHIFTED,
                             raise_on_error=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        A, st, stats = step()
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": "batched spectra (profiling)", "sets": len(pick),
                      "tiers": [d["tier"] for d in pick], "n_omega": len(om),
                      "arnoldi_steps": stats[0]["iterations"], "status": st,
                      "ms_per_step": round(a.elapsed_time(b) / max(args.steps, 1), 2)}))


def run_steady_only(args):
    """Profiling case of the stationary half of the step: the batched mixed-precision
    stationary solve of all 64 drawn sets (tier-4 structure, each set at its own tier),
    --steps solves after --warmup, timed with CUDA events; per-set iterations printed."""
    import torch

    import paper_2306_07522_gb300 as heom
    draws = c3_draws()
    models = c3_models(draws)
    even, odd = c3_build(heom, draws, models)
    x = torch.zeros((even.n_ado, 4, 4, N_SETS), dtype=torch.complex128, device="cuda")

    def step():
        return heom.steady(even, x, tol=TOL, max_iter=4000, prec=heom.MIXED, raise_on_error=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        st, stats = step()
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": "batched stationary states (profiling)", "sets": N_SETS, "status": st,
                      "iterations": [s["iterations"] for s in stats],
                      "refinements": [s["refinements"] for s in stats],
                      "ms_per_step": round(a.elapsed_time(b) / max(args.steps, 1), 2)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no plain-path, e2e or CPU-baseline legs)")
    ap.add_argument("--only", choices=["apply", "spectra", "steady"], default=None,
                    help="profiling cases: the apply alone, a reduced batched-spectra step, or the stationary solve")
    ap.add_argument("--sets", type=int, default=8, help="--only spectra: parameter sets")
    ap.add_argument("--n-omega", type=int, default=256, help="--only spectra: frequencies")
    ap.add_argument("--max-iter", type=int, default=2000, help="--only spectra: Arnoldi steps")
    ap.add_argument("--batch", type=int, default=2000)
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args()
    if args.only == "apply":
        run_apply_only(args)
        return
    if args.only == "spectra":
        run_spectra_only(args)
        return
    if args.only == "steady":
        run_steady_only(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
