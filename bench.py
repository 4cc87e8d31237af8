#!/usr/bin/env python3
"""Benchmark of the HEOM hot path on GB300.

Workload (the configuration the headline metric is quoted on): single-impurity Anderson
model, d = 4, eps = -5, U = 10, two Lorentzian leads (Gamma = 2, W = 10, kT = 0.5,
mu = +-1), Pade with 2 poles (3 exponents per lead x spin x nu = 24 fermionic exponents),
tier 3 -> 2,325 ADOs. One step = the stationary state (M rho = 0, Tr rho = 1) plus the
density of states at 1,000 frequencies in [-20, 20] (2,000 shifted odd-parity solves), both
to a 1e-8 FP64 residual with the chosen form (FP32 BiCGStab inside FP64 refinement, all
frequencies batched into one solve). Inputs are synthetic (the paper's parameters; no data).

Reported: ADO-applies/s of the whole step (value), the roofline of the dominant kernel
class measured live with CUDA events, the end-to-end rate through the public API from host
buffers (e2e), steady solves/s and spectrum points/s of the chosen form against the plain
FP64 path, and the CPU oracle on a bounded sample (cpu_baseline).

``--impl reference`` times the CPU oracle (the only reference this project has) on the
same workload and unit; under torchrun only rank 0 runs it.
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
N_OMEGA = 1000
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
    import numpy as np

    import workloads as W
    model = W.siam_model(tier=3)
    om = W.omega_grid(N_OMEGA) + 1e-3 * rank  # each replica its own grid (weak scaling)
    return model, np.asarray(om)


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

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("gloo")
    model, om = _workload(rank)
    d = model.d
    dop = model.fermion_baths[0][0]

    # setup (untimed): exponents, hierarchies, buffers
    even = heom.build_hierarchy(heom.problem_from_model(model, 1))
    odd = heom.build_hierarchy(heom.problem_from_model(model, -1))
    N = even.n_ado
    x_ss = torch.zeros((N, d, d), dtype=torch.complex128, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # chosen form: the stationary state of one parameter set by FP64 BiCGStab in one
    # cooperative launch (a single column is latency-bound: FP32 inner solves would only add
    # refinement restarts), the shift-invariant Arnoldi solve for all frequencies of the DOS
    def step(steady_prec=heom.FP64, spec_prec=heom.SHIFTED):
        st1, s1 = heom.steady(even, x_ss, tol=TOL, max_iter=4000, prec=steady_prec)
        A, st2, s2 = heom.spectrum(odd, x_ss, dop, om, tol=TOL, max_iter=4000, prec=spec_prec)
        return A, s1, s2

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K chosen-form steps, no launch accounting (its CUDA events between
    # kernels would add to the step time)
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

    # roofline of the dominant kernel class (largest device time in the timed region)
    dom = max(prof, key=lambda c: prof[c]["ms"])
    pk, pk_kind = _peaks()
    achieved = prof[dom]["bytes"] / (prof[dom]["ms"] / 1e3) / 1e9 if prof[dom]["ms"] > 0 else 0.0
    traffic = _traffic_record(dom)
    roofline = {"bound": "hbm", "kernel_class": dom, "achieved": round(achieved, 1),
                "peak": pk, "unit": "GB/s", "frac": round(achieved / pk, 4),
                "peak_source": f"{pk_kind} hbm_gbs",
                "traffic": traffic, "launches": prof[dom]["launches"],
                "avg_launch_us": round(1e3 * prof[dom]["ms"] / max(prof[dom]["launches"], 1), 2),
                "algorithmic_bytes_per_launch": prof[dom]["bytes"] / max(prof[dom]["launches"], 1),
                "share_of_step": round(prof[dom]["ms"] / prof_step_ms, 4),
                "measured_in": "a second pass of the K timed steps with per-launch CUDA events"}
    classes = {c: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None}
               for c, v in prof.items() if v["launches"]}

    # residual / iteration summary of the last step
    s1, s2 = stats[-1]
    worst_res = max([s1[0]["residual"]] + [x["residual"] for x in s2])
    iters = [x["iterations"] for x in s2]

    out_extra = {}
    if rank == 0 and not args.quick:
        out_extra.update(_plain_vs_chosen(heom, torch, dev, model, om, even, odd, x_ss, dop,
                                          step_ms / args.steps))
        out_extra["e2e"] = _e2e(heom, torch, model, om, dop, min(args.steps, 3))
        out_extra["apply_roofline"] = _apply_roofline(heom, torch, model)
        out_extra["cpu_baseline"] = _cpu_baseline(model)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+c128",
        "data": "synthetic (paper parameters; no dataset)",
        "config": {"workload": "SIAM d=4 tier 3 (2,325 ADOs, 24 Pade exponents): stationary "
                               "state + DOS at 1,000 omega in [-20,20], residual 1e-8",
                   "n_ado": N, "n_omega": N_OMEGA, "columns_per_dos_solve": 2 * N_OMEGA,
                   "solver": "stationary: FP64 BiCGStab, one cooperative persistent launch; "
                             "DOS: shift-invariant Arnoldi (FP64 apply, float-float Gram-"
                             "Schmidt; one Krylov space per sign for all frequencies)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed (256 MB write) before every timed step"},
        "roofline": roofline,
        "kernel_classes": classes,
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed": round(wall, 3),
        "ms_per_step_with_launch_events": round(prof_step_ms / args.steps, 3),
        "spectrum_points_per_s": round(args.steps * len(om) / (step_ms / 1e3), 1),
        "worst_residual": worst_res,
        "dos_iterations": {"min": min(iters), "max": max(iters), "mean": round(sum(iters) / len(iters), 1)},
    }
    line.update(out_extra)
    if "e2e" not in line:
        line["e2e"] = None
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def _apply_roofline(heom, torch, model, batch=1024, reps=5):
    """The apply alone on an L2-exceeding batch (the workload's hierarchy x 1,024 FP32
    columns, 305 MB per vector) after the autotuner's choice: algorithmic GB/s and the
    fraction of the measured HBM copy bandwidth."""
    g = heom.build_hierarchy(heom.problem_from_model(model, 1))
    tune = heom.autotune(g, batch, heom.FP32)
    gen = torch.Generator(device="cuda").manual_seed(2306)
    x = torch.randn((g.n_ado, model.d, model.d, batch), dtype=torch.complex64, device="cuda",
                    generator=gen)
    y = torch.empty_like(x)
    for _ in range(3):
        heom.apply(g, x, y)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        heom.apply(g, x, y)
    b.record()
    torch.cuda.synchronize()
    us = 1e3 * a.elapsed_time(b) / reps
    byts = 2.0 * g.n_ado * model.d ** 2 * 8 * batch
    pk, kind = _peaks()
    gbps = byts / (us * 1e-6) / 1e9
    return {"kernel": "heom_apply (FP32)", "columns": batch, "us_per_launch": round(us, 2),
            "ado_applies_per_s": round(g.n_ado * batch / (us * 1e-6), 1),
            "achieved_GBps": round(gbps, 1), "peak_GBps": pk, "frac": round(gbps / pk, 4),
            "peak_source": f"{kind} hbm_gbs", "autotune": tune,
            "note": "inputs (305 MB) exceed L2; back-to-back launches"}


def _plain_vs_chosen(heom, torch, dev, model, om, even, odd, x_ss, dop, chosen_step_ms):
    """Stationary solves/s and spectrum points/s of the chosen form against plain FP64."""
    import numpy as np

    import workloads as W
    res = {}
    # spectrum: one plain FP64 step (stationary + all frequencies), timed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    heom.steady(even, x_ss, tol=TOL, max_iter=4000, prec=heom.FP64)
    A64, st, s64 = heom.spectrum(odd, x_ss, dop, om, tol=TOL, max_iter=4000, prec=heom.FP64)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    res["spectrum_points_per_s_plain_fp64"] = round(len(om) / plain_s, 1)
    res["step_speedup_chosen_vs_plain"] = round(plain_s * 1e3 / chosen_step_ms, 2)
    # the mixed-precision batched BiCGStab form of the same step, for reference
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    heom.steady(even, x_ss, tol=TOL, max_iter=4000, prec=heom.MIXED)
    Am, st, sm = heom.spectrum(odd, x_ss, dop, om, tol=TOL, max_iter=4000, prec=heom.MIXED)
    torch.cuda.synchronize()
    res["spectrum_points_per_s_mixed_bicgstab"] = round(len(om) / (time.perf_counter() - t0), 1)
    # stationary states of many parameter sets (learned-warm-start workload shape)
    n_sets = 256
    draws = W.draw_warmstart_samples(n_sets, seed=7522)
    Hs, coefs, rates = [], [], []
    for U, eps, G, kT, mu in draws:
        p = heom.problem_from_model(W.siam_model(eps=eps, U=U, Gamma=G, kT=kT, mu=mu, tier=3))
        Hs.append(p["H"])
        coefs.append(np.concatenate([b["coef"] for b in p["baths"]]))
        rates.append(np.concatenate([b["rate"] for b in p["baths"]]))
    batch = heom.build_hierarchy(heom.problem_from_model(model, 1))
    heom.set_params(batch, np.array(Hs), np.array(coefs), np.array(rates))
    xb = torch.zeros((batch.n_ado, 4, 4, n_sets), dtype=torch.complex128, device=dev)
    heom.steady(batch, xb, tol=TOL, max_iter=4000, prec=heom.MIXED)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stb, sb = heom.steady(batch, xb, tol=TOL, max_iter=4000, prec=heom.MIXED,
                          raise_on_error=False)
    torch.cuda.synchronize()
    chosen_rate = n_sets / (time.perf_counter() - t0)
    # plain: one FP64 solve per call, on the first 8 sets
    single = heom.build_hierarchy(heom.problem_from_model(model, 1))
    x1 = torch.zeros((single.n_ado, 4, 4), dtype=torch.complex128, device=dev)
    n_plain = 8
    t0 = time.perf_counter()
    for j in range(n_plain):
        heom.set_params(single, np.array(Hs[j:j + 1]), np.array(coefs[j:j + 1]),
                        np.array(rates[j:j + 1]))
        heom.steady(single, x1, tol=TOL, max_iter=4000, prec=heom.FP64, raise_on_error=False)
    torch.cuda.synchronize()
    plain_rate = n_plain / (time.perf_counter() - t0)
    res["steady_solves_per_s"] = {
        "chosen": round(chosen_rate, 1), "plain": round(plain_rate, 1),
        "chosen_form": f"MIXED, {n_sets} parameter sets batched", "plain_form": "FP64, one per call",
        "worst_residual_chosen": max(x["residual"] for x in sb),
        "all_converged": all(x["status"] == 0 for x in sb)}
    return res


def _e2e(heom, torch, model, om, dop, n_steps):
    """Same metric through the public API from host inputs: exponents and hierarchies built
    from the physical parameters (tables copied to the device), both solves, A(w) back on
    the host, hierarchies destroyed -- every step."""
    heom.profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_steps):
        even = heom.build_hierarchy(heom.problem_from_model(model, 1))
        odd = heom.build_hierarchy(heom.problem_from_model(model, -1))
        x = torch.zeros((even.n_ado, model.d, model.d), dtype=torch.complex128, device="cuda")
        heom.steady(even, x, tol=TOL, max_iter=4000, prec=heom.FP64)
        A, _, _ = heom.spectrum(odd, x, dop, om, tol=TOL, max_iter=4000, prec=heom.SHIFTED)
        del even, odd, x
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    prof = heom.profile_read()
    h2d, d2h = heom.profile_copies()
    heom.profile_enable(False)
    applies = sum(prof[c]["units"] for c in heom.APPLY_CLASSES)
    return {"value": round(applies / dt, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d / n_steps), "d2h_bytes_per_step": int(d2h / n_steps),
            "steps": n_steps, "ms_per_step": round(1e3 * dt / n_steps, 2)}


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


def _cpu_baseline(model):
    """The CPU oracle, as it stands, on a bounded sample of the same workload: its apply
    (scipy CSR SpMV, single-threaded) in the metric's unit, plus its own solvers (sparse LU)
    for one stationary state and one frequency of the DOS."""
    import numpy as np

    from oracle import hierarchy as hy
    from oracle import liouvillian as lv
    from oracle import solvers as so
    prob = hy.model_to_problem(model)
    h = hy.problem_hierarchy(prob)
    t0 = time.perf_counter()
    M = lv.build_matrix(prob, h)
    t_build = time.perf_counter() - t0
    applies, dt = _oracle_apply_rate(M, h.n_ado, model.d, reps=10)
    t0 = time.perf_counter()
    X = so.steady_state(M, model.d)
    t_ss = time.perf_counter() - t0
    Mo = lv.build_matrix(hy.model_to_problem(model, -1), h)
    t0 = time.perf_counter()
    so.dos(Mo, X, model.fermion_baths[0][0], np.array([0.5]))
    t_w = time.perf_counter() - t0
    return {"value": round(applies / dt, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"10 CSR SpMVs of 32 ADO vectors on the {h.n_ado}-ADO matrix "
                       f"({t_build:.1f} s to assemble); one sparse-LU stationary solve; one "
                       f"DOS frequency (two sparse-LU solves); host cores {os.cpu_count()}, "
                       "scipy SpMV and SuperLU single-threaded"),
            "steady_solves_per_s": round(1.0 / t_ss, 4),
            "spectrum_points_per_s": round(1.0 / t_w, 4)}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import hierarchy as hy
    from oracle import liouvillian as lv
    model, om = _workload(0)
    prob = hy.model_to_problem(model)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    for _ in range(args.warmup):
        _oracle_apply_rate(M, h.n_ado, model.d, reps=2)
    tot_a, tot_t = 0, 0.0
    for _ in range(args.steps):
        a_, t_ = _oracle_apply_rate(M, h.n_ado, model.d, reps=5)
        tot_a += a_
        tot_t += t_
    res = {"value": tot_a / tot_t, "ms_per_step": 1e3 * tot_t / args.steps, "n_ado": h.n_ado,
           "cores": 1,
           "sample": ("each step: 5 CSR SpMVs (scipy, single-threaded) of 32 ADO vectors on "
                      f"the oracle's assembled {h.n_ado}-ADO matrix; host cores {os.cpu_count()}")}
    line = {
        "impl": "reference", "metric": METRIC, "value": round(res["value"], 1), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(res["ms_per_step"], 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic (paper parameters; no dataset)",
        "config": {"workload": "SIAM d=4 tier 3 (2,325 ADOs, 24 Pade exponents): stationary "
                               "state + DOS at 1,000 omega in [-20,20], residual 1e-8",
                   "n_ado": res["n_ado"]},
        "cpu_baseline": {"value": round(res["value"], 1), "unit": UNIT, "cores": res["cores"],
                         "kind": "oracle", "sample": res["sample"]},
        "e2e": {"value": round(res["value"], 1), "unit": UNIT, "h2d_bytes_per_step": 0,
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
                      "frac_hbm": round(byts / (us * 1e-6) / 1e9 / pk, 4), "peak": kind}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no plain-path, e2e or CPU-baseline legs)")
    ap.add_argument("--only", choices=["apply"], default=None,
                    help="kernel micro-benchmark (for profiling) instead of the step benchmark")
    ap.add_argument("--batch", type=int, default=2000)
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args()
    if args.only == "apply":
        run_apply_only(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
