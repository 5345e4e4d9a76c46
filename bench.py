"""Benchmark: PFC time steps per second on the 1024^2 crystal-growth workload
(3 hexagonal seeds, gamma = 0.25, h = pi/4, adaptive dt in [1e-2, 10],
eta = 5000, left-RAS on 64 x 64 cores with one overlap cell per side).

One bench step = one full time step of the scheme (Newton + GMRES + RAS,
energy, mass, adaptive dt) through the C ABI.  The headline is the mixed,
learned-guess form (BF16 subdomain factors applied in FP32; FP32 JVP;
float-float Gram-Schmidt dot products and multi-axpys on a float-pair Krylov
basis; FP64 residual, Newton update, GMRES least squares, energy, mass and time
step), timed with every time step one captured CUDA graph (device-side Newton,
GMRES and line-search control).  Beside it: the same form with the float-float
JVP, the plain FP64 NKS, the FP32 / BF16 factor forms with the phi^n guess, the
same forms at 2048^2 and on the 256^3 BCC case, and the ensemble, mobility,
Neumann and crack workloads.  Per form: iterations, the
per-kernel rooflines of a separate profiled pass, and the errors against the
FP64 oracle's trajectories (tests/golden).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: the time stepper is not sharded across GPUs here; with N > 1 each
rank runs an independent replica (weak scaling) and `value` sums the replicas'
steps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import importlib.util
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "hex1024"
METRIC = "PFC time steps/s (1024^2 2D crystal growth, adaptive dt)"
PREC_NAME = {0: "f64", 1: "f32", 2: "bf16"}

# DRAM bytes (read + write) of one launch from one ncu capture, keyed by (kernel family, factor
# precision, 2D apply kernel); a kernel changed since its capture is left out (traffic null).
TRAFFIC = {("apply", 2, 5): 540.705536e6 + 3.566080e6}


def measured_peaks():
    """HBM copy GB/s and dense BF16 TFLOP/s measured on the GB300s, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d.get("hbm_gbs", 6800.0)), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# FP32 and FP64 arithmetic peaks of one GB300 (152 SMs at 2070 MHz): 128 FP32 lanes per SM,
# 2 flops per FMA; FP64 at 1/64 of the FP32 rate.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = FP32_PEAK_TFLOPS / 64


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="pfc_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- the CPU oracle (cpu_baseline leg)
ORACLE_STEP = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs
w = inputs.workload({workload!r})
p = O.Params(parts=w["parts"], overlap=1, dt_min=w["dt_min"], dt_max=w["dt_max"], eta=w["eta"])
t0 = time.perf_counter()
phi1, info = O.newton_solve(w["phi"], w["dt_max"], w["h"], w["gamma"], p)
el = time.perf_counter() - t0
print(json.dumps({{"seconds": el, "newton_its": info.newton_its, "gmres_its": info.gmres_its,
                  "converged": bool(info.converged), "dt": w["dt_max"]}}))
"""


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_whole_step(threads: int = 1) -> dict:
    """One whole time step of the workload by the FP64 CPU oracle as it stands (Jacobian
    assembly, Schwarz setup with dense block LU, right-preconditioned GMRES(30), line
    search; its own Newton and GMRES counts) at dt = dt_max from the initial field, timed
    in a fresh process with `threads` BLAS threads."""
    code = ORACLE_STEP.format(root=ROOT, workload=WORKLOAD)
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if res.returncode != 0:
        raise RuntimeError("oracle step failed: " + res.stderr[-2000:])
    r = json.loads(res.stdout.strip().splitlines()[-1])
    r["threads"] = threads
    return r


def oracle_text(r: dict) -> str:
    return (f"one whole {WORKLOAD} time step at dt = {r['dt']:g} from the initial field (FP64 oracle: "
            f"{r['newton_its']} Newton, {r['gmres_its']} GMRES iterations, dense block LU, "
            f"{r['threads']} BLAS thread(s)) in {r['seconds']:.1f} s on {cpu_model()} ({os.cpu_count()} cores)")


def reference_arm(args):
    """The base contract's reference arm: the oracle, timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # Each timed step is one whole oracle time step (~1.5 min on one core); the oracle has no
    # state to warm up.  At most two whole steps are timed so that the run ends within minutes.
    nsteps = max(1, min(args.steps, args.reference_steps))
    runs = [oracle_whole_step(1) for _ in range(nsteps)]
    sec = sum(r["seconds"] for r in runs) / nsteps
    v = 1.0 / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": nsteps, "warmup": 0, "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [1024, 1024], "subdomains": [64, 64], "overlap_per_side": 1},
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": oracle_text(runs[0]) + f"; {nsteps} whole step(s) timed, no warm-up"},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if args.reference_all_cores:
        allc = oracle_whole_step(os.cpu_count() or 1)
        line["cpu_baseline"]["all_cores"] = {"value": 1.0 / allc["seconds"], "unit": "steps/s",
                                             "cores": allc["threads"], "sample": oracle_text(allc)}
    print(json.dumps(line))


# ---------------------------------------------------------------- oracle trajectories (tests/golden)
def _goldens():
    spec = importlib.util.spec_from_file_location("goldens", os.path.join(ROOT, "tests", "golden", "goldens.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def golden_errors(case: str, prec: int, learned: bool, **extra) -> dict:
    """Runs a fresh solver of the given form over the steps of an oracle trajectory (committed
    record, written by tests/golden/make_goldens.py from the FP64 oracle) and states the errors
    of the result: max |phi - phi_oracle| over the record's cells after the last step, and the
    largest relative energy error and mass drift over the steps."""
    import numpy as np

    G = _goldens()
    if not os.path.exists(G.path_of(case)):
        return {"golden": case, "missing": True}
    rec = G.load(case)
    s, close = make_solver(rec["meta"]["workload"], prec, learned, **extra)
    try:
        infos = s.run(int(rec["meta"]["steps"]))
        phi = s.get_field()
    finally:
        close()
    e = np.array([i["energy"] for i in infos])
    m = np.array([i["mass"] for i in infos])
    return {"golden": case, "steps": len(infos), "cells": rec["meta"]["field"],
            "max_abs_phi": G.field_error(rec, phi),
            "max_rel_energy": float(np.max(np.abs(e - rec["energy"]) / np.abs(rec["energy"]))),
            "max_rel_mass_drift": float(np.max(np.abs(m - rec["meta"]["mass0"])) / abs(rec["meta"]["mass0"])),
            "max_rel_dt": float(np.max(np.abs(np.array([i["dt"] for i in infos]) - rec["dt"]) / rec["dt"])),
            "newton_its": [int(i["newton_its"]) for i in infos], "oracle_newton_its": rec["newton_its"].tolist()}


# ---------------------------------------------------------------- multi-GPU replicas
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed over the slowest rank's time (replicas: weak scaling)."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------- solvers
EXTRAS = ("hex2048", "bcc256", "batch32x256", "forms")  # the workloads after the 1024^2 line
# The stopping tolerances of the paper's experiments (Sec. 5: eps_r = 1e-8, eps_a = 1e-10 for Newton,
# xi_r = 1e-3, xi_a = 1e-11 for GMRES).  The other forms use the tighter 1e-10 / 1e-6 of the 64^2
# workload, under which the oracle trajectories were written; these two forms report the same
# workload at the paper's own settings.
PAPER_TOL = {"newton_rtol": 1e-8, "newton_atol": 1e-10, "gmres_rtol": 1e-3, "gmres_atol": 1e-11}
# The headline form: BF16 factors, learned guess, the FP32 JVP inside GMRES (the matrix-vector
# product is not among the parts that stay FP64: residual, Newton update, Arnoldi
# orthogonalisation and least squares, energy, mass, time step).
HEADLINE = "bf16_learned_jvp32"
USE_GRAPH = [1]  # pfc_params.use_graph of every solver (--no-graph for ncu runs)
APPLY_VARIANT = [-1]  # pfc_params.apply_variant of every solver (-1: autotuned; pinned for ncu runs)


def make_solver(workload: str, prec: int, learned: bool = False, stream=True, **form):
    """A solver for a workload (fresh field set), its guess network and a close function."""
    form.setdefault("use_graph", USE_GRAPH[0])
    form.setdefault("apply_variant", APPLY_VARIANT[0])
    import torch

    from paper_1703_01202_gb300 import inputs, pfc
    from paper_1703_01202_gb300 import learned as lrn

    w = inputs.workload(workload)
    params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec, dt_min=w["dt_min"],
                                dt_max=w["dt_max"], eta=w["eta"],
                                guess=pfc.PFC_GUESS_LEARNED if learned else pfc.PFC_GUESS_PREV, **form)
    # a stream of its own: every step runs as one captured graph whenever per-kernel timing is off
    s = pfc.Solver(w["shape"], w["h"], w["gamma"], params, stream=torch.cuda.Stream() if stream else None)
    net = None
    if learned:  # the committed network, trained on 512^2 trajectories of this workload's distribution
        theta, s_out = lrn.load()
        net = pfc.GuessNet(w["shape"])
        net.set_params(theta)
        pfc.set_guess_net(s, net, s_out)
    s.set_field(w["phi"])

    def close():
        s.close()
        if net is not None:
            net.close()
        torch.cuda.empty_cache()

    return s, close


def kernel_rooflines(pk: dict, hbm_gbs: float) -> dict:
    """Per kernel family of the profiled pass: mean launch time, achieved algorithmic GB/s and
    its fraction of the measured HBM copy rate (the factor: achieved TFLOP/s against the FP32 or
    FP64 pipe's peak)."""
    out = {}
    for k, v in pk.items():
        if v["launches"] == 0 or v["ms"] <= 0:
            continue
        sec = v["ms"] * 1e-3
        r = {"launches": v["launches"], "us_per_launch": 1e3 * v["ms"] / v["launches"],
             "achieved_gbs": v["bytes"] / sec / 1e9, "frac_hbm": v["bytes"] / sec / 1e9 / hbm_gbs,
             "stored_over_algorithmic": v["bytes_stored"] / v["bytes"] if v["bytes"] else None}
        if v["flops"] > 0:
            r["achieved_tflops"] = v["flops"] / sec / 1e12
        out[k] = r
    return out


def timed_steps(s, steps: int, world: int, local: int):
    """`steps` adaptive steps of solver s between CUDA events on its stream (barrier and
    synchronise on both sides); returns (ms, infos, clocks, launches)."""
    import torch

    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    from paper_1703_01202_gb300 import pfc

    c0 = pfc.launch_counts()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    infos = s.run(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ck = clocks.stop()
    c1 = pfc.launch_counts()
    launches = {"kernels": c1["kernels"] - c0["kernels"], "graphs": c1["graphs"] - c0["graphs"]}
    return max_over_ranks(world, e0.elapsed_time(e1)), infos, ck, launches


def run_variant(workload: str, prec: int, steps: int, warmup: int, world: int, local: int, learned=False,
                profile_steps=4, e2e=False, golden=None, hbm=6800.0, **extra):
    """Warm-up, `steps` timed steps on the graph path, `profile_steps` more with per-kernel
    events (host-driven GMRES loop), the end-to-end host-buffer steps when asked, and the
    errors against an oracle trajectory."""
    import numpy as np
    import torch

    s, close = make_solver(workload, prec, learned, **extra)
    s.run(warmup)
    tuning = s.tuning()
    ms, infos, ck, launches = timed_steps(s, steps, world, local)
    out = {
        "ms_per_step": ms / steps,
        "steps_per_s": steps / (ms / 1e3),
        "newton_per_step": sum(i["newton_its"] for i in infos) / steps,
        "gmres_per_step": sum(i["gmres_its"] for i in infos) / steps,
        "learned_guess_used": sum(1 for i in infos if i["guess_used"] == 3),
        "dt_last": infos[-1]["dt"],
        "energy_last": infos[-1]["energy"],
        "gpu_launches": launches["kernels"],
        "graph_launches": launches["graphs"],
        "clocks": ck,
        "tuning": tuning,
        "factor_prec": PREC_NAME[prec],
        "phi_after": None,
    }
    if profile_steps > 0:
        s.profile(True)
        s.run(profile_steps)
        pk = s.profile_kernels()
        s.profile(False)
        out["kernels"] = kernel_rooflines(pk, hbm)
        out["profiled_steps"] = profile_steps
        a = pk["apply"]
        out["apply"] = {"launches": a["launches"], "ms_avg": a["ms"] / max(a["launches"], 1),
                        "bytes_algorithmic": a["bytes"] / max(a["launches"], 1),
                        "bytes_stored": a["bytes_stored"] / max(a["launches"], 1)}
    out["phi_after"] = s.get_field()  # after warm-up + timed + profiled steps (the same count for every form)
    if e2e:
        # same metric through the C ABI with host buffers: every step copies phi^n in from
        # pinned host memory and phi^{n+1} back out (each step one graph)
        shape = tuple(s.shape)
        pin_in = torch.empty(shape, dtype=torch.float64).pin_memory()
        pin_out = torch.empty(shape, dtype=torch.float64).pin_memory()
        a_in, a_out = pin_in.numpy(), pin_out.numpy()
        a_in[...] = s.get_field()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            dt = s.next_dt()
            s.step_host(a_in, dt, a_out)
            a_in, a_out = a_out, a_in
        torch.cuda.synchronize()
        el = max_over_ranks(world, time.perf_counter() - t0)
        out["e2e"] = {"value": steps * world / el, "unit": "steps/s", "h2d_bytes_per_step": int(a_in.nbytes),
                      "d2h_bytes_per_step": int(a_out.nbytes)}
    close()
    if golden:
        out["errors_vs_oracle"] = golden_errors(golden, prec, learned, **extra)
    return out


def run_batch32(steps: int, warmup: int, prec: int = 2):
    """The ensemble workload: 32 independent 256^2 noise runs (gamma_i drawn
    U(0.1, 0.35)), each on its own stream, stepped together by pfc_run_batch.
    Returns aggregate steps/s (all runs) and one run's steps/s alone."""
    import torch

    from paper_1703_01202_gb300 import inputs, pfc

    w = inputs.workload("batch32x256")

    def make(g, st):
        # a run whose step fails (GMRES(30) stagnates on the indefinite Jacobian of the
        # gamma > 0.2 liquid at dt = 10) retries that step with dt / 2
        params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec, dt_min=w["dt_min"],
                                    dt_max=w["dt_max"], eta=w["eta"], gmres_max_it=1200, dt_halvings=6)
        return pfc.Solver(w["shape"], w["h"], g, params, stream=st)

    solvers = [make(g, torch.cuda.Stream()) for g in w["gammas"]]
    for s, phi in zip(solvers, w["phis"]):
        s.set_field(phi)
    pfc.run_batch(solvers, warmup)
    torch.cuda.synchronize()
    c0 = pfc.launch_counts()
    t0 = time.perf_counter()
    recs = pfc.run_batch(solvers, steps)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    c1 = pfc.launch_counts()
    launches = c1["kernels"] - c0["kernels"]
    for s in solvers:
        s.close()
    one = make(w["gammas"][0], None)
    one.set_field(w["phis"][0])
    one.run(warmup)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    one.run(steps)
    torch.cuda.synchronize()
    el1 = time.perf_counter() - t1
    one.close()
    torch.cuda.empty_cache()
    member_steps = len(solvers) * steps
    return {"runs": len(solvers), "steps_per_run": steps, "steps_per_s": member_steps / el,
            "single_run_steps_per_s": steps / el1, "gpu_launches": launches,
            "kernels_per_member_step": launches / member_steps,
            "graph_launches": c1["graphs"] - c0["graphs"],
            "host_launch_calls_per_member_step": (c1["graphs"] - c0["graphs"]) / member_steps,
            "form": "one captured graph launch per 64 ensemble steps: every run's device-side time loop "
                    "(controller, retries, whole Newton steps) as a parallel branch",
            "newton_per_step": sum(r["newton_its"] for rr in recs for r in rr) / (len(recs) * steps),
            "gmres_per_step": sum(r["gmres_its"] for rr in recs for r in rr) / (len(recs) * steps),
            "dt_cuts": sum(r["dt_cuts"] for rr in recs for r in rr), "factor_prec": PREC_NAME[prec]}


def run_form(steps: int, warmup: int, prec: int, workload: str = WORKLOAD, **form):
    """Adaptive steps of a workload with one of the scheme's other forms (mobility, boundary),
    timed with CUDA events on the solver's stream (GMRES cycles as graphs in 2D)."""
    import torch

    s, close = make_solver(workload, prec, dt_halvings=6, **form)
    s.run(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    infos = s.run(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    close()
    return {"steps": steps, "steps_per_s": steps / (ms / 1e3),
            "newton_per_step": sum(i["newton_its"] for i in infos) / steps,
            "gmres_per_step": sum(i["gmres_its"] for i in infos) / steps,
            "dt_last": infos[-1]["dt"], "energy_last": infos[-1]["energy"], "factor_prec": PREC_NAME[prec]}


def guarded(fn, *a, **kw):
    """An extra workload's record, or the error that stopped it (the bench line still prints)."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported in the line, not hidden
        return {"failed": f"{type(e).__name__}: {e}"}


def strip(v: dict) -> dict:
    return {k: x for k, x in v.items() if k not in ("clocks", "e2e", "phi_after")}


def versus_f64(variants: dict) -> None:
    """max |phi - phi_F64 GPU| after the same warm-up, timed and profiled steps (the same dt sequence
    up to the controller's rounding), for every form of a grid that has a plain FP64 run."""
    import numpy as np

    for k, v in variants.items():  # the paper-tolerance forms against the FP64 run at the same tolerances
        base = "f64_paper_tol" if k.endswith("_paper_tol") else "f64"
        ref = variants.get(base, {}).get("phi_after")
        if k != base and ref is not None and v.get("phi_after") is not None:
            v["max_abs_phi_vs_f64_gpu"] = float(np.abs(v["phi_after"] - ref).max())


def precond_sweep(args):
    """The preconditioner and overlap sweep of Sec. 5 (Table 2's comparison) on the 1024^2 workload:
    AS (Eq. invM), left-RAS (Eq. ras) and right-RAS (Eq. ash) with 0-3 overlap cells per side, BF16
    factors, phi^n guess; steps `warmup`+1 .. `warmup`+`steps` timed (no bench line)."""
    import torch

    from paper_1703_01202_gb300 import build, inputs, pfc

    build.build()
    w = inputs.workload(WORKLOAD)
    rows = []
    cases = [(kind, name, ov, 0) for kind, name in ((pfc.PFC_AS, "as"), (pfc.PFC_LEFT_RAS, "left-ras"),
                                                   (pfc.PFC_RIGHT_RAS, "right-ras")) for ov in (0, 1, 2, 3)]
    cases += [(pfc.PFC_LEFT_RAS, "left-ras", 1, r) for r in (1, 3, 8)]  # factors kept across steps
    for kind, name, ov, reuse in cases:
        params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=ov, factor_prec=pfc.PFC_BF16,
                                    ras_kind=kind, dt_min=w["dt_min"], dt_max=w["dt_max"], eta=w["eta"],
                                    dt_halvings=4, reuse_factor=reuse)
        s = pfc.Solver(w["shape"], w["h"], w["gamma"], params, stream=torch.cuda.Stream())
        s.set_field(w["phi"])
        row = {"kind": name, "overlap_per_side": ov, "reuse_factor": reuse}
        try:
            s.run(args.warmup)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            infos = s.run(args.steps)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            row.update({"ms_per_step": 1e3 * el / args.steps,
                        "newton_per_step": sum(i["newton_its"] for i in infos) / args.steps,
                        "gmres_per_step": sum(i["gmres_its"] for i in infos) / args.steps,
                        "dt_cuts": sum(i["dt_cuts"] for i in infos), "dt_last": infos[-1]["dt"],
                        "apply_variant": s.tuning()["apply_variant"]})
        except pfc.PfcError as e:
            row["failed"] = str(e)
        s.close()
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"precond_sweep": rows, "workload": WORKLOAD, "factor_prec": "bf16", "guess": "phi^n",
                      "steps": args.steps, "warmup": args.warmup}))


def kernel_loop(args):
    """Runs one kernel family `steps` times on the workload's initial field
    (each pfc_precond_apply factors and applies once; cnn: the guess network's
    forward pass), for ncu captures."""
    import torch

    from paper_1703_01202_gb300 import build, inputs, pfc

    build.build()
    w = inputs.workload(args.kernel_workload)
    if args.kernel_grid:  # the workload's recipe on another grid (3D: a case small enough for ncu)
        nd = len(w["shape"])
        w["shape"] = (args.kernel_grid,) * nd
        w["parts"] = (args.kernel_parts,) * nd
        w["phi"] = (inputs.bcc_seeds_3d(w["shape"], w["h"], nseeds=1, d0=5 * math.pi, seed=1003) if nd == 3
                    else inputs.hex_seeds_2d(w["shape"], w["h"], seed=1001))
    prec = {"all": 2, "f64": 0, "f32": 1, "bf16": 2, "bf16_learned": 2}[args.variant]
    params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec,
                                apply_variant=args.apply_variant)
    s = pfc.Solver(w["shape"], w["h"], w["gamma"], params)
    phi = torch.from_numpy(w["phi"]).cuda()
    r = torch.from_numpy(inputs.noise_field(w["shape"], 0.0, 1.0, 7)).cuda()
    net = None
    if args.kernel_loop == "cnn":  # the committed guess network's forward pass on the workload's features
        from paper_1703_01202_gb300 import learned

        net = pfc.GuessNet(w["shape"])
        net.set_params(learned.load()[0])
        feat = torch.stack([phi - phi.mean(), 0.01 * r, torch.full_like(phi, 1.0)])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        if net is not None:
            net.forward(feat)
        elif args.kernel_loop == "apply":
            s.precond_apply(phi, phi, 10.0, r)
        elif args.kernel_loop == "jvp":
            s.jvp(phi, phi, r, 10.0)
        else:
            s.residual(phi, phi, 10.0)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    print(json.dumps({"kernel_loop": args.kernel_loop, "variant": args.variant, "calls": args.steps,
                      "workload": args.kernel_workload,
                      "ms_per_call": [round(1e3 * t, 3) for t in times], "tuning": s.tuning()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--reference-steps", type=int, default=1,
                    help="reference arm: whole oracle time steps timed (at most --steps)")
    ap.add_argument("--reference-all-cores", action="store_true",
                    help="reference arm: also time one whole oracle step with one BLAS thread per host core")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=4,
                    help="steps after the timed region with per-kernel CUDA events (rooflines)")
    ap.add_argument("--variant", default="all",
                    choices=["all", "f64", "f32", "bf16", "bf16_learned", "bf16_learned_fastdots",
                             "bf16_learned_jvp32", "f64_paper_tol", "bf16_learned_paper_tol"],
                    help="run one form only (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 2048^2, 256^3, ensemble and other-form workloads")
    ap.add_argument("--no-golden", action="store_true", help="skip the error runs against the oracle trajectories")
    ap.add_argument("--extras", default="all",
                    help="comma list of the other workloads to run: " + ",".join(EXTRAS) + " (default all)")
    ap.add_argument("--no-graph", action="store_true",
                    help="profiling aid: host-driven steps (the same kernels; ncu cannot profile the kernel "
                         "nodes of graphs with conditional nodes)")
    ap.add_argument("--precond-sweep", action="store_true",
                    help="AS / left-RAS / right-RAS x overlap 0-3 on the workload (no bench line)")
    ap.add_argument("--kernel-loop", default=None, choices=["apply", "jvp", "residual", "cnn"],
                    help="profiling aid: run one kernel family repeatedly on a workload (no bench line)")
    ap.add_argument("--kernel-workload", default=WORKLOAD)
    ap.add_argument("--kernel-grid", type=int, default=0, help="--kernel-loop: cells per axis instead of the workload's")
    ap.add_argument("--kernel-parts", type=int, default=4, help="--kernel-loop with --kernel-grid: cores per axis")
    ap.add_argument("--apply-variant", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4, 5],
                    help="Schwarz apply kernel of every solver (-1: autotuned; ncu's serialised replay would "
                         "otherwise tune to another kernel than a plain run)")
    args = ap.parse_args()
    if args.no_graph:
        USE_GRAPH[0] = 0
    APPLY_VARIANT[0] = args.apply_variant
    if args.kernel_loop:
        kernel_loop(args)
        return
    if args.precond_sweep:
        precond_sweep(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world, rank, local = dist_setup(args)
    from paper_1703_01202_gb300 import build

    if rank == 0:
        build.build()
    barrier(world)
    peaks = measured_peaks()
    hbm = peaks["hbm_gbs"]
    golden = None if args.no_golden else "hex1024_s10"
    # (name, factor precision, learned guess, opt-in forms)
    forms = (("f64", 0, False, {}), ("f32", 1, False, {}), ("bf16", 2, False, {}), ("bf16_learned", 2, True, {}),
             ("bf16_learned_fastdots", 2, True, {"gmres_fast_dots": 1}),
             ("bf16_learned_jvp32", 2, True, {"jvp_fp32": 1}),
             ("f64_paper_tol", 0, False, PAPER_TOL), ("bf16_learned_paper_tol", 2, True, PAPER_TOL))
    variants = {}
    for name, prec, lg, extra in forms:
        if args.variant in ("all", name):
            paper = name.endswith("_paper_tol")  # the oracle trajectory was written at the tighter tolerances
            variants[name] = run_variant(WORKLOAD, prec, args.steps, args.warmup, world, local, learned=lg,
                                         profile_steps=0 if paper and args.variant == "all" else args.profile_steps,
                                         e2e=(name == HEADLINE or args.variant == name),
                                         golden=None if paper else golden, hbm=hbm, **extra)
            if paper:
                variants[name]["tolerances"] = dict(PAPER_TOL)
    versus_f64(variants)
    head_name = HEADLINE if HEADLINE in variants else args.variant
    head = variants[head_name]
    ap_ = head.get("apply", {})
    achieved = ap_["bytes_algorithmic"] / (ap_["ms_avg"] * 1e-3) / 1e9 if ap_.get("launches") else None
    traffic = TRAFFIC.get(("apply", 2, head["tuning"]["apply_variant"])) if head_name.startswith("bf16") else None
    line = {
        "metric": METRIC,
        "value": whole_job_rate(args.steps, world, head["ms_per_step"] * args.steps / 1e3),
        "unit": "steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64 residual / Newton / GMRES least squares / energy / mass / dt; f32 subdomain LU stored "
                  "bf16; f32 JVP; float-float Gram-Schmidt sweeps on a float-pair basis; guess network bf16 "
                  "with f32 accumulation" if head_name == HEADLINE else head_name),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [1024, 1024], "subdomains": [64, 64], "overlap_per_side": 1,
                   "form": head_name, "guess": "learned network (safeguarded by phi^n and the extrapolation)",
                   "timed_path": "every time step one CUDA graph launch (device-side Newton, GMRES and line-search "
                                 "control), no per-kernel events in the timed region",
                   "l2": "inputs larger than L2 (factors 0.4-0.6 GB per apply, Krylov basis 0.25 GB)",
                   "replicas": world},
        "roofline": {"bound": "hbm", "kernel": "Schwarz apply (left-RAS banded triangular solves, chunked records)",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm if achieved else None, "peak_source": peaks["source"],
                     "algorithmic_bytes_per_launch": ap_.get("bytes_algorithmic"),
                     "stored_bytes_per_launch": ap_.get("bytes_stored"),
                     "traffic": traffic,
                     "traffic_over_algorithmic": traffic / ap_["bytes_algorithmic"] if traffic and ap_ else None,
                     "tensor_pipe_frac": 0.0,
                     "timing": f"CUDA events around each apply on the solver's stream over {args.profile_steps} "
                               "profiled steps after the timed region"},
        "rooflines": head.get("kernels"),
        "peaks": {"hbm_gbs": hbm, "fp32_tflops": FP32_PEAK_TFLOPS, "fp64_tflops": FP64_PEAK_TFLOPS},
        "clocks": head["clocks"],
        "gpu_launches": head["gpu_launches"],
        "graph_launches": head["graph_launches"],
        "e2e": head.get("e2e"),
        "iterations": {"newton_per_step": head["newton_per_step"], "gmres_per_step": head["gmres_per_step"]},
        "errors_vs_oracle": head.get("errors_vs_oracle"),
        "variants": {k: strip(v) for k, v in variants.items()},
    }
    extras = set(EXTRAS) if args.extras == "all" else set(args.extras.split(","))
    if not args.no_extras and extras:
        # the other workloads, each on this rank's GPU
        work = {}
        if "hex2048" in extras:
            grid2048 = {}
            for name, prec, lg, st, form in (("f64", 0, False, 20, {}), ("f32", 1, False, 20, {}),
                                             ("bf16", 2, False, 20, {}), ("bf16_learned", 2, True, 20, {}),
                                             ("bf16_learned_jvp32", 2, True, 20, {"jvp_fp32": 1})):
                grid2048[name] = guarded(run_variant, "hex2048", prec, st, 3, world, local, learned=lg,
                                         profile_steps=2, golden=None if args.no_golden else "hex2048_s3", hbm=hbm,
                                         **form)
            versus_f64(grid2048)
            work["hex2048"] = {k: strip(v) for k, v in grid2048.items()}
        if "bcc256" in extras:
            bcc = {}
            for name, prec, form in (("f64", 0, {}), ("f32", 1, {}), ("bf16", 2, {}),
                                     ("bf16_jvp32", 2, {"jvp_fp32": 1})):
                bcc[name] = guarded(run_variant, "bcc256", prec, 5, 1, world, local, profile_steps=1,
                                    golden=None if args.no_golden else "bcc64_s50", hbm=hbm, **form)
                if isinstance(bcc[name], dict) and "errors_vs_oracle" in bcc[name]:
                    bcc[name]["errors_vs_oracle"]["grid"] = "64^3 (the oracle trajectory's grid)"
            work["bcc256"] = {k: strip(v) for k, v in bcc.items()}
        if "batch32x256" in extras:
            work["batch32x256_bf16"] = guarded(run_batch32, max(2, args.steps // 2), 2)
        if "forms" in extras:
            work["hex1024_mobility_f32"] = guarded(run_form, max(4, args.steps // 4), 3, 1, mobility=1)
            work["hex1024_neumann_bf16"] = guarded(run_form, max(4, args.steps // 4), 3, 2, boundary=1)
            work["crack4096x1024_bf16"] = guarded(run_form, max(4, args.steps // 4), 3, 2,
                                                  workload="crack4096x1024")
        line["workloads"] = work
    if rank == 0 and not args.no_cpu_baseline:
        r = oracle_whole_step(1)
        line["cpu_baseline"] = {"value": 1.0 / r["seconds"], "unit": "steps/s", "cores": 1, "kind": "oracle",
                                "sample": oracle_text(r)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
