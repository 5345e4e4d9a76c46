"""Benchmark: PFC time steps per second on the 1024^2 crystal-growth workload
(3 hexagonal seeds, gamma = 0.25, h = pi/4, adaptive dt in [1e-2, 10],
eta = 5000, left-RAS on 64 x 64 cores with one overlap cell per side).

One bench step = one full time step of the scheme (Newton + GMRES + RAS,
energy, mass, adaptive dt) through the C ABI.  Variants: plain FP64 NKS and
the mixed path (FP32 / BF16 subdomain factors).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: the time stepper is not sharded across GPUs here; with N > 1 each
rank runs an independent replica (weak scaling) and `value` sums the replicas'
steps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
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
EXTRA_3D_STEPS = 2
METRIC = "PFC time steps/s (1024^2 2D crystal growth, adaptive dt)"


# DRAM bytes (read + write) of one 2D Schwarz apply launch on this workload from one ncu capture
# (profiles/ras_apply2d_hex1024_bf16.md, profiles/ras_apply2d_chunked_hex1024_bf16.md), keyed by
# (factor precision, apply kernel); a kernel not captured since its last change reports null.
APPLY_TRAFFIC = {(2, 4): 456.238592e6 + 3.252992e6, (2, 5): 540.646400e6 + 3.399424e6}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


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


# Per-step iteration counts of the FP64 path on this workload at the controller's dt (measured on a
# GB300 with exact block LU, the oracle's preconditioner): the oracle sample below is scaled by them
# when the bench has not measured them itself.
ORACLE_NEWTON_PER_STEP = 4.0
ORACLE_GMRES_PER_STEP = 146.0


def oracle_sample(newton: float, gmres: float, blocks_sampled: int = 512) -> dict:
    """Times the CPU oracle (one host thread) on a bounded sample of one time step
    of the workload at dt = dt_max and scales it to seconds per step:
      newton * (Jacobian assembly + 2 residuals) + Schwarz setup
      + gmres * (Schwarz apply + CSR matvec + Gram-Schmidt against 15 vectors).
    The Schwarz setup and apply are timed on the first `blocks_sampled` of the
    equal-size blocks and scaled by the block count."""
    code = f"""
import json, sys, time
import numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs
w = inputs.workload({WORKLOAD!r})
phi, h, g, dt = w["phi"], w["h"], w["gamma"], w["dt_max"]
t0 = time.perf_counter()
c = time.perf_counter(); F = O.residual(phi, phi, dt, h, g); t_res = time.perf_counter() - c
c = time.perf_counter(); J = O.assemble_jacobian(phi, phi, dt, h, g); t_jac = time.perf_counter() - c
blocks = O.decompose(phi.shape, w["parts"], 1)
sub = blocks[:{blocks_sampled}]
scale = len(blocks) / len(sub)
c = time.perf_counter(); pre = O.Schwarz(J, sub, "left-ras", "lu"); t_sch = (time.perf_counter() - c) * scale
c = time.perf_counter()
for _ in range(3):
    pre.apply(F)
t_app = (time.perf_counter() - c) / 3 * scale
v = F.ravel()
c = time.perf_counter()
for _ in range(3):
    J @ v
t_mv = (time.perf_counter() - c) / 3
rng = np.random.default_rng(0)
V = rng.standard_normal((15, v.size))
c = time.perf_counter()
x = v.copy()
for i in range(15):
    x -= (V[i] @ x) * V[i]
nrm = np.linalg.norm(x)
t_orth = time.perf_counter() - c
step = {newton!r} * (t_jac + 2 * t_res) + t_sch + {gmres!r} * (t_app + t_mv + t_orth)
print(json.dumps({{"seconds_per_step": step, "sample_seconds": time.perf_counter() - t0,
                  "parts": {{"residual": t_res, "jacobian": t_jac, "schwarz_setup": t_sch, "apply": t_app,
                            "matvec": t_mv, "gram_schmidt15": t_orth}}}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if res.returncode != 0:
        raise RuntimeError("oracle sample failed: " + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def oracle_sample_text(r: dict, newton: float, gmres: float) -> str:
    return (f"{WORKLOAD} step at dt = dt_max, FP64 oracle on 1 host thread: residual, Jacobian, Schwarz setup "
            f"and apply on 512 of 4096 blocks (scaled), matvec and 15-vector Gram-Schmidt timed "
            f"({r['sample_seconds']:.1f} s of CPU work), scaled by {newton:g} Newton and {gmres:g} GMRES "
            f"iterations per step")


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


def run_variant(prec: int, steps: int, warmup: int, world: int, local: int, measure_e2e: bool,
                apply_variant: int = -1, learned: bool = False, use_graph: int = 1):
    import numpy as np
    import torch

    from paper_1703_01202_gb300 import inputs, pfc
    from paper_1703_01202_gb300 import learned as lrn

    w = inputs.workload(WORKLOAD)
    params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec, dt_min=w["dt_min"],
                                dt_max=w["dt_max"], eta=w["eta"], apply_variant=apply_variant,
                                guess=pfc.PFC_GUESS_LEARNED if learned else pfc.PFC_GUESS_PREV, use_graph=use_graph)
    # a stream of its own: GMRES cycles run as captured graphs whenever per-apply timing is off
    s = pfc.Solver(w["shape"], w["h"], w["gamma"], params, stream=torch.cuda.Stream())
    net = None
    if learned:  # the committed network, trained on 512^2 trajectories of this workload's distribution
        theta, s_out = lrn.load()
        net = pfc.GuessNet(w["shape"])
        net.set_params(theta)
        pfc.set_guess_net(s, net, s_out)
    s.set_field(w["phi"])
    s.run(warmup)
    tuning = s.tuning()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    s.profile(True)
    k0 = s.profile_read()["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    infos = s.run(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ck = clocks.stop()
    prof = s.profile_read()
    s.profile(False)
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(world, ms)
    out = {
        "ms_per_step": ms / steps,
        "steps_per_s": steps / (ms / 1e3),
        "newton_per_step": sum(i["newton_its"] for i in infos) / steps,
        "gmres_per_step": sum(i["gmres_its"] for i in infos) / steps,
        "learned_guess_used": sum(1 for i in infos if i["guess_used"] == pfc.PFC_GUESS_LEARNED),
        "dt_last": infos[-1]["dt"],
        "energy_last": infos[-1]["energy"],
        "apply_launches": prof["apply_launches"],
        "apply_ms_avg": prof["apply_ms"] / max(prof["apply_launches"], 1),
        "apply_bytes": prof["apply_bytes"],
        "gpu_launches": prof["kernel_launches"] - k0,
        "clocks": ck,
        "tuning": tuning,
    }
    if measure_e2e:
        # same metric through the C ABI with host buffers: every step copies phi^n in
        # from pinned host memory and phi^{n+1} back out
        pin_in = torch.empty(w["shape"], dtype=torch.float64).pin_memory()
        pin_out = torch.empty(w["shape"], dtype=torch.float64).pin_memory()
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
    s.close()
    del s
    if net is not None:
        net.close()
    torch.cuda.empty_cache()
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
    k0 = solvers[0].profile_read()["kernel_launches"]
    t0 = time.perf_counter()
    recs = pfc.run_batch(solvers, steps)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    launches = solvers[0].profile_read()["kernel_launches"] - k0
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
    return {"runs": len(solvers), "steps_per_run": steps, "steps_per_s": len(solvers) * steps / el,
            "single_run_steps_per_s": steps / el1, "gpu_launches": launches,
            "newton_per_step": sum(r["newton_its"] for rr in recs for r in rr) / (len(recs) * steps),
            "gmres_per_step": sum(r["gmres_its"] for rr in recs for r in rr) / (len(recs) * steps),
            "dt_cuts": sum(r["dt_cuts"] for rr in recs for r in rr),
            "factor_prec": {0: "f64", 1: "f32", 2: "bf16"}[prec]}


def run_bcc256(steps: int, warmup: int, prec: int):
    """The 3D workload: 256^3 BCC growth, 7 x 7 x 7 uneven cores, ILU(0) blocks."""
    import torch

    from paper_1703_01202_gb300 import inputs, pfc

    w = inputs.workload("bcc256")
    params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec, dt_min=w["dt_min"],
                                dt_max=w["dt_max"], eta=w["eta"])
    s = pfc.Solver(w["shape"], w["h"], w["gamma"], params)
    s.set_field(w["phi"])
    s.run(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    infos = s.run(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    del s
    torch.cuda.empty_cache()
    return {"steps": steps, "steps_per_s": steps / (ms / 1e3),
            "newton_per_step": sum(i["newton_its"] for i in infos) / steps,
            "gmres_per_step": sum(i["gmres_its"] for i in infos) / steps,
            "dt_last": infos[-1]["dt"], "factor_prec": {0: "f64", 1: "f32", 2: "bf16"}[prec]}


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


def guarded(fn, *a):
    """An extra workload's record, or the error that stopped it (the bench line still prints)."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported in the line, not hidden
        return {"failed": f"{type(e).__name__}: {e}"}


def run_mobility(steps: int, warmup: int, prec: int = 1):
    """The 1024^2 workload with variable mobility M = 1 - phi^2 (the paper's Test B (c)); phi^n
    guess, GMRES cycles as graphs, FP64 JVP (the mobility form's).  F32 factors: the mobility
    blocks are worse conditioned at dt = 10, and BF16 factors let GMRES(30) stall there."""
    out = run_form(steps, warmup, prec, mobility=1)
    out["mobility"] = "1 - phi^2"
    return out


def run_neumann(steps: int, warmup: int, prec: int = 2):
    """The 1024^2 workload between Neumann-type walls (Sec. 2): mirror-image stencils, wall-clipped
    subdomains with folded block matrices (factored by the generic band LU), phi^n guess, GMRES
    cycles as graphs, float-float JVP."""
    out = run_form(steps, warmup, prec, boundary=1)
    out["boundary"] = "neumann"
    return out


def run_crack(steps: int, warmup: int, prec: int = 1):
    """Test C's crack-propagation workload: 4096 x 1024 cells of a stretched crystal with a liquid
    notch, gamma = 1, dt in [1, 5], eta = 100; phi^n guess, GMRES cycles as graphs."""
    out = run_form(steps, warmup, prec, workload="crack4096x1024")
    out["workload"] = "crack4096x1024"
    return out


def run_form(steps: int, warmup: int, prec: int, workload: str = WORKLOAD, **form):
    """Adaptive steps of a workload (by default the 1024^2 one) with one of the scheme's other
    forms (mobility, boundary), timed with CUDA events on the solver's stream."""
    import torch

    from paper_1703_01202_gb300 import inputs, pfc

    w = inputs.workload(workload)
    params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec, dt_min=w["dt_min"],
                                dt_max=w["dt_max"], eta=w["eta"], dt_halvings=6, **form)
    s = pfc.Solver(w["shape"], w["h"], w["gamma"], params, stream=torch.cuda.Stream())
    s.set_field(w["phi"])
    s.run(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    infos = s.run(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    return {"steps": steps, "steps_per_s": steps / (ms / 1e3),
            "newton_per_step": sum(i["newton_its"] for i in infos) / steps,
            "gmres_per_step": sum(i["gmres_its"] for i in infos) / steps,
            "dt_last": infos[-1]["dt"], "energy_last": infos[-1]["energy"],
            "factor_prec": {0: "f64", 1: "f32", 2: "bf16"}[prec]}


def kernel_loop(args):
    """Runs one kernel family `steps` times on the workload's initial field
    (each pfc_precond_apply factors and applies once), for ncu captures."""
    import torch

    from paper_1703_01202_gb300 import build, inputs, pfc

    build.build()
    w = inputs.workload(WORKLOAD)
    prec = {"all": 2, "f64": 0, "f32": 1, "bf16": 2, "bf16_learned": 2}[args.variant]
    params = pfc.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec,
                                apply_variant=args.apply_variant)
    s = pfc.Solver(w["shape"], w["h"], w["gamma"], params)
    phi = torch.from_numpy(w["phi"]).cuda()
    r = torch.from_numpy(inputs.noise_field(w["shape"], 0.0, 1.0, 7)).cuda()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        if args.kernel_loop == "apply":
            s.precond_apply(phi, phi, 10.0, r)
        elif args.kernel_loop == "jvp":
            s.jvp(phi, phi, r, 10.0)
        else:
            s.residual(phi, phi, 10.0)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    print(json.dumps({"kernel_loop": args.kernel_loop, "variant": args.variant, "calls": args.steps,
                      "ms_per_call": [round(1e3 * t, 3) for t in times], "tuning": s.tuning()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", default="all", choices=["all", "f64", "f32", "bf16", "bf16_learned"],
                    help="run one factor-precision variant only (profiling runs)")
    ap.add_argument("--no-graph", action="store_true",
                    help="profiling aid: run GMRES cycles from the host loop (every launch visible to ncu)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ensemble (32 x 256^2) and 3D (256^3) workloads")
    ap.add_argument("--apply-variant", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4, 5],
                    help="2D Schwarz apply kernel (-1: autotuned at the first factorisation)")
    ap.add_argument("--precond-sweep", action="store_true",
                    help="AS / left-RAS / right-RAS x overlap 0-3 on the workload (no bench line)")
    ap.add_argument("--kernel-loop", default=None, choices=["apply", "jvp", "residual"],
                    help="profiling aid: run one kernel family repeatedly on the workload (no bench line)")
    args = ap.parse_args()
    if args.kernel_loop:
        kernel_loop(args)
        return
    if args.precond_sweep:
        precond_sweep(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return
        nw, gm = ORACLE_NEWTON_PER_STEP, ORACLE_GMRES_PER_STEP
        for _ in range(min(args.warmup, 1)):
            oracle_sample(nw, gm)
        samples = [oracle_sample(nw, gm) for _ in range(max(1, args.steps))]
        sec = statistics.median(r["seconds_per_step"] for r in samples)
        v = 1.0 / sec
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": len(samples), "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": oracle_sample_text(samples[0], nw, gm) + "; median over steps"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    world, rank, local = dist_setup(args)
    from paper_1703_01202_gb300 import build

    if rank == 0:
        build.build()
    barrier(world)
    variants = {}
    for name, prec, lg in (("f64", 0, False), ("f32", 1, False), ("bf16", 2, False), ("bf16_learned", 2, True)):
        if args.variant in ("all", name):
            variants[name] = run_variant(prec, args.steps, args.warmup, world, local,
                                         measure_e2e=(name == "bf16_learned" or args.variant != "all"),
                                         apply_variant=args.apply_variant, learned=lg,
                                         use_graph=0 if args.no_graph else 1)
    head = variants["bf16_learned" if "bf16_learned" in variants else args.variant]
    peak, peak_kind = measured_peaks()
    achieved = head["apply_bytes"] / (head["apply_ms_avg"] * 1e-3) / 1e9
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
        "dtype": "f64 (subdomain factors stored bf16 and applied in f32; guess network bf16/f32)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [1024, 1024], "subdomains": [64, 64], "overlap_per_side": 1,
                   "guess": "learned network (safeguarded by phi^n and the extrapolation)",
                   "l2": "inputs larger than L2 (factors 0.45-1.7 GB per apply)", "replicas": world},
        "roofline": {"bound": "hbm", "kernel": "ras_apply (left-RAS banded triangular solves)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind,
                     "traffic": APPLY_TRAFFIC.get((2, head["tuning"]["apply_variant"]))},
        "clocks": head["clocks"],
        "gpu_launches": head["gpu_launches"],
        "e2e": head["e2e"],
        "iterations": {"newton_per_step": head["newton_per_step"], "gmres_per_step": head["gmres_per_step"]},
        "variants": {k: {kk: vv for kk, vv in v.items() if kk not in ("clocks", "e2e")} for k, v in variants.items()},
    }
    if not args.no_extras:
        # the other workloads, each on this rank's GPU: the 32-run 256^2 ensemble (pfc_run_batch),
        # the 1024^2 one with variable mobility and between Neumann walls, the 4096 x 1024 crack
        # case and the 256^3 BCC case (F32 and BF16 ILU(0) factors)
        line["workloads"] = {
            "batch32x256_bf16": guarded(run_batch32, max(2, args.steps // 2), 2),
            "hex1024_mobility_f32": guarded(run_mobility, max(4, args.steps // 4), 3),
            "hex1024_neumann_bf16": guarded(run_neumann, max(4, args.steps // 4), 3),
            "crack4096x1024_bf16": guarded(run_crack, max(4, args.steps // 4), 3, 2),
            "bcc256_f32": guarded(run_bcc256, EXTRA_3D_STEPS, 1, 1),
            "bcc256_bf16": guarded(run_bcc256, EXTRA_3D_STEPS, 1, 2),
        }
    if rank == 0 and not args.no_cpu_baseline:
        f64 = variants.get("f64")
        nw = f64["newton_per_step"] if f64 else ORACLE_NEWTON_PER_STEP
        gm = f64["gmres_per_step"] if f64 else ORACLE_GMRES_PER_STEP
        r = oracle_sample(nw, gm)
        line["cpu_baseline"] = {"value": 1.0 / r["seconds_per_step"], "unit": "steps/s", "cores": 1,
                                "kind": "oracle", "sample": oracle_sample_text(r, nw, gm)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
