#!/usr/bin/env python
"""Throughput of the free-boundary ETD2 step on one GB300.

Workload (default star3d): 3D single species on a 128^3 node grid over
[-6,6]^3, u_t = Lap u + u(1-u), beta = 1, mu = 1, star-shaped initial domain
r0 = 1.5(1 + 0.2 Y), dt = 5e-3, Krylov tolerance 1e-7 (FP64) / 1e-5 (mixed),
m <= 40; synthetic seeded inputs (paper_2209_15095_gb300.inputs).

One step = levelset_advance + etd_init_domain + etd_step (every row of the
hot path: extension, Stefan speed, HJ-WENO5/TVD-RK3 advection,
reinitialisation every 5 steps, classification and ghost metadata, ETD2 via
the adaptive-Krylov phi-combination).  Metric: Mcell-updates/s = computational
points / step time.  Both precisions are measured; `value` is the FP64 path,
`mixed` the FP32-mixed path with its error against the FP64 path.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on
the library's stream; the L2 is flushed (a 512 MiB write) between timed
steps, outside the events.  `e2e` repeats the step through the same C-ABI
calls with the fields copied from pinned host memory before and back after
each step, inside the timed region.

--impl reference times the FP64 CPU oracle (oracle/) on the host cores on a
bounded sample of the same workload.  Under torchrun (N > 1) every rank runs
an independent replica (the method has no multi-GPU path in this build).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-updates/s per ETD step"
UNIT = "Mcell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="star3d")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-etd2rk", action="store_true", help="skip every leg of the other integrators")
    ap.add_argument("--rk-schemes", default="etd2rk,etd3rk,etd4rk,etd3",
                    help="comma-separated integrators other than ETD2 timed on the same step (FP64)")
    ap.add_argument("--no-poisson", action="store_true")
    ap.add_argument("--mixed-tols", default="1.1e-6",
                    help="extra FP32-mixed legs at these Krylov tolerances (comma-separated): speed-up and error in u")
    ap.add_argument("--clocks", default="on", choices=["on", "off"])
    ap.add_argument("--no-stress", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint_ball3d gradient leg")
    ap.add_argument("--adjoint-steps", type=int, default=100, help="ETD2 steps of the adjoint leg's trajectory")
    ap.add_argument("--stress-steps", type=int, default=3)
    ap.add_argument("--stress-n", type=int, default=512, help="grid nodes per axis of the stress ball")
    ap.add_argument("--stress-precision", default="both", choices=["both", "fp64", "mixed"])
    ap.add_argument("--stress-only", action="store_true",
                    help="run only the stress shape and print its results (a profiling aid, not the bench line)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_ranks(t_local, cells_local, device):
    """Whole-job figures of N independent replicas: the timed seconds are the
    maximum over the ranks (the slowest replica sets the job's time) and the
    computational-point updates their sum; returns (cells, seconds).  With
    one process, the local figures."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(cells_local), float(t_local)
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cc = torch.tensor([float(cells_local)], dtype=torch.float64, device=device)
    dist.all_reduce(cc, op=dist.ReduceOp.SUM)
    return cc.item(), tt.item()


def sync_ranks(device):
    """Device synchronisation, then a barrier across the replicas (if any):
    brackets the timed steps so that every rank starts and ends them
    together."""
    import torch
    import torch.distributed as dist

    torch.cuda.synchronize(device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def workload(name):
    from paper_2209_15095_gb300 import inputs

    return getattr(inputs, name)()


# --------------------------------------------------------------- reference arm
ORACLE_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
from paper_2209_15095_gb300 import inputs
from oracle.grid import Grid
from oracle.freeboundary import FreeBoundary, Species
w = getattr(inputs, %(name)r)()
g = Grid(w.n, w.lo, w.hi)
sp = [Species(w.phi0[s], w.u0[s], w.beta[s], w.mu[s]) for s in range(len(w.phi0))]
fb = FreeBoundary(g, sp, w.reaction, w.rparams, w.tol, w.m_max, reinit_every=getattr(w, "reinit_every", 5),
                  reinit_at_start=False)
budget, maxsteps, warm = %(budget)f, %(steps)d, %(warm)d
for _ in range(warm):
    fb.step(w.dt)
# parallel replicas start their timed steps together (bounded wait)
sync_dir, nrep, rid = %(sync_dir)r, %(nrep)d, %(rid)d
if sync_dir:
    import os
    open(os.path.join(sync_dir, "ready_%%d" %% rid), "w").close()
    t_wait = time.time()
    while len(os.listdir(sync_dir)) < nrep and time.time() - t_wait < 300.0:
        time.sleep(0.05)
cells, t_tot, n = 0, 0.0, 0
while n < maxsteps and t_tot < budget:
    t0 = time.perf_counter()
    fb.step(w.dt)
    t_tot += time.perf_counter() - t0
    cells += sum(int(s.comp.sum()) for s in fb.sp)
    n += 1
print(json.dumps({"cells": cells, "seconds": t_tot, "steps": n, "warm": warm}))
"""


def oracle_sample(name, budget, steps, warm, replicas=1):
    """The FP64 oracle (single-threaded numpy) on a bounded sample of the
    workload, in `replicas` independent processes that start their timed
    steps together (one per host core for the all-core figure).  Returns the
    per-process results and the aggregate rate (cells / longest timed span)."""
    import tempfile

    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    sync_dir = tempfile.mkdtemp(prefix="oracle_sync_") if replicas > 1 else ""
    procs = []
    for rid in range(replicas):
        code = ORACLE_SAMPLE % {"root": ROOT, "name": name, "budget": budget, "steps": steps, "warm": warm,
                                "sync_dir": sync_dir, "nrep": replicas, "rid": rid}
        procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True, env=env))
    res = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    if sync_dir:
        import shutil

        shutil.rmtree(sync_dir, ignore_errors=True)
    cells = sum(r["cells"] for r in res)
    secs = max(r["seconds"] for r in res)
    return {"cells": cells, "seconds": secs, "steps": sum(r["steps"] for r in res), "warm": res[0]["warm"],
            "replicas": replicas, "per_replica_steps": [r["steps"] for r in res]}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    warm = min(args.warmup, 1)
    cores = host_cores()
    res = oracle_sample(args.workload, budget=120.0, steps=max(1, args.steps), warm=warm, replicas=cores)
    value = res["cells"] / res["seconds"] / 1e6
    sample = ("%d independent replicas of the FP64 oracle (single-threaded numpy), one per host core, each "
              "running free-boundary steps of %s (level set + domain + ETD2) after %d untimed step(s) from the "
              "initial data without the start-up reinitialisation, timed steps capped at 120 s per replica; "
              "%d steps in all; value = all replicas' cells / the longest timed span"
              % (cores, args.workload, res["warm"], res["steps"]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": min(res["per_replica_steps"]), "warmup": res["warm"],
        "ms_per_step": 1e3 * res["seconds"] / max(1, min(res["per_replica_steps"])),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, enabled=True):
        self.proc = None
        self.index = index
        self.path = None
        if not enabled:
            return
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed regions are tens of milliseconds: start them only once the
        # sampler is producing rows
        t0 = time.time()
        while time.time() - t0 < 15.0:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        top = max(r[0] for r in rows)
        load = [r[0] for r in rows if r[0] >= 0.5 * top] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": rows[0][1], "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2209_15095_gb300 import build

    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    from paper_2209_15095_gb300 import etd

    w = workload(args.workload)
    nsp = len(w.phi0)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    results = {}

    def make_ctx(precision, scheme="etd2", tol=None):
        with torch.cuda.stream(stream):
            if tol is None:
                tol = w.tol if precision == "fp64" else getattr(w, "tol_mixed", w.tol)
            return etd.Context(w.n, w.lo, w.hi, nspecies=nsp, precision=precision, tol=tol, m_max=w.m_max,
                               reaction=w.reaction, rparams=w.rparams, mu=w.mu, beta=w.beta, device=dev,
                               scheme=scheme)

    def initial_state(ctx):
        phis = [torch.tensor(p, dtype=torch.float64, device=dev) for p in w.phi0]
        us = [torch.tensor(np.where(w.phi0[s] < 0, w.u0[s], 0.0), dtype=torch.float64, device=dev)
              for s in range(nsp)]
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            for s in range(nsp):
                ctx.levelset_prepare(phis[s], getattr(w, "reinit_at_start", False))
                ctx.init_domain(s, phis[s])
        return phis, us

    def one_step(ctx, phis, us, k, ev=None):
        reinit = w.reinit_every > 0 and (k + 1) % w.reinit_every == 0
        if ev:
            ev[0].record(stream)
        for s in range(nsp):
            ctx.levelset_advance(s, phis[s], us[s], w.dt, reinit)
        if ev:
            ev[1].record(stream)
        for s in range(nsp):
            ctx.init_domain(s, phis[s])
        if ev:
            ev[2].record(stream)
        ctx.step(w.dt, us)
        if ev:
            ev[3].record(stream)

    def run(precision, scheme="etd2", tol=None):
        ctx = make_ctx(precision, scheme, tol)
        phis, us = initial_state(ctx)
        k = 0
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                one_step(ctx, phis, us, k)
                k += 1
            ctx.sync()
            sync_ranks(dev)
            times, parts, cells, iters, subs, ls_flops = [], [], 0, 0, 0, 0.0
            nre = 0
            for _ in range(args.steps):
                flush.zero_()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                nre += int(w.reinit_every > 0 and (k + 1) % w.reinit_every == 0)
                one_step(ctx, phis, us, k, ev)
                k += 1
                st = ctx.last_stats()  # synchronises; outside the events
                ls_flops += sum(levelset_flops(ctx.levelset_last_stats(), len(w.n)) for _ in range(nsp))
                times.append(ev[0].elapsed_time(ev[3]))
                parts.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
                cells += sum(s_["ncomp"] for s_ in st)
                iters += sum(s_["krylov_iters"] for s_ in st)
                subs += sum(s_["substeps"] for s_ in st)
        ctx.sync()
        sync_ranks(dev)
        return {"ctx": ctx, "phis": phis, "us": us, "times": times, "parts": parts, "cells": cells,
                "iters": iters, "substeps": subs, "k": k, "ls_flops": ls_flops, "reinit_steps": nre}

    if args.stress_only:
        if rank == 0:
            del flush
            torch.cuda.empty_cache()
            print(json.dumps({"stress": run_stress(etd, stream, dev, args.stress_steps, args.stress_n,
                                                   args.stress_precision)}))
        return
    clocks = ClockSampler(local, enabled=args.clocks == "on" and rank == 0)
    r64 = run("fp64")
    rmx = None if args.no_mixed else run("mixed")
    # the same mixed run at the FP64 run's Krylov tolerance: the error of the
    # FP32 arithmetic alone
    rmt = None if args.no_mixed or getattr(w, "tol_mixed", w.tol) == w.tol else run("mixed", tol=w.tol)
    rsw = [] if args.no_mixed else [(float(t), run("mixed", tol=float(t))) for t in args.mixed_tols.split(",") if t]
    rks = {} if args.no_etd2rk else {sc: run("fp64", sc) for sc in args.rk_schemes.split(",") if sc}
    pois = None if args.no_poisson or rank != 0 else run_poisson(etd, stream, dev)
    e2e = None if args.no_e2e else run_e2e(args, w, make_ctx, initial_state, one_step, stream, flush, dev)
    adj = {}
    if not args.no_adjoint and rank == 0:
        for prec in ("fp64", "mixed"):
            adj[prec] = run_adjoint(etd, dev, prec, args.adjoint_steps)
    stress = None
    if not args.no_stress and rank == 0:
        del flush
        torch.cuda.empty_cache()
        stress = run_stress(etd, stream, dev, args.stress_steps, args.stress_n, args.stress_precision)
    clk = clocks.stop()

    cells_all, t64 = aggregate_ranks(sum(r64["times"]) / 1e3, r64["cells"], dev)
    value = cells_all / t64 / 1e6
    if rank != 0:
        return
    nparts = np.array(r64["parts"])
    avg_parts = nparts.mean(axis=0)
    names = ["levelset_kernel", "init_domain_kernel", "phipm_kernel"]
    # key order: the contract's keys, then details, then (last, so that a
    # truncated log keeps them) the compact mixed-precision, stress and
    # adjoint summaries
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t64 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(w.n), "dt": w.dt, "krylov_tol": w.tol,
                   "m_max": w.m_max, "steps_from": args.warmup, "l2": "flushed (512 MiB write) between timed steps",
                   "parallelism": "replicas" if args.gpus > 1 else "single GPU"},
        "gpu_launches": args.steps * (2 * nsp + 1),
        "breakdown_ms": {n: float(v) for n, v in zip(names, avg_parts)},
        "krylov": {"iters_per_step": r64["iters"] / args.steps, "substeps_per_step": r64["substeps"] / args.steps,
                   "ncomp_mean": r64["cells"] / args.steps,
                   # point-iterations of the Krylov basis per second of Krylov launches
                   "cell_iters_per_s": (r64["cells"] / args.steps) * (r64["iters"] / args.steps)
                                       / (float(avg_parts[2]) / 1e3)},
        # the whole grid's nodes per second of the full step (n^N / t)
        "grid_nodes_per_s": math.prod(w.n) / (t64 / args.steps),
        "etd_only_ms_per_step": float(avg_parts[2]),
    }
    if e2e is not None:
        out["e2e"] = e2e
    out["roofline"] = roofline(r64, w, avg_parts, names)
    if clk is not None:
        out["clocks"] = clk
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    nevals = {"etd2rk": 2, "etd3rk": 3, "etd4rk": 4, "etd3": 1}
    for sc, rrk in rks.items():
        trk = sum(rrk["times"]) / 1e3
        out[sc] = {"value": rrk["cells"] / trk / 1e6, "ms_per_step": 1e3 * trk / args.steps, "dtype": "f64",
                   "note": "same step with the %s integrator (%d Krylov evaluation%s per step)"
                           % (sc.upper(), nevals.get(sc, 0), "" if nevals.get(sc, 0) == 1 else "s"),
                   "krylov_iters_per_step": rrk["iters"] / args.steps,
                   "substeps_per_step": rrk["substeps"] / args.steps,
                   "breakdown_ms": {n: float(v) for n, v in zip(names, np.array(rrk["parts"]).mean(axis=0))}}
    if pois is not None:
        out["poisson"] = pois
    if rmx is not None:
        out["mixed_breakdown_ms"] = {n: float(v) for n, v in zip(names, np.array(rmx["parts"]).mean(axis=0))}
    if rmt is not None:
        tmt = sum(rmt["times"]) / 1e3
        out["mixed_matched_tol"] = {
            "value": _r(rmt["cells"] / tmt / 1e6), "speedup_vs_fp64": _r(t64 / tmt),
            "max_rel_err_u_vs_fp64": _r(mixed_error(r64, rmt, nsp)), "krylov_tol": w.tol}
    if stress is not None:
        out["stress"] = stress
    if adj:
        out["adjoint"] = adj
    if rsw:
        out["mixed_tol_sweep"] = []
        for tol, rr in rsw:
            tt = sum(rr["times"]) / 1e3
            out["mixed_tol_sweep"].append({
                "krylov_tol": tol, "value": _r(rr["cells"] / tt / 1e6), "speedup_vs_fp64": _r(t64 / tt),
                "max_rel_err_u_vs_fp64": _r(mixed_error(r64, rr, nsp))})
    if rmx is not None:
        tmx = sum(rmx["times"]) / 1e3
        out["mixed"] = {"value": _r(rmx["cells"] / tmx / 1e6), "ms_per_step": _r(1e3 * tmx / args.steps),
                        "speedup_vs_fp64": _r(t64 / tmx), "max_rel_err_u_vs_fp64": _r(mixed_error(r64, rmx, nsp)),
                        "krylov_tol": getattr(w, "tol_mixed", w.tol), "dtype": "f32+f64"}
    print(json.dumps(out))


def _r(x, digits=4):
    """x rounded to `digits` significant digits (compact JSON)."""
    if x is None or x == 0 or not math.isfinite(x):
        return x
    return float("%.*g" % (digits, x))


def cpu_baseline(name):
    """The oracle on the host: one free-boundary step from the initial data,
    in one process per host core (all starting together), and the same step
    single-threaded in one process."""
    cores = host_cores()
    try:
        allc = oracle_sample(name, budget=25.0, steps=1, warm=0, replicas=cores)
        one = oracle_sample(name, budget=25.0, steps=1, warm=0, replicas=1)
    except Exception as e:  # reported, never silently replaced
        return {"error": str(e)[:300]}
    return {"value": allc["cells"] / allc["seconds"] / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "1 oracle free-boundary step of %s from its initial data (FP64 numpy, without the start-up "
                      "reinitialisation) in %d single-threaded processes, one per host core, started together; "
                      "value = their cells / the longest step time" % (name, cores),
            "single_core": {"value": one["cells"] / one["seconds"] / 1e6, "cores": 1}}


def mixed_error(r64, rmx, nsp):
    import numpy as np

    errs = []
    for s in range(nsp):
        a = r64["us"][s].cpu().numpy()
        b = rmx["us"][s].cpu().numpy()
        both = (r64["phis"][s].cpu().numpy() < 0) & (rmx["phis"][s].cpu().numpy() < 0)
        errs.append(float(np.max(np.abs(a - b)[both]) / max(np.max(np.abs(a)), 1e-300)))
    return max(errs)


# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA per clock x 2
# flops x 2.07 GHz (a measured FMA loop reaches 1.005 TFLOP/s on this GPU).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# levelset_kernel<3> on star3d from one ncu capture (command and figures in
# profiles/levelset_kernel_star3d.md), valid only for the kernel sources whose
# SHA-256 prefix is recorded here; any change to them reports null.
LS_TRAFFIC = {"sources": ("levelset.cu", "levelset.cuh", "common.cuh"), "sha256": "a1d876dc469ba6b0",
              "no_reinit": 22.07e6, "reinit": 22.66e6}


def levelset_traffic(reinit_fraction):
    import hashlib

    h = hashlib.sha256()
    for f in LS_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_2209_15095_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != LS_TRAFFIC["sha256"]:
        return None
    return (1.0 - reinit_fraction) * LS_TRAFFIC["no_reinit"] + reinit_fraction * LS_TRAFFIC["reinit"]


def levelset_flops(info, ndim):
    """Algorithmic FP64 flops of one level-set launch, counted from the
    formulation the kernel evaluates (add/mul/div/sqrt/min/max 1, fma 2):
    one Godunov/HJ-WENO5 node-stage costs 106 flops per axis (6 differences,
    the Jiang-Peng pair of one-sided derivatives with shared second
    differences and one shared division: 92, the Godunov selection: 4, the
    rest 4) plus 7 per node (square root, 1/h, the RK3 update); the Stefan
    speed 85 per tube node (two N-linear interpolations by axis-wise lerps).
    Advection: tube x 3 stages x substeps; reinitialisation: tube x 3 x
    ceil(12 sqrt N) stages.  The extension sweeps (2(N+1) flops per region
    node and sweep) and the work-set build are not counted (a conservative
    count)."""
    stage = 106 * ndim + 7
    k = math.ceil(12 * math.sqrt(ndim))
    f = info["tube"] * (3 * info["nsub"] * stage + 85)
    if info["reinit"]:
        f += info["reinit_tube"] * 3 * k * stage
    return float(f)


def roofline(r, w, avg_parts, names):
    """Dominant kernel: the largest share of the step.  The Krylov kernel is
    reported against HBM bandwidth with its algorithmic bytes; the level-set
    kernel, FP64-ALU bound, against the FP64 rate."""
    import numpy as np

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    dom = int(np.argmax(avg_parts))
    steps = len(r["times"])
    ncomp = r["cells"] / steps
    iters = r["iters"] / steps
    subs = r["substeps"] / steps
    bytes_step = krylov_bytes(ncomp, iters, subs, 8)
    t_phipm = avg_parts[2] / 1e3
    krylov = {"bound": "hbm", "kernel": names[2], "achieved": bytes_step / t_phipm / 1e9, "peak": hbm,
              "unit": "GB/s", "frac": bytes_step / t_phipm / 1e9 / hbm, "traffic": None,
              "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)",
              "algorithmic_bytes_per_launch": bytes_step}
    t_ls = avg_parts[0] / 1e3
    flops = r["ls_flops"] / steps
    ls = {"bound": "alu", "kernel": names[0], "achieved": flops / t_ls / 1e12, "peak": FP64_PEAK_TFLOPS,
          "unit": "TFLOP/s", "frac": flops / t_ls / 1e12 / FP64_PEAK_TFLOPS,
          "traffic": levelset_traffic(r["reinit_steps"] / steps) if w.name == "star3d" else None,
          "peak_source": "FP64 nominal: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (unit counts and clock); the measured FP64 FMA rate on this GB300 is 1.005 TFLOP/s",
          "algorithmic_flops_per_launch": flops}
    out = ls if dom == 0 else krylov
    out = dict(out)
    out["dominant_share"] = float(avg_parts[dom] / avg_parts.sum())
    out["dominant_kernel"] = names[dom]
    out["krylov_kernel"] = krylov if dom == 0 else None
    return out


def krylov_bytes(ncomp, iters, subs, s):
    """Algorithmic bytes of one Krylov launch: per point, every basis vector
    (read v_j, v_{j-1}, write v_{j+1}, read D_p and the index: 3s + 8 + 4
    with the diagonal in FP64, 3s + 4 + 4 in FP32), two matvecs with a vector
    add per substep (same count each), the combination (m + 2 vectors in T,
    y read and written in FP64) and the set-up (48 B)."""
    b = (8.0 if s == 8 else 4.0) + 4.0
    return ncomp * (iters * (3 * s + b) + subs * 2 * (3 * s + b) + (iters + 2 * subs) * s + subs * 16 + 48)


def run_adjoint(etd, dev, precision, nsteps=100, every=10, nquad=8):
    """Gradient leg on adjoint_ball3d (128^3 on [-6, 6]^3, fixed ball r = 4,
    beta = 1 + 0.3 g with g a seeded Gaussian random field, alpha u (1 - u/K)):
    the loss L = 1/2 |u(T) - u*|^2 after `nsteps` ETD2 steps of dt = 1e-2, u*
    from alpha = 1.1 and 1.05 beta; gradients with respect to u_0, beta and
    alpha through the autograd wrapper, checkpoints every `every` steps.
    Timed with CUDA events: the forward trajectory, the backward pass
    (segment recomputation and the adjoint steps) and one adjoint step alone.
    Checked against central finite differences of an FP64 forward at Krylov
    tolerance 1e-12 on five sampled entries (two of u_0, two of beta, alpha)."""
    import numpy as np
    import torch

    from paper_2209_15095_gb300 import inputs
    from paper_2209_15095_gb300.autograd import trajectory

    w = inputs.adjoint_ball3d()
    alpha, K = w.rparams

    def mk(prec, tol):
        return etd.Context(w.n, w.lo, w.hi, nspecies=1, precision=prec, tol=tol, m_max=w.m_max,
                           reaction="logistic_ak", rparams=(alpha, K), adjoint=True, device=dev)

    ctx = mk(precision, w.tol)
    ref = mk("fp64", 1e-12)
    f64 = dict(dtype=torch.float64, device=dev)
    phi = torch.tensor(w.phi0[0], **f64)
    beta = torch.tensor(w.beta[0], **f64)
    u0 = torch.tensor(w.u0[0], **f64)
    with torch.no_grad():
        ustar = trajectory(ref, u0, beta * w.beta_target_scale, torch.tensor([w.rparams_target[0]], **f64), phi,
                           w.dt, nsteps, K=K, checkpoint_every=every, nquad=nquad)

    def once(n):
        du0 = u0.clone().requires_grad_(True)
        db = beta.clone().requires_grad_(True)
        da = torch.tensor([alpha], **f64).requires_grad_(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize(dev)
        ev[0].record()
        uT = trajectory(ctx, du0, db, da, phi, w.dt, n, K=K, checkpoint_every=every, nquad=nquad)
        ev[1].record()
        loss = 0.5 * ((uT - ustar) ** 2).sum()
        loss.backward()
        ev[2].record()
        ev[2].synchronize()
        return ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), du0.grad, db.grad, da.grad, loss.item()

    once(3)  # warm-up
    tf, tb, gu, gb, ga, L = once(nsteps)
    # one adjoint step alone (5 calls)
    lam = (u0 - ustar).contiguous()
    acc, gbz, gaz = torch.zeros_like(u0), torch.zeros_like(u0), torch.zeros(1, **f64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(5):
        ctx.adjoint_step(0, w.dt, u0, u0, False, lam, acc, gbz, gaz, nquad)
    e1.record()
    e1.synchronize()
    t_adj = e0.elapsed_time(e1) / 5
    ncomp = ctx.read_domain(0, arrays=False)["ncomp"]

    def loss_fd(u0_, beta_, alpha_):
        with torch.no_grad():
            out = trajectory(ref, u0_, beta_, torch.tensor([alpha_], **f64), phi, w.dt, nsteps, K=K,
                             checkpoint_every=every, nquad=nquad)
            return 0.5 * float(((out - ustar) ** 2).sum())

    # sampled entries: computational nodes near two fixed points inside the ball
    x = inputs.grid_coords(w.n, w.lo, w.hi)
    flat = []
    for c in ((0.5, -0.7, 1.1), (-1.3, 0.4, -0.6)):
        d2 = sum((x[i] - c[i]) ** 2 for i in range(3))
        flat.append(int(np.argmin(d2)))
    errs = []
    eps = 1e-6
    for kind, arr, grad in (("u0", u0, gu), ("beta", beta, gb)):
        for fl in flat:
            p_, m_ = arr.clone().view(-1), arr.clone().view(-1)
            p_[fl] += eps
            m_[fl] -= eps
            if kind == "u0":
                fd = (loss_fd(p_.view(w.n), beta, alpha) - loss_fd(m_.view(w.n), beta, alpha)) / (2 * eps)
            else:
                fd = (loss_fd(u0, p_.view(w.n), alpha) - loss_fd(u0, m_.view(w.n), alpha)) / (2 * eps)
            errs.append(abs(grad.view(-1)[fl].item() - fd) / abs(fd))
    fd = (loss_fd(u0, beta, alpha + eps) - loss_fd(u0, beta, alpha - eps)) / (2 * eps)
    errs.append(abs(ga.item() - fd) / abs(fd))
    return {"workload": "adjoint_ball3d", "grid": list(w.n), "ncomp": ncomp, "steps": nsteps,
            "checkpoint_every": every, "nquad": nquad, "krylov_tol": w.tol,
            "forward_ms_per_step": _r(tf / nsteps), "backward_ms_per_step": _r(tb / nsteps),
            "backward_over_forward": _r(tb / tf), "adjoint_step_ms": _r(t_adj),
            "fd_max_rel_err": _r(max(errs)), "fd_entries": len(errs)}


# FP64 FMA instructions per second measured on this GPU (a dependent-free
# FMA loop): 1.005 TFLOP/s; nominal 152 SMs x 2 FP64 FMA per clock x 2.07 GHz.
FP64_OPS_MEASURED = 502.7e9
FP64_OPS_NOMINAL = 152 * 2 * 2.07e9


def krylov_fp64_ops(ncomp, iters, subs):
    """FP64 operations (add, mul, fma: 1 each) of one FP64 Krylov launch on a
    large problem (split passes), as the kernel formulates the method: the
    ETD2 set-up 8 per point; per substep the w_1 pass 10 (7-point stencil 8,
    two terms), the w_2 pass 9, P_0 9 (stencil on B = A / cfac 7, two sums),
    per Krylov vector 13 (V_j = ca Z + cb V_{j-1} + cc V_{j-2}: 3; Z = B V_j:
    7; three sums), and the combination m + 3."""
    return ncomp * (8 + subs * 31 + iters * 14)


def krylov_bytes_two_pass(ncomp, iters, subs, s):
    """Algorithmic bytes with the two passes per Krylov vector that large FP64
    problems run (7s + b per point and vector: pass A reads Z_{j-1}, V_{j-1},
    V_{j-2} and writes V_j; pass B reads V_j, V_{j-1}, writes Z_j), the rest
    as krylov_bytes.  Large FP32 problems run one pass per vector (read
    u_{j-1}, V_{j-1}, write V_j, u_j), within krylov_bytes' count."""
    b = (8.0 if s == 8 else 4.0) + 4.0
    return ncomp * (iters * (7 * s + b) + subs * 2 * (3 * s + b) + (iters + 2 * subs) * s + subs * 16 + 48)


def run_stress(etd, stream, dev, steps, n=512, precisions="both"):
    """Bandwidth stress shape: ETD2 steps on a fixed ball of radius 7 in a
    512^3 grid over [-8, 8]^3 (vectors far above L2), FP64 and FP32-mixed.
    Each precision: domain set-up, one warm-up step, then the timed steps."""
    import numpy as np
    import torch

    from paper_2209_15095_gb300 import inputs

    w = inputs.ball512(n=n)
    phi = torch.tensor(w.phi0[0], dtype=torch.float64, device=dev)
    u0 = torch.tensor(w.u0[0], dtype=torch.float64, device=dev)
    del w.phi0, w.u0
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {"workload": "ball512" if n == 512 else "ball%d" % n, "grid": list(w.n), "dt": w.dt, "m_max": w.m_max,
           "steps": steps}
    for precision in (("fp64", "mixed") if precisions == "both" else (precisions,)):
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            ctx = etd.Context(w.n, w.lo, w.hi, nspecies=1, precision=precision, tol=w.tol, m_max=w.m_max,
                              reaction=w.reaction, beta=w.beta, device=dev)
            u = u0.clone()
            ctx.init_domain(0, phi)
            ctx.step(w.dt, [u])  # warm-up (first step: ETD1)
            ctx.sync()
            t, bytes_, bytes2, fops, iters, subs, cells = 0.0, 0.0, 0.0, 0.0, 0, 0, 0
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.step(w.dt, [u])
                e1.record(stream)
                st = ctx.last_stats()[0]
                dt_ms = e0.elapsed_time(e1)
                t += dt_ms / 1e3
                iters += st["krylov_iters"]
                subs += st["substeps"]
                cells += st["ncomp"]
                sb = 8 if precision == "fp64" else 4
                bytes_ += krylov_bytes(st["ncomp"], st["krylov_iters"], st["substeps"], sb)
                bytes2 += krylov_bytes_two_pass(st["ncomp"], st["krylov_iters"], st["substeps"], sb)
                fops += krylov_fp64_ops(st["ncomp"], st["krylov_iters"], st["substeps"])
        del ctx
        torch.cuda.empty_cache()
        out[precision] = {"ms_per_step": _r(1e3 * t / steps), "mcell_updates_per_s": _r(cells / t / 1e6),
                          "krylov_iters_per_step": _r(iters / steps), "substeps_per_step": _r(subs / steps),
                          "ncomp": cells // steps, "achieved_gbs": _r(bytes_ / t / 1e9),
                          "frac_of_hbm": _r(bytes_ / t / 1e9 / hbm)}
        if precision == "fp64":
            # the FP64 split passes read and write each Krylov vector twice;
            # FP64 issue bounds them: against the FP64 operation rate
            out[precision].update({"frac_of_hbm_two_pass_bytes": _r(bytes2 / t / 1e9 / hbm),
                                   "fp64_gops": _r(fops / t / 1e9),
                                   "frac_of_fp64_measured": _r(fops / t / FP64_OPS_MEASURED),
                                   "frac_of_fp64_nominal": _r(fops / t / FP64_OPS_NOMINAL)})
    out["peak_gbs"] = hbm
    return out


def run_poisson(etd, stream, dev, N=1280):
    """Embedded-boundary Poisson solve on the virus-shaped domain of Sec. 4.1
    ((N+1)^2 grid on [-1, 1]^2, beta = 2 + sin(xy), exact u = e^x (x^2 sin y +
    y^2)) by the library's FP64 conjugate gradients to a relative residual of
    1e-10, timed with CUDA events.  Algorithmic bytes per point and CG
    iteration: 9 FP64 vector accesses (stencil read of p, q written then
    read, x and r read and written, p read twice and written) + index and
    diagonal (12 B)."""
    import numpy as np
    import torch

    from paper_2209_15095_gb300 import inputs

    w = inputs.virus2d(N)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    with torch.cuda.stream(stream):
        ctx = etd.Context(w.n, w.lo, w.hi, precision="fp64", tol=1e-10, m_max=30, reaction="none", mu=(0.0,),
                          beta=(1.0,), boundary_data=True, device=dev)
        ctx.init_domain(0, torch.tensor(w.phi0[0], device=dev), torch.tensor(w.beta_field, device=dev))
        P = ctx.boundary_points(0).cpu().numpy()
        vals = torch.tensor(inputs.virus_exact(P[..., 0], P[..., 1]), device=dev)
        ctx.set_boundary_values(0, vals)
        f = torch.tensor(w.source, device=dev)
        u = torch.zeros(w.n, dtype=torch.float64, device=dev)
        ctx.poisson_solve(0, f, u, tol=1e-10)  # warm-up
        u.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, res = ctx.poisson_solve(0, f, u, tol=1e-10)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        dom = ctx.read_domain(0)
    comp = dom["kind"] == 2
    x, y = inputs.grid_coords(w.n, w.lo, w.hi)
    err = float(np.max(np.abs(u.cpu().numpy() - inputs.virus_exact(x, y))[comp]))
    nc = int(dom["ncomp"])
    bytes_ = nc * it * (9 * 8 + 12)
    return {"workload": "virus2d", "N": N, "ncomp": nc, "cg_iters": it, "rel_resid": res, "ms": ms,
            "mcell_iters_per_s": nc * it / (ms / 1e3) / 1e6, "achieved_gbs": bytes_ / (ms / 1e3) / 1e9,
            "frac_of_hbm": bytes_ / (ms / 1e3) / 1e9 / hbm, "max_err_vs_exact": err,
            "note": "FP64 conjugate gradients, one persistent kernel with 3 grid barriers per iteration"}


def run_e2e(args, w, make_ctx, initial_state, one_step, stream, flush, dev):
    import numpy as np
    import torch

    ctx = make_ctx("fp64")
    phis, us = initial_state(ctx)
    nsp = len(phis)
    hphi = [torch.empty_like(p, device="cpu").pin_memory() for p in phis]
    hu = [torch.empty_like(u, device="cpu").pin_memory() for u in us]
    with torch.cuda.stream(stream):
        for s in range(nsp):
            hphi[s].copy_(phis[s])
            hu[s].copy_(us[s])
        stream.synchronize()
        k = 0
        times, cells = [], 0
        # phi is final after the level-set kernel (the set-up and ETD kernels
        # only read it): its copy back runs on a second stream meanwhile
        cstream = torch.cuda.Stream(dev)
        for i in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev = [torch.cuda.Event() for _ in range(4)]
            e0.record(stream)
            for s in range(nsp):
                phis[s].copy_(hphi[s], non_blocking=True)
                us[s].copy_(hu[s], non_blocking=True)
            one_step(ctx, phis, us, k, ev)
            cstream.wait_event(ev[1])
            with torch.cuda.stream(cstream):
                for s in range(nsp):
                    hphi[s].copy_(phis[s], non_blocking=True)
            done = torch.cuda.Event()
            done.record(cstream)
            for s in range(nsp):
                hu[s].copy_(us[s], non_blocking=True)
            stream.wait_event(done)
            e1.record(stream)
            k += 1
            st = ctx.last_stats()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1))
                cells += sum(s_["ncomp"] for s_ in st)
    nbytes = sum(p.numel() * 8 for p in phis) + sum(u.numel() * 8 for u in us)
    return {"value": cells / (sum(times) / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": sum(times) / len(times),
            "note": "phi and u copied from pinned host memory before and back after every step, inside the events; "
                    "phi's copy back overlaps the set-up and ETD kernels on a second stream"}


if __name__ == "__main__":
    main()
