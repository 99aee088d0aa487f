#!/usr/bin/env python3
"""Newton iterations per second of the fully-coupled hydraulic-fracture step
on one GB300 (assembly + ILU(0) block-Jacobi GMRES), through the C ABI.

Workload: 3D penny-shaped fracture, cube of 50 m side split into 18^3 cubes of
six P2 tetrahedra (34,992 elements, 1,051,129 unknowns), point injection at
the centre of z = 0, the facets of that plane crackable.  A step is one Newton
iteration of the time-stepping loop (Newton until converged, fracture
criterion, end of step); each linear solve is driven to a relative residual of
1e-8.  The headline runs the FP32-inner / FP64-refinement path; the FP64 path
is timed beside it on the same state.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica of the workload (the method's
instances are independent; nothing is exchanged), rank 0 prints one JSON line.
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

import numpy as np  # noqa: E402

METRIC = "Newton iters/s (assembly+GMRES) at ~1M DOF, FP64 vs mixed @1e-8; p99 latency"
UNIT = "Newton it/s"
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(name):
    from hf_inputs import c3_penny, kgd_2d, penny_3d
    if name == "c3":
        return c3_penny()
    if name == "small3d":
        return penny_3d(n=6, name="penny3d_n6")
    if name == "c1":
        return kgd_2d(n=44, name="c1_kgd2d_n44")
    raise ValueError(name)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) > 8:
                for n, v in zip(names, r[5:9]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def solver_kw(args, prec, graphs=None):
    """Solver options of the timed path: GMRES to a relative residual of 1e-8,
    each precision with its own cycle length and Gram-Schmidt passes."""
    mixed = prec == "mixed"
    return dict(precision=prec, restart=args.restart if mixed else args.fp64_restart,
                reorth=args.reorth if mixed else args.fp64_reorth, rtol=1e-8, inner_rtol=1e-3,
                max_iters=args.max_iters, jacobi_block=args.jacobi_block, newton_tol=1e-8,
                use_graphs=args.graphs if graphs is None else graphs, coarse=args.coarse)


def make_problem(wl, precision, stream_ptr, G, restart):
    from paper_1911_10275_gb300 import HFMesh
    g = HFMesh.from_mesh(wl.mesh, stream=stream_ptr)
    inj, wts = wl.injection()
    g.hf_set_material(wl.E, wl.nu, wl.sigma_c, wl.delta_c, wl.b_stab)
    g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, wl.dt, 0.0, True, wl.fluid_length)
    g.hf_set_solver(precision=precision, restart=restart, rtol=1e-8, inner_rtol=1e-3, max_iters=3000,
                    jacobi_block=G, newton_tol=1e-8)
    return g


class NewtonLoop:
    """Time stepping as the paper drives it: Newton to convergence, the
    fracture criterion, Newton again if it switched facets, then the end of
    the step.  As any driver of a Newton solver does, a step whose Newton
    iterations fail (no convergence within the cap, a linear solve that did
    not converge, or a non-finite state) is restarted from its initial state
    with half the time step; the step grows back after successes."""

    def __init__(self, g, wl, newton_cap=8):
        from paper_1911_10275_gb300 import HFError
        self.HFError = HFError
        self.g = g
        self.wl = wl
        self.cap = newton_cap
        self.dt0 = wl.dt
        self.dt = wl.dt
        self.it_in_step = 0
        self.rounds = 0
        self.reports = []
        self.latencies = []
        self.cutbacks = 0
        self.accepted = 0
        self.saved = g.hf_get_state()

    def _set_dt(self, dt):
        wl = self.wl
        inj, wts = wl.injection()
        self.dt = dt
        self.g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, dt, 0.0, True, wl.fluid_length)

    def _restart_step(self):
        U, P, a, b, w, t = self.saved
        self._set_dt(max(self.dt / 2, self.dt0 / 1024))
        self.g.hf_set_state(U, P, a, b, w, t)
        self.it_in_step = 0
        self.rounds = 0
        self.cutbacks += 1

    def step(self):
        t0 = time.perf_counter()
        try:
            rep = self.g.hf_newton_step()
        except self.HFError:
            rep = {"gmres_iters": 0, "converged": 0, "lin_converged": 0, "refinements": 0, "du_rel": float("nan"),
                   "dp_rel": float("nan"), "lin_res": float("nan"), "failed": 1}
            self._restart_step()
            self.reports.append(rep)
            self.latencies.append(time.perf_counter() - t0)
            return rep
        self.reports.append(rep)
        self.it_in_step += 1
        if rep["converged"]:
            new_alpha = self.g.hf_check_fracture_criterion()
            self.rounds += 1
            if new_alpha == 0 or self.rounds >= 4:
                self.g.hf_accept_step()
                self.accepted += 1
                self.it_in_step = 0
                self.rounds = 0
                self.saved = self.g.hf_get_state()
                if self.dt < self.dt0:
                    self._set_dt(min(self.dt0, self.dt * 1.5))
            else:
                self.it_in_step = 0
        elif self.it_in_step >= self.cap or not rep["lin_converged"]:
            self._restart_step()
        self.latencies.append(time.perf_counter() - t0)
        return rep


def algorithmic_bytes(stats, dim, elt):
    """Bytes one launch must move at minimum:
    SpMV: every stored element-block value once, x and y once, neighbour ids;
    preconditioner: diagonal inverses plus in-subdomain L/U blocks once, its
    input and output vector once."""
    ned = 30 if dim == 3 else 12
    nfr = 18 if dim == 3 else 6
    ne = stats["elements"]
    N = ne * ned + stats["n_p"]
    spmv_vals = ne * ned * ned + stats["interior_slots"] * ned * nfr
    prec_vals = ne * ned * ned + stats["subdomain_slots"] * ned * nfr
    return {"spmv": spmv_vals * elt + 2 * N * elt + ne * (dim + 1) * 4,
            "precond": prec_vals * elt + 2 * N * elt + ne * 8}


def traffic_from_profiles(kernel):
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        return d.get(kernel)
    except Exception:
        return None


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    wl = workload(args.config)
    stream = torch.cuda.Stream(device=dev)
    prec = "mixed" if args.precision == "mixed" else "fp64"
    g = make_problem(wl, prec, stream.cuda_stream, args.jacobi_block, args.restart)
    g.hf_set_solver(**solver_kw(args, prec))
    U, P, al, be = wl.seed()
    g.hf_set_state(U, P, al, be)
    loop = NewtonLoop(g, wl)
    for _ in range(args.warmup):
        loop.step()
    stats = g.hf_get_stats()
    launches0 = stats["kernel_launches"]
    g.hf_set_profiling(True)
    loop.reports.clear()
    loop.latencies.clear()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        loop.step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ktimes = g.hf_get_kernel_times()
    g.hf_set_profiling(False)
    timing_source = "CUDA events on the library stream inside the timed region"
    if args.graphs and ktimes["spmv"][1] == 0:
        # this driver/toolkit gave no timing for events recorded inside graphs:
        # time the kernels with events on the same state, graphs off, right after
        code = g.hf_get_stats()["graph_timing_error"]
        g.hf_set_solver(**solver_kw(args, prec, graphs=0))
        g.hf_set_profiling(True)
        for _ in range(2):
            loop.step()
        ktimes = g.hf_get_kernel_times()
        g.hf_set_profiling(False)
        g.hf_set_solver(**solver_kw(args, prec))
        timing_source = ("CUDA events over 2 Newton iterations right after the timed region, same state, "
                         f"graphs off (graph-node event timing unavailable: CUDA error {code})")
    stats = g.hf_get_stats()
    launches = stats["kernel_launches"] - launches0
    reports = list(loop.reports)
    lat = sorted(loop.latencies)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = args.steps * world / (ms / 1000.0)

    # end to end through the public API with host buffers: the same time
    # loop, but every step uploads the state from pinned host memory and reads
    # the updated state back
    e2e = None
    if args.e2e_steps > 0:
        le = loop  # continue the timed time loop from where it stopped
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        host = [pin(x) for x in g.hf_get_state()[:5]] + [0.0]
        h2d = sum(x.nbytes for x in host[:5])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            g.hf_set_state(*host[:5], host[5])
            le.step()
            out = g.hf_get_state()
            for dst, src in zip(host[:5], out[:5]):
                dst[...] = src
            host[5] = out[5]
        torch.cuda.synchronize(dev)
        te = time.perf_counter() - t0
        e2e = {"value": args.e2e_steps / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(h2d), "steps": args.e2e_steps}

    # FP64 beside it on the same starting state (fewer steps)
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        g.hf_set_solver(**solver_kw(args, "fp64"))
        g.hf_set_state(U, P, al, be)
        l64 = NewtonLoop(g, wl)
        for _ in range(min(args.warmup, 2)):
            l64.step()
        l64.reports.clear()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            l64.step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": args.fp64_steps / (ms64 / 1000.0), "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": ms64 / args.fp64_steps,
                "gmres_iters_per_newton": float(np.mean([r["gmres_iters"] for r in l64.reports])),
                "restart": args.fp64_restart, "reorth": args.fp64_reorth}
        g.hf_set_solver(**solver_kw(args, prec))

    # roofline of the dominant kernel class, from the events of the timed region
    elt = 4 if prec == "mixed" else 8
    algo = algorithmic_bytes(stats, wl.mesh.dim, elt)
    cand = {k: ktimes[k] for k in ("spmv", "precond")}
    dom = max(cand, key=lambda k: cand[k][0])
    kms, kl = cand[dom]
    peak, peak_src = peaks()
    achieved = algo[dom] / (kms / kl / 1000.0) / 1e9 if kl else 0.0
    kname = {"spmv": f"k_spmv<{'float' if elt == 4 else 'double'},3,0>",
             "precond": f"k_ilu_apply<{'float' if elt == 4 else 'double'},3>"}[dom]
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": int(algo[dom]), "launches": kl,
                "avg_launch_us": 1000.0 * kms / kl if kl else None,
                "traffic": traffic_from_profiles(kname)}
    total_ms = sum(v[0] for v in ktimes.values())
    breakdown = {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in ktimes.items() if v[1]}

    gmres = [r["gmres_iters"] for r in reports]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-inner/f64-refinement" if prec == "mixed" else "f64",
        "data": "synthetic (seeded structured P2 mesh and seed crack)",
        "config": {"workload": wl.name, "dofs": int(g.N), "elements": int(wl.mesh.n_elems),
                   "precision": prec, "gmres_rtol": 1e-8, "restart": args.restart, "reorth": bool(args.reorth),
                   "preconditioner": ("block-Jacobi ILU(0) + rigid-body coarse level (%d coarse unknowns)"
                                      % stats.get("coarse_unknowns", 0)) if args.coarse else "block-Jacobi ILU(0)",
                   "jacobi_block": args.jacobi_block, "cuda_graphs": bool(args.graphs),
                   "parallelism": f"replicas x{world}",
                   "l2": "working set larger than L2 (matrix + factor %.2f GB per replica)" %
                         (2 * algo["spmv"] / 1e9)},
        "fp64": fp64,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roofline,
        "kernel_ms": breakdown,
        "kernel_timing_source": timing_source,
        "kernel_ms_total_share_of_step": total_ms / ms if ms else None,
        "gmres_iters_per_newton": float(np.mean(gmres)) if gmres else None,
        "newton_latency_ms": {"p50": 1000 * lat[len(lat) // 2], "p99": 1000 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]}
        if lat else None,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and args.cpu_baseline:
        out["cpu_baseline"] = oracle_baseline(wl, args.cpu_budget)
    g.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def oracle_baseline(wl, budget_s):
    """The oracle as it stands on the host cores, on a bounded sample of the
    same workload: the residual and Jacobian terms of a sample of elements and
    interior facets, scaled to the whole mesh.  The oracle's sparse direct
    solve cannot run at this size (fill-in), so the figure excludes the linear
    solve and is an upper bound on the oracle's Newton rate."""
    from oracle import Oracle, Params
    inj, wts = wl.injection()
    t0 = time.perf_counter()
    prm = Params(E=wl.E, nu=wl.nu, sigma_c=wl.sigma_c, delta_c=wl.delta_c, b_stab=wl.b_stab, mu=wl.mu, Q0=wl.Q0,
                 inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=wl.delta_f, dt=wl.dt, L_ref=wl.fluid_length)
    o = Oracle(wl.mesh, prm)
    U, P, al, be = wl.seed()
    o.set_state(U, P, al, be)
    t_setup = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    interior = np.nonzero(wl.mesh.face_elems[:, 1] >= 0)[0]
    n_e = n_f = 0
    t_e = t_f = 0.0
    deadline = time.perf_counter() + budget_s
    while time.perf_counter() < deadline:
        e = int(rng.integers(0, o.ne))
        t1 = time.perf_counter()
        o.element_stiffness(e)
        t_e += time.perf_counter() - t1
        n_e += 1
        f = int(interior[rng.integers(0, interior.size)])
        t1 = time.perf_counter()
        o.intact_blocks(f)
        t_f += time.perf_counter() - t1
        n_f += 1
    t_full = t_e / n_e * o.ne + t_f / n_f * interior.size
    return {"value": 1.0 / t_full, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle assembly of {n_e} random elements and {n_f} random interior facets of "
                      f"{wl.name} ({o.ne} elements, {interior.size} interior facets), scaled to the full "
                      f"mesh ({t_full:.1f} s per Newton iteration); sparse direct solve excluded "
                      f"(infeasible at this size), so an upper bound; set-up {t_setup:.1f} s"}


def _solver_for_requests(args, tuner=None):
    base = {"precision": args.precision, "rtol": 1e-8, "inner_rtol": 1e-3, "max_iters": args.request_max_iters,
            "newton_tol": 1e-8, "use_graphs": 1, "jacobi_block": args.jacobi_block, "restart": args.restart,
            "reorth": args.reorth, "coarse": args.coarse}
    if tuner is None:
        return lambda wl: dict(base)
    return lambda wl: {**tuner.solver_for(wl, args.precision), "max_iters": args.request_max_iters}


REQUEST_STEP = {"newton_max": 8, "criterion_rounds": 4, "max_cutbacks": 4}


def serving_run(args, count, rate, slots, seed=191110275, warm=True):
    """Poisson stream of KGD and penny requests through the native request
    loop; returns the latency summary and the run's description."""
    import torch
    from hf_inputs import serving_requests
    from paper_1911_10275_gb300 import HFRuntime
    from paper_1911_10275_gb300.serving import run_stream, latency_summary
    cache = {}
    t_gen = time.perf_counter()
    arrivals, reqs = serving_requests(count, rate=rate, seed=seed, steps=args.serve_steps, mesh_cache=cache)
    t_gen = time.perf_counter() - t_gen
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    rt = HFRuntime(slots=slots, hbm_budget_bytes=budget)
    solver_for = _solver_for_requests(args)
    if warm:  # one small request first, so that module loading is not in the first latency
        run_stream(rt, [0.0], reqs[:1], 1, solver_for, step=REQUEST_STEP)
    recs = run_stream(rt, arrivals, reqs, args.serve_steps, solver_for, step=REQUEST_STEP)
    st = rt.stats()
    rt.close()
    summ = latency_summary(recs)
    summ.update({"requests": count, "rate_req_s": rate, "slots": slots, "steps_per_request": args.serve_steps,
                 "hbm_budget_gb": round(budget / 1e9, 1), "peak_admitted_gb": round(st["peak_bytes"] / 1e9, 2),
                 "peak_running": st["peak_running"], "precision": args.precision,
                 "unknowns_range": [int(min(r["n_u"] + r["n_p"] for r in recs)),
                                    int(max(r["n_u"] + r["n_p"] for r in recs))],
                 "kinds": {"kgd2d": sum(1 for w in reqs if w.mesh.dim == 2),
                           "penny3d": sum(1 for w in reqs if w.mesh.dim == 3)},
                 "mesh_generation_s": round(t_gen, 1)})
    return summ, recs


def _log_records(recs):
    for r in recs:
        print(f"{r['name']:26s} status={r['status']} unknowns={r['n_u'] + r['n_p']} steps={r['steps_done']} "
              f"newton={r['newton_iters']} gmres={r['gmres_iters']} cutbacks={r['cutbacks']} "
              f"latency={r['latency']:.2f}s queue={r['queue'] if r['queue'] is None else round(r['queue'], 2)}",
              file=sys.stderr)


def run_serve(args):
    """The serving configuration: a Poisson stream of solve requests (half
    2D KGD, half 3D penny), admitted by HBM budget into `slots` concurrent
    requests; p50/p99 latency and throughput."""
    import torch
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    summ, recs = serving_run(args, args.serve_requests, args.serve_rate, args.slots)
    clocks = sampler.stop()
    if args.verbose:
        _log_records(recs)
    out = {"metric": "serving latency p99 (ms) under a Poisson request stream", "value": summ.get("p99_ms"),
           "unit": "ms", "n_gpus": 1, "higher_is_better": False, "mode": "serve", "data": "synthetic",
           "dtype": "f32-inner/f64-refinement" if args.precision == "mixed" else "f64",
           "config": {"workload": f"serving stream: KGD n in [50, 316] and penny n in [8, 22], "
                                  f"{args.serve_requests} requests of {args.serve_steps} steps"},
           "serving": summ, "clocks": clocks}
    print(json.dumps(out))


def run_sweep(args):
    """The batched sweep: independent 2D KGD instances of uneven size, all
    submitted at once to the request loop, solver shape per size class from
    the autotuner; aggregate Newton iterations per second and makespan."""
    import torch
    from hf_inputs import sweep_instances
    from paper_1911_10275_gb300 import HFRuntime
    from paper_1911_10275_gb300.autotune import Tuner
    from paper_1911_10275_gb300.serving import run_stream, latency_summary
    torch.cuda.set_device(0)
    cache = {}
    wls = sweep_instances(args.sweep_count, mesh_cache=cache, steps=args.sweep_steps)
    tuner = None
    t_tune = 0.0
    if args.autotune:
        tuner = Tuner()
        t0 = time.perf_counter()
        for wl in wls:
            tuner.tune(wl, args.precision)
        t_tune = time.perf_counter() - t0
    free, _ = torch.cuda.mem_get_info()
    rt = HFRuntime(slots=args.slots, hbm_budget_bytes=int(0.8 * free))
    solver_for = _solver_for_requests(args, tuner)
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    recs = run_stream(rt, [0.0] * len(wls), wls, args.sweep_steps, solver_for, step=REQUEST_STEP)
    span = time.perf_counter() - t0
    clocks = sampler.stop()
    if args.verbose:
        _log_records(recs)
    st = rt.stats()
    rt.close()
    summ = latency_summary(recs)
    newton = sum(r["newton_iters"] for r in recs if r["status"] == 0)
    out = {"metric": "batched sweep: aggregate Newton iterations per second", "value": newton / span,
           "unit": "Newton it/s", "n_gpus": 1, "higher_is_better": True, "mode": "sweep", "data": "synthetic",
           "dtype": "f32-inner/f64-refinement" if args.precision == "mixed" else "f64",
           "config": {"workload": f"{len(wls)} KGD instances, 1k-50k P2 triangles, {args.sweep_steps} steps each",
                      "slots": args.slots, "autotuned": bool(args.autotune)},
           "makespan_s": span, "instance_steps_per_s": sum(r["steps_done"] for r in recs) / span,
           "completed": summ.get("completed"), "failed": summ.get("failed"),
           "peak_running": st["peak_running"], "autotune_s": t_tune,
           "tuned": tuner.report() if tuner else None, "clocks": clocks}
    print(json.dumps(out))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = workload(args.config)
    base = oracle_baseline(wl, args.cpu_budget)
    out = {"metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000.0 / base["value"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
           "data": "synthetic (seeded structured P2 mesh and seed crack)",
           "config": {"workload": wl.name, "precision": "fp64 oracle"},
           "cpu_baseline": base,
           "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--jacobi-block", dest="jacobi_block", type=int, default=32)
    ap.add_argument("--restart", type=int, default=60)
    ap.add_argument("--reorth", type=int, default=1)
    ap.add_argument("--fp64-restart", dest="fp64_restart", type=int, default=60)
    ap.add_argument("--fp64-reorth", dest="fp64_reorth", type=int, default=0)
    ap.add_argument("--max-iters", dest="max_iters", type=int, default=8000)
    ap.add_argument("--coarse", type=int, default=1)
    ap.add_argument("--graphs", type=int, default=1)
    ap.add_argument("--fp64-steps", dest="fp64_steps", type=int, default=3)
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=4)
    ap.add_argument("--cpu-budget", dest="cpu_budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--mode", default="newton", choices=["newton", "serve", "sweep"])
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-requests", dest="serve_requests", type=int, default=0)
    ap.add_argument("--serve-rate", dest="serve_rate", type=float, default=200.0)
    ap.add_argument("--serve-steps", dest="serve_steps", type=int, default=5)
    ap.add_argument("--sweep-count", dest="sweep_count", type=int, default=256)
    ap.add_argument("--sweep-steps", dest="sweep_steps", type=int, default=10)
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--verbose", type=int, default=0)
    ap.add_argument("--request-max-iters", dest="request_max_iters", type=int, default=3000)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "sweep":
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
