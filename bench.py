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
    from hf_inputs import c2_kgd_viscosity, c3_penny, kgd_2d, penny_3d
    if name == "c3":
        return c3_penny()
    if name == "c2":
        return c2_kgd_viscosity()
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


# The timed solver settings.  GMRES tolerances are the loosest that keep every
# Newton iterate within relative 1e-8 of the FP64 oracle's (openings,
# pressures, displacements), as tests/test_gpu_accuracy.py checks along the
# oracle's trajectory: FP32 inner sweeps reducing the residual 1e4-fold inside
# FP64 refinement to 1e-11, and plain FP64 GMRES to 1e-11; cycles of 90 and
# 32-element subdomains (the fastest of G in {16, 32, 64}, m in {40, 60, 90},
# inner reduction in {1e-2, 1e-3, 1e-4} on the first Newton iterations).
HEADLINE = {"mixed": dict(precision="mixed", restart=90, reorth=3, rtol=1e-11, inner_rtol=1e-4),
            "fp64": dict(precision="fp64", restart=90, reorth=3, rtol=1e-11, inner_rtol=1e-4)}
COMMON = dict(jacobi_block=32, coarse=1, use_graphs=1, newton_tol=1e-8, max_iters=8000)


def solver_kw(args, prec, graphs=None):
    """Solver options of the timed path: GMRES to the relative residual of
    each precision (--rtol, --fp64-rtol), each precision with its own cycle
    length and Gram-Schmidt passes."""
    mixed = prec == "mixed"
    return dict(precision=prec, restart=args.restart if mixed else args.fp64_restart,
                reorth=args.reorth if mixed else args.fp64_reorth, rtol=args.rtol if mixed else args.fp64_rtol,
                inner_rtol=args.inner_rtol,
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
    iterations fail (no convergence within the cap, a linear solve that
    missed its tolerance by more than a decade, or a non-finite state) is
    restarted from its initial state with half the time step; the step grows
    back after successes."""

    def __init__(self, g, wl, newton_cap=8, rtol=None):
        from paper_1911_10275_gb300 import HFError
        self.HFError = HFError
        # a linear solve that stagnated within a decade of its tolerance is
        # accepted (the attainable accuracy of FP64 GMRES right after the
        # fracture criterion switched facets); one further off fails the step
        self.rtol = rtol if rtol is not None else 1e-8
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
        elif self.it_in_step >= self.cap or not (rep["lin_converged"] or rep["lin_res"] <= 10 * self.rtol):
            self._restart_step()
        self.latencies.append(time.perf_counter() - t0)
        return rep


def algorithmic_bytes(stats, dim, elt, nc=0):
    """Bytes one launch must move at minimum, per kernel class:
    SpMV: every stored element-block value once, x and y once, neighbour ids;
    preconditioner (ILU(0) apply): diagonal inverses plus in-subdomain L/U
    blocks once, its input and output vector once, the 8-byte task records;
    coarse level per apply: restriction (r and the nodal coordinates of the
    modes), the dense inverse, prolongation (coordinates, z read and written)."""
    ned = 30 if dim == 3 else 12
    nfr = 18 if dim == 3 else 6
    ne = stats["elements"]
    nu = ne * ned
    N = nu + stats["n_p"]
    spmv_vals = ne * ned * ned + stats["interior_slots"] * ned * nfr
    prec_vals = ne * ned * ned + stats["subdomain_slots"] * ned * nfr
    return {"spmv": spmv_vals * elt + 2 * N * elt + ne * (dim + 1) * 4,
            "precond": prec_vals * elt + 2 * N * elt + ne * 8,
            "coarse": (nu * elt + nu * elt) + nc * nc * elt + (nu * elt + 2 * nu * elt) if nc else 0,
            "N": N}


def gs_bytes(N, elt, steps, cols, reorths, reorth_cols, reorth_mode):
    """Algorithmic bytes of the Gram-Schmidt kernels over `steps` Arnoldi
    steps (cols = the sum of j + 1 over them).  Delayed CGS2 (mode 3) streams
    the j final basis vectors twice per step (the fused dot products, then
    the fused update) and the lagged vector and w twice each, and writes v_j
    and the next lagged vector: 2 j + 6 vectors.  Classical Gram-Schmidt
    streams the j + 1 vectors twice per pass and w five times; a second pass
    adds two basis sweeps and three of w."""
    if reorth_mode == 3:
        return N * elt * (2 * (cols - steps) + 6 * steps)
    return N * elt * (2 * cols + 5 * steps + 2 * reorth_cols + 3 * reorths)


def traffic_from_profiles(kernel):
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        return d.get(kernel)
    except Exception:
        return None


GOLDEN = {"c3_penny3d_n18_mixed": os.path.join(ROOT, "tests", "golden", "c3_newton_oracle.json")}


def load_golden(wl):
    """The oracle's trajectory of this workload, written by
    tests/golden/make_c3_newton.py (oracle only), or None."""
    p = GOLDEN.get(wl.name)
    if not p or not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def errors_vs_golden(rec, u_idx, U, P, W):
    """Relative errors of one Newton iterate against the oracle's: U on the
    stored sample of unknowns, every non-zero oracle pressure, the openings at
    the face nodes of every cohesive or fluid facet, each over the infinity
    norm of the oracle's full field."""
    eu = float(np.abs(U[u_idx] - np.asarray(rec["U"])).max() / rec["U_inf"])
    pi = np.asarray(rec["P_index"], dtype=np.int64)
    ep = float(np.abs(P[pi] - np.asarray(rec["P"])).max() / rec["P_inf"]) if pi.size else 0.0
    wf = np.asarray(rec["w_faces"], dtype=np.int64)
    ew = float(np.abs(W[wf] - np.asarray(rec["w"])).max() / rec["w_inf"]) if wf.size else 0.0
    return {"U": eu, "P": ep, "w": ew}


def _reset(g, wl, seed):
    """Back to the seed state at t = 0 with the full time step."""
    inj, wts = wl.injection()
    g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, wl.dt, 0.0, True, wl.fluid_length)
    g.hf_set_state(*seed)


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
    seed = wl.seed()
    golden = load_golden(wl)

    # warm-up: the first W Newton iterations of the time loop (graphs captured)
    _reset(g, wl, seed)
    loop = NewtonLoop(g, wl, rtol=args.rtol if prec == "mixed" else args.fp64_rtol)
    for _ in range(args.warmup):
        loop.step()

    # timed region: the first K Newton iterations of the time loop again, from
    # the same seed state, state resident on the device
    _reset(g, wl, seed)
    loop = NewtonLoop(g, wl, rtol=args.rtol if prec == "mixed" else args.fp64_rtol)
    st0 = g.hf_get_stats()
    g.hf_set_profiling(2)       # events around each whole GMRES cycle only
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
    cyc_ms, cyc_steps = g.hf_get_kernel_times()["gmres_cycles"]
    g.hf_set_profiling(False)
    st1 = g.hf_get_stats()
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    reports = list(loop.reports)
    lat = sorted(loop.latencies)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = args.steps * world / (ms / 1000.0)

    # kernel classes: the same trajectory once more with CUDA events around
    # every kernel class on the library's stream (graphs off: events recorded
    # inside captured graphs give no timings on this toolkit), at least 10
    # iterations
    n_prof = max(10, args.steps)
    g.hf_set_solver(**solver_kw(args, prec, graphs=0))
    _reset(g, wl, seed)
    lp = NewtonLoop(g, wl, rtol=args.rtol if prec == "mixed" else args.fp64_rtol)
    sp0 = g.hf_get_stats()
    g.hf_set_profiling(True)
    for _ in range(n_prof):
        lp.step()
    ktimes = g.hf_get_kernel_times()
    g.hf_set_profiling(False)
    sp1 = g.hf_get_stats()
    g.hf_set_solver(**solver_kw(args, prec))
    arnoldi = sum(r["gmres_iters"] for r in lp.reports)
    elt = 4 if prec == "mixed" else 8
    algo = algorithmic_bytes(st1, wl.mesh.dim, elt, st1.get("coarse_unknowns", 0))
    N = algo["N"]
    orth_bytes = gs_bytes(N, elt, arnoldi, sp1["gs_cols"] - sp0["gs_cols"], sp1["gs_reorths"] - sp0["gs_reorths"],
                          sp1["gs_reorth_cols"] - sp0["gs_reorth_cols"], args.reorth if prec == "mixed" else args.fp64_reorth)
    peak, peak_src = peaks()
    cls = {
        "spmv": (algo["spmv"] * ktimes["spmv"][1], ktimes["spmv"][0], ktimes["spmv"][1],
                 f"k_spmv<{'float' if elt == 4 else 'double'},3,0>"),
        "precond": (algo["precond"] * ktimes["precond"][1], ktimes["precond"][0], ktimes["precond"][1],
                    f"k_ilu_apply<{'float' if elt == 4 else 'double'},3>"),
        "orth": (orth_bytes, ktimes["orth"][0], ktimes["orth"][1],
                 (f"k_dc_dot/k_dc_upd<{'float' if elt == 4 else 'double'}> (delayed CGS2)" if
                  (args.reorth if prec == "mixed" else args.fp64_reorth) == 3 else
                  f"k_gs_dot/k_gs_sub/k_gs_fin<{'float' if elt == 4 else 'double'}> (Gram-Schmidt)")),
        "precond_aux": (algo["coarse"] * ktimes["precond"][1], ktimes["precond_aux"][0], ktimes["precond_aux"][1],
                        "coarse level + pressure rows"),
    }
    dom = max(cls, key=lambda k: cls[k][1])
    b_dom, ms_dom, n_dom, kname = cls[dom]
    achieved = b_dom / (ms_dom / 1000.0) / 1e9 if ms_dom > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": kname, "class": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "algorithmic_bytes": int(b_dom),
                "launches": n_dom, "ms": ms_dom, "traffic": traffic_from_profiles(kname.split(" ")[0])}
    if isinstance(roofline["traffic"], dict):
        # measured traffic / algorithmic bytes of the captured launch, applied
        # to this run's algorithmic bytes per Arnoldi step (the class's unit)
        t = roofline["traffic"]
        per_step = b_dom / max(arnoldi, 1)
        roofline["traffic"] = t["bytes"] / t["algorithmic"] * per_step
        roofline["traffic_unit"] = (f"bytes per Arnoldi step (dot + update kernels), ncu capture at j = "
                                    f"{t['captured_at_j']} scaled by the run's algorithmic bytes per step")
        roofline["algorithmic_bytes_per_step"] = per_step
    sol_bytes = sum(v[0] for v in cls.values())
    sol_ms = sum(v[1] for v in cls.values())
    # the same bytes per Arnoldi step against the real schedule: whole GMRES
    # cycles (graph replays, coarse level beside the ILU apply) timed inside
    # the timed region
    bytes_per_step = sol_bytes / max(arnoldi, 1)
    cyc_achieved = bytes_per_step * cyc_steps / (cyc_ms / 1000.0) / 1e9 if cyc_ms > 0 else 0.0
    solve_phase = {"classes": {k: {"GB": round(v[0] / 1e9, 3), "ms": round(v[1], 3), "launches": v[2],
                                   "GB_s": round(v[0] / (v[1] / 1e3) / 1e9, 1) if v[1] else None}
                               for k, v in cls.items()},
                   "arnoldi_steps": arnoldi, "GB_per_arnoldi_step": round(sol_bytes / max(arnoldi, 1) / 1e9, 4),
                   "us_per_arnoldi_step": round(1000.0 * sol_ms / max(arnoldi, 1), 2),
                   "achieved": cyc_achieved, "peak": peak, "frac": cyc_achieved / peak,
                   "timed_cycles": {"ms": round(cyc_ms, 3), "arnoldi_steps": int(cyc_steps),
                                    "us_per_arnoldi_step": round(1000.0 * cyc_ms / max(cyc_steps, 1), 2),
                                    "source": "CUDA events around each GMRES cycle (graph replay) inside the "
                                              "timed region; bytes per step from the class accounting below"},
                   "serialised_classes": {"achieved": sol_bytes / (sol_ms / 1000.0) / 1e9 if sol_ms else 0.0,
                                          "frac": (sol_bytes / (sol_ms / 1000.0) / 1e9) / peak if sol_ms else 0.0,
                                          "note": "sum of the per-class event times of the graphs-off replay "
                                                  "(no overlap of the coarse level)"},
                   "second_gs_pass_rate": round((sp1["gs_reorths"] - sp0["gs_reorths"]) / max(arnoldi, 1), 4),
                   "mean_j_plus_1": round((sp1["gs_cols"] - sp0["gs_cols"]) / max(arnoldi, 1), 2),
                   "source": f"CUDA events per kernel class on the library stream over {n_prof} Newton iterations "
                             f"of the timed trajectory, graphs off"}
    breakdown = {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in ktimes.items() if v[1]}

    # end to end through the public API with host buffers: the same K
    # iterations from the same seed, every step uploading the state from
    # pinned host memory and reading the updated state back
    e2e = None
    acc_mixed = None
    if args.e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        _reset(g, wl, seed)
        le = NewtonLoop(g, wl, rtol=args.rtol if prec == "mixed" else args.fp64_rtol)
        host = [pin(x) for x in g.hf_get_state()[:5]] + [0.0]
        res = [pin(x) for x in g.hf_get_opening_pressure()[:2]]
        h2d = sum(x.nbytes for x in host[:5])
        d2h = h2d + sum(x.nbytes for x in res)
        states = []
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g.hf_set_state(*host[:5], host[5])
            le.step()
            out = g.hf_get_state()
            for dst, src in zip(host[:5], out[:5]):
                dst[...] = src
            host[5] = out[5]
            for dst, src in zip(res, g.hf_get_opening_pressure()[:2]):
                dst[...] = src
            if golden is not None:
                states.append((host[0].copy(), host[1].copy(), res[0].copy()))
        torch.cuda.synchronize(dev)
        te = time.perf_counter() - t0
        e2e = {"value": args.steps / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": args.steps,
               "note": "the same Newton iterations as the timed region; every step uploads the state from "
                       "pinned host memory and reads back the state, the face-node openings and the pressures"}
        if golden is not None:
            acc_mixed = accuracy(wl, golden, states)

    # FP64 beside it: the same trajectory, timed, then checked
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        g.hf_set_solver(**solver_kw(args, "fp64"))
        _reset(g, wl, seed)
        l64 = NewtonLoop(g, wl, rtol=args.fp64_rtol)
        for _ in range(min(args.warmup, 2)):
            l64.step()
        _reset(g, wl, seed)
        l64 = NewtonLoop(g, wl, rtol=args.fp64_rtol)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            l64.step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": args.fp64_steps / (ms64 / 1000.0), "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": ms64 / args.fp64_steps, "gmres_rtol": args.fp64_rtol,
                "gmres_iters_per_newton": float(np.mean([r["gmres_iters"] for r in l64.reports])),
                "gmres_iters_per_step": [int(r["gmres_iters"]) for r in l64.reports],
                "lin_res_per_step": [float("%.3g" % r["lin_res"]) for r in l64.reports],
                "restart": args.fp64_restart, "reorth": args.fp64_reorth}
        if golden is not None:
            _reset(g, wl, seed)
            lc = NewtonLoop(g, wl, rtol=args.fp64_rtol)
            states = []
            for _ in range(args.fp64_steps):
                lc.step()
                U, P = g.hf_get_state()[:2]
                states.append((U, P, g.hf_get_opening_pressure()[0]))
            fp64["accuracy_vs_oracle"] = accuracy(wl, golden, states)
        g.hf_set_solver(**solver_kw(args, prec))

    gmres = [r["gmres_iters"] for r in reports]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-inner/f64-refinement" if prec == "mixed" else "f64",
        "data": "synthetic (seeded structured P2 mesh and seed crack)",
        "config": {"workload": wl.name, "dofs": int(g.N), "elements": int(wl.mesh.n_elems),
                   "precision": prec, "gmres_rtol": args.rtol, "inner_rtol": args.inner_rtol, "restart": args.restart,
                   "reorth": args.reorth,
                   "preconditioner": ("block-Jacobi ILU(0) + rigid-body coarse level (%d coarse unknowns)"
                                      % st1.get("coarse_unknowns", 0)) if args.coarse else "block-Jacobi ILU(0)",
                   "jacobi_block": args.jacobi_block, "cuda_graphs": bool(args.graphs),
                   "timed_work": f"Newton iterations 1..{args.steps} of the time loop from the seed state "
                                 f"(after {args.warmup} untimed iterations of the same loop)",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (matrix + factor %.2f GB per replica, L2 129 MB)" %
                         ((algo["spmv"] + algo["precond"]) / 1e9)},
        "accuracy_vs_oracle": acc_mixed,
        "fp64": fp64,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roofline,
        "solve_phase": solve_phase,
        "kernel_ms": breakdown,
        "gmres_iters_per_newton": float(np.mean(gmres)) if gmres else None,
        "gmres_iters_per_step": [int(x) for x in gmres],
        "newton_latency_ms": {"p50": 1000 * lat[len(lat) // 2], "p99": 1000 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]}
        if lat else None,
        "clocks": clocks,
    }
    g.close()
    if rank == 0 and world == 1 and args.serve_sample > 0:
        # a bounded sample of the request stream: the p99 latency the metric
        # names, measured on requests drawn from the serving configuration
        import copy
        a2 = copy.copy(args)
        a2.serve_steps = 1
        t0 = time.perf_counter()
        summ, recs = serving_run(a2, args.serve_sample, 200.0, args.slots)
        summ["wall_s"] = round(time.perf_counter() - t0, 1)
        summ["sample"] = (f"{args.serve_sample} requests of the Poisson stream at 200 requests/s (half KGD with "
                          f"5k-200k P2 triangles, half penny with 65k-2M unknowns), one time step each, "
                          f"{args.slots} slots, FP32 inner / FP64 refinement to 1e-8, Newton to 1e-8")
        out["serving"] = summ
    if rank == 0 and world == 1 and args.cpu_baseline:
        out["cpu_baseline"] = oracle_baseline(args.cpu_n)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def accuracy(wl, golden, states):
    """Per-iteration relative errors (U sample, pressures, face-node openings)
    of the GPU iterates against the oracle's trajectory of the same loop."""
    u_idx = np.asarray(golden["u_index"], dtype=np.int64)
    per = []
    for rec, (U, P, W) in zip(golden["iters"], states):
        e = errors_vs_golden(rec, u_idx, U, P, W)
        per.append({"k": rec["k"], **{k: float("%.3g" % v) for k, v in e.items()}})
    worst = {k: max(p[k] for p in per) for k in ("U", "P", "w")} if per else None
    return {"max_rel_err": worst, "per_step": per, "steps_compared": len(per),
            "oracle": "tests/golden/c3_newton_oracle.json (FP64 oracle trajectory, ILU(0)-GMRES to 1e-13)"}


def oracle_baseline(n):
    """The oracle as it stands on the host cores: one full Newton iteration
    (assembly summed over a pool of host processes, then the oracle's
    ILU(0)-GMRES solve to a relative residual of 1e-13) of the penny workload
    at mesh size n from its seed state.  Reported at that size, not scaled."""
    from hf_inputs import penny_3d
    from oracle import Oracle, Params, parallel
    from oracle.iterative import solve_linear_iterative
    wl = penny_3d(n=n, crackable="plane", name=f"penny3d_n{n}_plane")
    inj, wts = wl.injection()
    prm = Params(E=wl.E, nu=wl.nu, sigma_c=wl.sigma_c, delta_c=wl.delta_c, b_stab=wl.b_stab, mu=wl.mu, Q0=wl.Q0,
                 inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=wl.delta_f, dt=wl.dt, cutoff_on=True,
                 L_ref=wl.fluid_length, newton_tol=1e-8)
    o = Oracle(wl.mesh, prm)
    o.set_state(*wl.seed())
    cores = os.cpu_count() or 1
    info = {}
    t0 = time.perf_counter()
    o.newton_step(solve=lambda J, b: solve_linear_iterative(J, b, rtol=1e-13, info=info),
                  assemble=lambda: parallel.assemble(o, workers=cores))
    t = time.perf_counter() - t0
    return {"value": 1.0 / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one full FP64 oracle Newton iteration (assembly over {cores} host processes, "
                      f"ILU(0)-GMRES to 1e-13 on one core: {info.get('iters')} iterations) of the penny workload "
                      f"at n = {n} ({o.N} unknowns, {o.ne} elements) from its seed state, {t:.1f} s; "
                      f"measured at that size, not scaled to the 1.05 M-unknown workload"}


def _solver_for_requests(args, tuner=None):
    base = {"precision": args.precision, "rtol": 1e-8, "inner_rtol": 1e-3, "max_iters": args.request_max_iters,
            "newton_tol": 1e-8, "use_graphs": 1, "jacobi_block": args.jacobi_block, "restart": args.restart,
            "reorth": args.reorth, "coarse": args.coarse}
    if tuner is None:
        return lambda wl: dict(base)
    return lambda wl: {**tuner.solver_for(wl, args.precision), "max_iters": args.request_max_iters}


REQUEST_STEP = {"newton_max": 8, "criterion_rounds": 4, "max_cutbacks": 10}


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
    from paper_1911_10275_gb300.replicas import my_share, max_over_ranks, sum_over_ranks
    from paper_1911_10275_gb300.serving import run_stream, latency_summary
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local if world > 1 else 0)
    cache = {}
    wls_all = sweep_instances(args.sweep_count, mesh_cache=cache, steps=args.sweep_steps)
    # instances split across ranks by their cost (element count times steps),
    # longest first onto the least-loaded rank; nothing is exchanged
    share = my_share([wl.mesh.n_elems * args.sweep_steps for wl in wls_all], rank, world)
    wls = [wls_all[i] for i in share]
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
    span = max_over_ranks(span)
    newton = sum_over_ranks(newton)
    steps_done = sum_over_ranks(sum(r["steps_done"] for r in recs))
    completed = int(sum_over_ranks(summ.get("completed", 0)))
    failed = int(sum_over_ranks(summ.get("failed", 0)))
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    out = {"metric": "batched sweep: aggregate Newton iterations per second", "value": newton / span,
           "unit": "Newton it/s", "n_gpus": world, "higher_is_better": True, "mode": "sweep", "data": "synthetic",
           "dtype": "f32-inner/f64-refinement" if args.precision == "mixed" else "f64",
           "config": {"workload": f"{len(wls_all)} KGD instances, 1k-50k P2 triangles, {args.sweep_steps} steps each "
                                  f"(rank 0 ran {len(wls)}; instances split across {world} ranks by cost)",
                      "slots": args.slots, "autotuned": bool(args.autotune)},
           "makespan_s": span, "instance_steps_per_s": steps_done / span,
           "completed": completed, "failed": failed,
           "peak_running": st["peak_running"], "autotune_s": t_tune,
           "tuned": tuner.report() if tuner else None, "clocks": clocks}
    print(json.dumps(out))


def run_reference(args):
    """The reference arm: the FP64 oracle itself, one full Newton iteration
    of the penny workload per step at a size that keeps the whole run within
    a few minutes (stated in the line)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_baseline(args.cpu_n)
    vals = [oracle_baseline(args.cpu_n) for _ in range(args.ref_steps)]
    base = vals[-1]
    value = len(vals) / sum(1.0 / v["value"] for v in vals)
    base["value"] = value
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(vals),
           "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
           "data": "synthetic (seeded structured P2 mesh and seed crack)",
           "config": {"workload": workload(args.config).name, "precision": "fp64 oracle",
                      "oracle_workload": f"penny n = {args.cpu_n} (a bounded sample: the 1.05 M-unknown workload "
                                         f"takes the oracle over 10 minutes per Newton iteration)"},
           "cpu_baseline": base,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    ap.add_argument("--restart", type=int, default=HEADLINE["mixed"]["restart"])
    ap.add_argument("--reorth", type=int, default=HEADLINE["mixed"]["reorth"])
    ap.add_argument("--fp64-restart", dest="fp64_restart", type=int, default=HEADLINE["fp64"]["restart"])
    ap.add_argument("--fp64-reorth", dest="fp64_reorth", type=int, default=HEADLINE["fp64"]["reorth"])
    ap.add_argument("--max-iters", dest="max_iters", type=int, default=8000)
    ap.add_argument("--coarse", type=int, default=1)
    ap.add_argument("--graphs", type=int, default=1)
    ap.add_argument("--fp64-steps", dest="fp64_steps", type=int, default=-1, help="-1: as many as --steps")
    ap.add_argument("--e2e", type=int, default=1)
    ap.add_argument("--rtol", type=float, default=HEADLINE["mixed"]["rtol"],
                    help="GMRES relative residual of the mixed path")
    ap.add_argument("--fp64-rtol", dest="fp64_rtol", type=float, default=HEADLINE["fp64"]["rtol"])
    ap.add_argument("--inner-rtol", dest="inner_rtol", type=float, default=HEADLINE["mixed"]["inner_rtol"])
    ap.add_argument("--cpu-n", dest="cpu_n", type=int, default=6, help="penny mesh size of the oracle baseline")
    ap.add_argument("--ref-steps", dest="ref_steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--mode", default="newton", choices=["newton", "serve", "sweep"])
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-requests", dest="serve_requests", type=int, default=0)
    ap.add_argument("--serve-sample", dest="serve_sample", type=int, default=12,
                    help="requests of the bounded serving sample in the default line (0: none)")
    ap.add_argument("--serve-rate", dest="serve_rate", type=float, default=200.0)
    ap.add_argument("--serve-steps", dest="serve_steps", type=int, default=5)
    ap.add_argument("--sweep-count", dest="sweep_count", type=int, default=256)
    ap.add_argument("--sweep-steps", dest="sweep_steps", type=int, default=10)
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--verbose", type=int, default=0)
    ap.add_argument("--request-max-iters", dest="request_max_iters", type=int, default=3000)
    args = ap.parse_args()
    if args.fp64_steps < 0:
        args.fp64_steps = args.steps
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
