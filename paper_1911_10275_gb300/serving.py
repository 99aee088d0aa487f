"""Client side of the request loop (hf_runtime_* in include/hf.h): turns
workloads into requests, submits them at their arrival times and gathers
per-request latency.  The scheduling, admission and all device work happen
in the native runtime; this module only marshals requests and reads clocks."""
from __future__ import annotations

import time

import numpy as np


def request_args(wl, state=None, t0=0.0):
    """Keyword arguments of HFRuntime.submit for a workload (mesh, material,
    point injection at the centre, seed state unless `state` is given)."""
    inj, wts = wl.injection()
    U, P, al, be = state if state is not None else wl.seed()
    return dict(E=wl.E, nu=wl.nu, sigma_c=wl.sigma_c, delta_c=wl.delta_c, b_stab=wl.b_stab, mu=wl.mu, Q0=wl.Q0,
                inj_dofs=inj, inj_weights=wts, delta_f=wl.delta_f, dt=wl.dt, p_vapor=0.0, cutoff_on=True,
                L_ref=getattr(wl, "fluid_length", wl.mesh.length), U0=U, P0=P, alpha0=al, beta0=be, t0=t0)


def submit_workload(rt, wl, n_steps, solver=None, step=None, state=None):
    return rt.submit(wl.mesh, n_steps=n_steps, solver=solver, step=step, **request_args(wl, state))


def run_stream(rt, arrivals, workloads, n_steps, solver_for, step=None, fetch=False, state_for=None):
    """Submit workloads[i] at runtime clock arrivals[i] (seconds from now),
    wait for all, and return one record per request: the hf_result fields
    plus 'latency' (done - submit) and 'queue' (admit - submit); with fetch,
    also the final state.  solver_for(wl) gives each request's solver
    options."""
    base = rt.now()
    ids = []
    for t, wl in zip(arrivals, workloads):
        delay = base + float(t) - rt.now()
        if delay > 0:
            time.sleep(delay)
        st = state_for(wl) if state_for else None
        ids.append(submit_workload(rt, wl, n_steps, solver=solver_for(wl), step=step, state=st))
    out = []
    for rid, wl in zip(ids, workloads):
        r = rt.wait(rid)
        r["name"] = wl.name
        r["latency"] = r["t_done"] - r["t_submit"]
        r["queue"] = r["t_admit"] - r["t_submit"] if r["t_admit"] > 0 else None
        if fetch:
            r["state"] = rt.fetch(rid, r)
        else:
            rt.fetch(rid, r)
        out.append(r)
    return out


def latency_summary(records):
    """p50 / p99 / max latency in ms over successful requests, throughput in
    requests/s over the span from the first submit to the last completion."""
    ok = [r for r in records if r["status"] == 0]
    failures = [{"name": r.get("name"), "status": int(r["status"]), "newton_iters": int(r["newton_iters"]),
                 "cutbacks": int(r["cutbacks"]), "steps_done": int(r.get("steps_done", -1))}
                for r in records if r["status"] != 0]
    if not ok:
        return {"completed": 0, "failed": len(records), "failures": failures}
    lat = np.array([r["latency"] for r in ok]) * 1000.0
    span = max(r["t_done"] for r in records) - min(r["t_submit"] for r in records)
    return {"completed": len(ok), "failed": len(records) - len(ok),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "mean_ms": float(lat.mean()),
            "throughput_req_s": len(ok) / span if span > 0 else None,
            "newton_iters": int(sum(r["newton_iters"] for r in ok)),
            "gmres_iters": int(sum(r["gmres_iters"] for r in ok)),
            "cutbacks": int(sum(r["cutbacks"] for r in ok)), "failures": failures}
