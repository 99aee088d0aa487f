"""The native time-step driver (hf_advance_step) against the oracle's time
loop, its cutback path, the device-memory bound, and the request loop
(hf_runtime_*): admission by budget, and every result the same alone and in
a mix of concurrent requests."""
import dataclasses

import numpy as np
import pytest

from hf_inputs import kgd_2d, penny_3d, balanced_fluid_length
from _setup import oracle_for, gpu_for, rel_err, oracle_advance_step

pytestmark = pytest.mark.gpu


def test_advance_step_matches_oracle_time_loop():
    """Three time steps of the small KGD problem; the second needs cutbacks
    (Newton does not converge with the full step), the others do not.  The
    driver's decisions (Newton iterations, cutbacks, sub-steps, facet
    switches) and the state after each step agree with the oracle."""
    wl = kgd_2d(n=8, length=16.0, steps=3, seed_cells=2)
    state = wl.seed()
    o = oracle_for(wl)
    o.set_state(*state)
    g = gpu_for(wl)
    g.hf_set_state(*state)
    cut = 0
    for step in range(3):
        rep = g.hf_advance_step()
        ro = oracle_advance_step(o)
        # a failed attempt may end earlier on the GPU (its GMRES stops short of
        # the tolerance on a diverging iterate, where the oracle's direct
        # solve goes on), so Newton counts may differ; the decisions may not
        assert (rep["cutbacks"], rep["substeps"]) == (ro["cutbacks"], ro["substeps"])
        cut += rep["cutbacks"]
        w, p, a, b = g.hf_get_opening_pressure()
        assert np.array_equal(a, o.alpha) and np.array_equal(b, o.beta)
        assert rel_err(w, o.opening_at_face_nodes(o.U)) < 1e-9
        assert rel_err(p, o.P) < 1e-9
        assert abs(g.hf_get_state()[5] - (step + 1) * wl.dt) < 1e-12
    assert cut > 0
    g.close()


def test_failed_step_restores_the_start_of_step_state():
    """An attempt that cannot converge (one Newton iteration allowed) is undone
    on the device at every cutback; the handle then steps exactly like a fresh
    one."""
    from paper_1911_10275_gb300 import HFError
    wl = kgd_2d(n=8, length=16.0, steps=2, seed_cells=2)
    state = wl.seed()
    g = gpu_for(wl, precision="mixed", rtol=1e-10, inner_rtol=1e-3, use_graphs=1, newton_tol=1e-10)
    g.hf_set_state(*state)
    before = g.hf_get_state()
    with pytest.raises(HFError) as ei:
        g.hf_advance_step(newton_max=1, max_cutbacks=2)
    assert ei.value.status == -4
    after = g.hf_get_state()
    for x, y in zip(before[:5], after[:5]):
        assert np.array_equal(x, y)
    assert after[5] == before[5]
    rep = g.hf_advance_step()
    fresh = gpu_for(wl, precision="mixed", rtol=1e-10, inner_rtol=1e-3, use_graphs=1, newton_tol=1e-10)
    fresh.hf_set_state(*state)
    rep_f = fresh.hf_advance_step()
    assert rep["newton_iters"] == rep_f["newton_iters"]
    s1, s2 = g.hf_get_state(), fresh.hf_get_state()
    for x, y in zip(s1[:4], s2[:4]):
        assert rel_err(x, y) <= 1e-12
    g.close()
    fresh.close()


@pytest.mark.parametrize("make", [lambda: kgd_2d(n=10, length=20.0), lambda: penny_3d(n=4, crackable="plane")])
def test_device_bytes_within_estimate(make):
    from paper_1911_10275_gb300 import hf_estimate_device_bytes
    wl = make()
    g = gpu_for(wl, jacobi_block=16, precision="mixed", rtol=1e-8, inner_rtol=1e-3)
    g.hf_set_state(*wl.seed())
    g.hf_advance_step()
    used = g.hf_get_stats()["device_bytes"]
    est = hf_estimate_device_bytes(wl.mesh, jacobi_block=16)
    assert used <= est <= 1.02 * used + 4096
    g.close()


def _mix():
    """Uneven requests: 2D and 3D, FP64 and mixed precision, different
    materials, fluids and injection rates."""
    reqs = [
        (kgd_2d(n=12, length=24.0, E=20e9, K_Ic=1e6, mu=1e-3, Q0=1e-3), {"precision": "fp64", "rtol": 1e-10}),
        (kgd_2d(n=20, length=40.0, E=8e9, K_Ic=0.5e6, mu=1e-2, Q0=5e-4), {"precision": "mixed"}),
        (penny_3d(n=4, crackable="plane"), {"precision": "mixed"}),
        (kgd_2d(n=16, length=30.0, E=30e9, K_Ic=2e6, mu=1e-1, Q0=2e-3), {"precision": "mixed", "use_graphs": 1}),
        (penny_3d(n=6, crackable="plane", E=20e9, mu=1e-1), {"precision": "fp64", "rtol": 1e-10}),
        (kgd_2d(n=10, length=20.0, E=15e9, K_Ic=1.5e6), {"precision": "mixed", "jacobi_block": 8}),
    ]
    base = {"rtol": 1e-10, "inner_rtol": 1e-3, "max_iters": 5000, "jacobi_block": 16, "newton_tol": 1e-9}
    # fluid rows at the scale of the displacement rows (see balanced_fluid_length)
    return [(dataclasses.replace(wl, L_ref=balanced_fluid_length(wl)), {**base, **s}) for wl, s in reqs]


def _run(rt, reqs, steps=2):
    from paper_1911_10275_gb300.serving import submit_workload
    ids = [submit_workload(rt, wl, steps, solver=s) for wl, s in reqs]
    out = []
    for i in ids:
        r = rt.wait(i, timeout=300.0)
        assert r is not None
        out.append((r, rt.fetch(i, r)))
    return out


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_1911_10275_gb300 import HFRuntime
    reqs = _mix()
    alone = []
    rt = HFRuntime(slots=1)
    for wl, s in reqs:
        alone.append(_run(rt, [(wl, s)])[0])
    rt.close()
    rt = HFRuntime(slots=4)
    mixed = _run(rt, reqs)
    st = rt.stats()
    rt.close()
    assert st["peak_running"] >= 2  # requests did overlap
    for (ra, sa), (rm, sm) in zip(alone, mixed):
        assert ra["status"] == 0 and rm["status"] == 0, (ra, rm)
        assert ra["steps_done"] == rm["steps_done"] == 2
        assert ra["newton_iters"] == rm["newton_iters"]
        for x, y in zip(sa, sm):
            if x.dtype == np.int8:
                assert np.array_equal(x, y)
            else:
                assert rel_err(y, x) <= 1e-12


def test_admission_keeps_device_memory_within_budget():
    from paper_1911_10275_gb300 import HFRuntime, hf_estimate_device_bytes
    reqs = _mix()
    est = [hf_estimate_device_bytes(wl.mesh, **s) for wl, s in reqs]
    budget = int(2.2 * max(est))
    rt = HFRuntime(slots=4, hbm_budget_bytes=budget)
    res = _run(rt, reqs, steps=1)
    st = rt.stats()
    assert all(r["status"] == 0 for r, _ in res)
    assert st["peak_bytes"] <= budget and st["peak_running"] <= 4
    assert all(r["device_bytes"] <= r["estimate_bytes"] for r, _ in res)
    # a request larger than the whole budget is refused, not run
    small = HFRuntime(slots=1, hbm_budget_bytes=min(est) // 2)
    from paper_1911_10275_gb300.serving import submit_workload
    i = submit_workload(small, reqs[0][0], 1, solver=reqs[0][1])
    r = small.wait(i, timeout=10.0)
    assert r["status"] == -2 and r["steps_done"] == 0
    small.close()
    rt.close()


def test_mixed_solve_falls_back_to_fp64_when_fp32_stalls():
    """The mixed solve's hand-over to FP64: when two FP32 refinement sweeps in
    a row fail to halve the FP64 residual, the solve factors the subdomains in
    FP64 and finishes in FP64.  The stall is made certain rather than left to
    the conditioning of an instance: an inner tolerance of 1 asks the FP32
    sweeps for no reduction at all, so they leave the residual unchanged.  The
    solve must then reach its tolerance through the FP64 path and agree with
    the plain FP64 solve of the same system."""
    from hf_inputs import sweep_instances
    wl = sweep_instances(2)[1]
    states = []
    reps = []
    for prec, inner in (("mixed", 1.0), ("fp64", 1e-3)):
        g = gpu_for(wl, cutoff=True, precision=prec, rtol=1e-8, inner_rtol=inner, max_iters=3000, jacobi_block=16,
                    restart=60, use_graphs=1)
        g.hf_set_state(*wl.seed())
        reps.append(g.hf_newton_step())
        states.append(g.hf_get_state())
        g.close()
    assert reps[0]["lin_converged"] and reps[1]["lin_converged"]
    assert reps[0]["lin_res"] <= 1e-8 and reps[1]["lin_res"] <= 1e-8
    assert reps[0]["fp64_fallback"] == 1 and reps[1]["fp64_fallback"] == 0
    for x, y in zip(states[0][:2], states[1][:2]):
        assert rel_err(x, y) <= 1e-6


def test_bounded_device_wait_gives_up_with_timeout_status():
    """Failure detection without a fault: the preconditioner's bounded
    mbarrier wait, run on a barrier nothing completes, gives up after the
    host-set number of polls and the call returns HF_ERR_TIMEOUT; the handle
    stays usable (a Newton step afterwards converges its linear solve)."""
    from paper_1911_10275_gb300 import HFError
    wl = kgd_2d(n=6, length=12.0, steps=1, seed_cells=2)
    g = gpu_for(wl)
    g.hf_set_state(*wl.seed())
    g.hf_set_wait_limit(64)
    with pytest.raises(HFError) as err:
        g.hf_check_wait_timeout()
    assert err.value.status == -6
    with pytest.raises(HFError):
        g.hf_set_wait_limit(0)
    g.hf_set_wait_limit(1 << 22)
    rep = g.hf_newton_step()
    assert rep["lin_converged"]
    g.close()


def test_runtime_request_matches_oracle_time_loop():
    """One small request through the request loop (hf_runtime_*: copy-in,
    admission, hf_advance_step per step on a slot's stream, copy-out) ends
    where the oracle's time loop ends: three steps of the small KGD problem
    of test_advance_step_matches_oracle_time_loop (cutbacks in the second),
    facet states equal, U, pressures and face-node openings within 1e-9."""
    from paper_1911_10275_gb300 import HFRuntime
    from paper_1911_10275_gb300.serving import request_args
    wl = kgd_2d(n=8, length=16.0, steps=3, seed_cells=2)
    o = oracle_for(wl)
    o.set_state(*wl.seed())
    for _ in range(3):
        oracle_advance_step(o)
    rt = HFRuntime(slots=1)
    args = {**request_args(wl), "cutoff_on": False}
    rid = rt.submit(wl.mesh, n_steps=3, solver={"precision": "fp64", "rtol": 1e-13, "max_iters": 20000,
                                                "jacobi_block": 16}, **args)
    r = rt.wait(rid, timeout=300.0)
    assert r is not None and r["status"] == 0 and r["steps_done"] == 3, r
    U, P, a, b = rt.fetch(rid, r)
    rt.close()
    assert np.array_equal(a, o.alpha) and np.array_equal(b, o.beta)
    assert rel_err(U, o.U) < 1e-9
    assert rel_err(P, o.P) < 1e-9
    assert rel_err(o.opening_at_face_nodes(U), o.opening_at_face_nodes(o.U)) < 1e-9
