"""Accuracy of the timed configuration: the benchmark's exact solver
settings (bench.HEADLINE: FP32 inner sweeps inside FP64 refinement to a
relative residual of 1e-9, and plain FP64 GMRES to 1e-11; 32-element
subdomains, coarse level, CUDA-graph cycles, restart 60) driven by the
benchmark's own time loop from the seed state, compared iterate by iterate
with the FP64 oracle's trajectory of the same loop.  The oracle solved each
Newton system with its own ILU(0)-GMRES to 1e-13 (files written by
tests/golden/make_c3_newton.py, oracle and input generator only).

Per Newton iterate, over the infinity norm of the oracle's field: the
openings at the face nodes of every cohesive or fluid facet, every non-zero
pressure and a fixed sample of displacement unknowns all agree to 1e-8, the
accuracy the benchmark claims for both precisions."""
import json
import os

import numpy as np
import pytest

import bench
from hf_inputs import c3_penny, penny_3d

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-8


def _run(wl, prec, golden, max_iters):
    from paper_1911_10275_gb300 import HFMesh
    g = HFMesh.from_mesh(wl.mesh)
    inj, wts = wl.injection()
    g.hf_set_material(wl.E, wl.nu, wl.sigma_c, wl.delta_c, wl.b_stab)
    g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, wl.dt, 0.0, True, wl.fluid_length)
    g.hf_set_solver(**bench.HEADLINE[prec], **bench.COMMON)
    g.hf_set_state(*wl.seed())
    loop = bench.NewtonLoop(g, wl, rtol=bench.HEADLINE[prec]["rtol"])
    u_idx = np.asarray(golden["u_index"], dtype=np.int64)
    worst = {"U": 0.0, "P": 0.0, "w": 0.0}
    rows = []
    for rec in golden["iters"][:max_iters]:
        rep = loop.step()
        U, P = g.hf_get_state()[:2]
        W = g.hf_get_opening_pressure()[0]
        e = bench.errors_vs_golden(rec, u_idx, U, P, W)
        rows.append((rec["k"], rep["gmres_iters"], e))
        for k in worst:
            worst[k] = max(worst[k], e[k])
        # the loop takes the same decisions as the oracle's
        assert bool(rep["converged"]) == rec["converged"], (rec["k"], rep, rec["du_rel"])
    g.close()
    return worst, rows


def _golden(name):
    p = os.path.join(GOLDEN, name)
    if not os.path.exists(p):
        pytest.skip(f"{name} not generated")
    with open(p) as f:
        return json.load(f)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_penny_n8_trajectory_matches_oracle(prec):
    """93k unknowns, 8 Newton iterations (two time-step rounds with a
    fracture-criterion switch between them)."""
    wl = penny_3d(n=8, crackable="plane", name="penny3d_n8_plane")
    gold = _golden("penny8_newton_oracle.json")
    worst, rows = _run(wl, prec, gold, 8)
    assert max(worst.values()) <= TOL, rows


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_benchmark_workload_trajectory_matches_oracle(prec):
    """The 1.05M-unknown penny the benchmark times, along as many Newton
    iterations as the oracle's stored trajectory holds (up to 12)."""
    wl = c3_penny()
    gold = _golden("c3_newton_oracle.json")
    worst, rows = _run(wl, prec, gold, 12)
    assert max(worst.values()) <= TOL, rows
