"""Configuration c1 (2D KGD, 44 x 44 squares of two P2 triangles: 3,872
elements, 46,553 unknowns; E = 20 GPa, K_Ic = 1 MPa sqrt(m), mu = 1e-3 Pa s,
Q0 = 1e-3 m^2/s; crack on the midline; pressure cut-off on; Newton to 1e-10;
FP64): ten time steps of hf_advance_step against the oracle's ten steps under
the same driving rules (tests/golden/c1_steps_oracle.json, written by
tests/golden/make_c1_steps.py from the oracle and the input generator only).

Per step: the same cutbacks and sub-steps, the same cohesive and fluid facets,
and U on a fixed sample, every non-zero pressure and the openings at the face
nodes of every cohesive or fluid facet within 1e-9 of the oracle (each over
the infinity norm of the oracle's field)."""
import json
import os

import numpy as np
import pytest

from hf_inputs import c1_kgd_toughness

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_steps_oracle.json")


def test_c1_ten_time_steps_match_oracle():
    if not os.path.exists(GOLDEN):
        pytest.skip("c1 oracle steps not generated")
    from paper_1911_10275_gb300 import HFMesh
    gold = json.load(open(GOLDEN))
    wl = c1_kgd_toughness()
    g = HFMesh.from_mesh(wl.mesh)
    inj, wts = wl.injection()
    g.hf_set_material(wl.E, wl.nu, wl.sigma_c, wl.delta_c, wl.b_stab)
    g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, wl.dt, 0.0, True, wl.fluid_length)
    g.hf_set_solver(precision="fp64", rtol=1e-13, max_iters=20000, jacobi_block=16, newton_tol=1e-10)
    g.hf_set_state(*wl.seed())
    u_idx = np.asarray(gold["u_index"], dtype=np.int64)
    for rec in gold["steps"]:
        rep = g.hf_advance_step()
        assert (rep["cutbacks"], rep["substeps"]) == (rec["cutbacks"], rec["substeps"]), (rec["k"], rep)
        U, P, a, b, _, t = g.hf_get_state()
        assert t == pytest.approx(rec["t"], abs=1e-12)
        assert sorted(np.nonzero(a)[0].tolist()) == rec["alpha_faces"]
        assert sorted(np.nonzero(b)[0].tolist()) == rec["beta_faces"]
        W = g.hf_get_opening_pressure()[0]
        eu = np.abs(U[u_idx] - np.asarray(rec["U"])).max() / rec["U_inf"]
        pi = np.asarray(rec["P_index"], dtype=np.int64)
        ep = np.abs(P[pi] - np.asarray(rec["P"])).max() / rec["P_inf"]
        wf = np.asarray(rec["w_faces"], dtype=np.int64)
        ew = np.abs(W[wf] - np.asarray(rec["w"])).max() / rec["w_inf"]
        assert max(eu, ep, ew) <= 1e-9, (rec["k"], eu, ep, ew)
    g.close()
