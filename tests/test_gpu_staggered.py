"""The staggered scheme of Sec. 4.3 ("Fully-coupled vs. staggered
hydro-mechanics with applied inflow boundary conditions") on the GPU:
hf_newton_step with scheme HF_SCHEME_STAGGERED solves the mechanical block
A dU = -R_u at the old pressure, then the lubrication block D dP = -R_p at the
new opening, with the fictitious essential pressure hf_set_fixed_pressure
imposes.  Parity: the first two staggered iterations agree with the oracle's
(oracle.Oracle.staggered_step) to 1e-9.  Behaviour: on the given-length KGD
crack with the injection rate imposed the fully-coupled iteration converges
while the staggered one does not, as the paper reports."""
import numpy as np
import pytest

from _setup import rel_err
from test_oracle_pins import _given_length_kgd, _given_length_oracle

pytestmark = pytest.mark.gpu


def _gpu(wl, fixed, scheme, rtol=1e-13):
    from paper_1911_10275_gb300 import HFMesh
    g = HFMesh.from_mesh(wl.mesh)
    inj, wts = wl.injection()
    g.hf_set_material(wl.E, wl.nu, wl.sigma_c, wl.delta_c, 10.0)
    g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, 1.0, 0.0, False, wl.fluid_length)
    g.hf_set_solver(precision="fp64", rtol=rtol, max_iters=20000, jacobi_block=16, scheme=scheme, newton_tol=1e-10)
    if fixed:
        g.hf_set_fixed_pressure(fixed, np.zeros(len(fixed)))
    g.hf_set_state(*wl.seed())
    return g


def test_staggered_iterations_match_oracle():
    wl, fixed = _given_length_kgd(n=8, L=16.0, ell=4.0)
    o = _given_length_oracle(wl, fixed)
    g = _gpu(wl, fixed, "staggered")
    for it in range(2):
        rg = g.hf_newton_step()
        ro = o.staggered_step()
        U, P = g.hf_get_state()[:2]
        assert rg["lin_converged"], rg
        assert rel_err(U, o.U) <= 1e-9
        assert rel_err(P, o.P) <= 1e-9
        assert rg["du_rel"] == pytest.approx(ro["du_rel"], rel=1e-7)
        assert rg["dp_rel"] == pytest.approx(ro["dp_rel"], rel=1e-7)
        # an identity row, met to the GMRES tolerance
        assert np.abs(P[fixed]).max() <= 1e-9 * np.abs(P).max()
    g.close()


def test_fixed_pressure_holds_in_the_coupled_scheme():
    """The essential pressure is an identity row in the coupled system too:
    a coupled Newton step keeps it and matches the oracle with the same
    condition."""
    wl, fixed = _given_length_kgd(n=8, L=16.0, ell=4.0)
    o = _given_length_oracle(wl, fixed)
    g = _gpu(wl, fixed, "coupled")
    g.hf_newton_step()
    o.newton_step()
    U, P = g.hf_get_state()[:2]
    assert rel_err(U, o.U) <= 1e-9 and rel_err(P, o.P) <= 1e-9
    assert np.abs(P[fixed]).max() <= 1e-9 * np.abs(P).max()
    g.close()


def test_staggered_diverges_where_coupled_converges():
    from paper_1911_10275_gb300 import HFError
    wl, fixed = _given_length_kgd(n=24, L=48.0, ell=6.0)
    g = _gpu(wl, [], "coupled", rtol=1e-12)
    for it in range(10):
        r = g.hf_newton_step()
        if r["converged"]:
            break
    assert r["converged"] and it <= 7
    g.close()
    g = _gpu(wl, fixed, "staggered", rtol=1e-12)
    dps, ok = [], True
    for it in range(12):
        try:
            r = g.hf_newton_step()
        except HFError:
            ok = False
            break
        dps.append(r["dp_rel"])
        if r["converged"] or not r["lin_converged"] or not np.isfinite(r["dp_rel"]):
            ok = r["converged"]
            break
    assert not ok or not r["converged"]
    assert len(dps) < 2 or dps[1] > dps[0] or min(dps) > 0.1
    g.close()
