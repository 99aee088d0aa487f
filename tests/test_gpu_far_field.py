"""Far-field stress (the outer load of the propagation test, Sec. 4.2): a
compressive stress sigma0 normal to the crack applied as the traction
-sigma0 n on the outer face parallel to the crack (hf_mesh_desc Neumann
facets, Eq. elastostatics with t on the Neumann boundary).

Pins: (i) the GPU step matches the oracle's with the same traction facets;
(ii) superposition, exact for the linear elastic problem because the
uniform stress field is reproduced exactly by the discretisation (patch
test): a traction-free crack held at pressure p under the far field opens
exactly as the same crack held at p - sigma0 with no far field.  The crack
pressures are held by essential pressure rows (hf_set_fixed_pressure), the
cohesive law is spent (delta_c tiny), so the crack lips carry only the fluid
pressure."""
import numpy as np
import pytest

from hf_inputs import kgd_2d, penny_3d, far_field_load, pressure_nodes
from oracle import Oracle, Params
from _setup import rel_err

pytestmark = pytest.mark.gpu


def _setup(wl, sigma0, p):
    m, nf, tr = far_field_load(wl.mesh, sigma0)
    pn = pressure_nodes(m)
    U, P, al, be = wl.seed()     # the seed opening is past delta_c: the lips carry no cohesive traction
    fixed = np.arange(pn.size)
    vals = np.full(pn.size, p)
    return m, nf, tr, (U, vals.copy(), al, be), fixed, vals


def _gpu(wl, m, nf, tr, state, fixed, vals):
    from paper_1911_10275_gb300 import HFMesh
    g = HFMesh.from_mesh(m, neu_face=nf, neu_traction=tr.ravel())
    inj, wts = wl.injection()
    g.hf_set_material(wl.E, wl.nu, 1e6, 1e-12, 10.0)
    g.hf_set_injection(wl.mu, 0.0, inj, wts, 1e-12, 1.0, 0.0, False, wl.fluid_length)
    g.hf_set_solver(precision="fp64", rtol=1e-13, max_iters=20000, jacobi_block=16, newton_tol=1e-10)
    g.hf_set_fixed_pressure(fixed, vals)
    g.hf_set_state(*state)
    for _ in range(6):
        r = g.hf_newton_step()
        if r["converged"]:
            break
    assert r["converged"]
    return g


@pytest.mark.parametrize("dim", [2, 3])
def test_far_field_superposition_and_parity(dim):
    wl = kgd_2d(n=12, length=24.0, crackable="midline", seed_cells=3) if dim == 2 else \
        penny_3d(n=6, length=24.0, crackable="plane", seed_cells=2)
    sigma0, p = 2e6, 5e6
    m, nf, tr, state, fixed, vals = _setup(wl, sigma0, p)
    ga = _gpu(wl, m, nf, tr, state, fixed, vals)
    wa = ga.hf_get_opening_pressure()[0]
    Ua = ga.hf_get_state()[0]
    m0, nf0, tr0, state0, _, vals0 = _setup(wl, 0.0, p - sigma0)
    gb = _gpu(wl, m0, nf0, tr0, state0, fixed, vals0)
    wb = gb.hf_get_opening_pressure()[0]
    crack = np.nonzero(m.face_crackable & (state[2] > 0))[0]
    assert np.abs(wa[crack]).max() > 0.0
    assert rel_err(wa[crack], wb[crack]) <= 1e-9
    # the oracle with the same traction facets and held pressures
    inj, wts = wl.injection()
    prm = Params(E=wl.E, nu=wl.nu, sigma_c=1e6, delta_c=1e-12, b_stab=10.0, mu=wl.mu, Q0=0.0,
                 inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=1e-12, dt=1.0, L_ref=wl.fluid_length,
                 newton_tol=1e-10, fixed_pdofs=tuple(int(i) for i in fixed), fixed_pvals=tuple(vals))
    o = Oracle(m, prm, neu_faces=nf, neu_traction=tr)
    o.set_state(*state)
    for _ in range(6):
        if o.newton_step()["converged"]:
            break
    assert rel_err(Ua, o.U) <= 1e-9
    assert rel_err(wa[crack], o.opening_at_face_nodes(o.U)[crack]) <= 1e-9
    ga.close()
    gb.close()
