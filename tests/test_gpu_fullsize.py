"""Parity at the size and in the launch configuration that bench.py times:
the 1.05M-unknown penny workload (34,992 P2 tetrahedra), FP32 inner solves
inside FP64 refinement, 32-element subdomains, CUDA-graph GMRES cycles.  The
oracle cannot assemble the whole system within a test, so it computes sampled
rows (elements next to the crack plus random ones, active and random pressure
unknowns) with its sampled assembly, whose rows are pinned equal to the
global assembly on small meshes."""
import numpy as np
import pytest

from hf_inputs import c3_penny
from _setup import oracle_for, gpu_for, with_extra_cohesive

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    wl = c3_penny()
    state, picked = with_extra_cohesive(wl, wl.seed(), count=4)
    o = oracle_for(wl)
    o.set_state(*state)
    g = gpu_for(wl, precision="mixed", jacobi_block=32, rtol=1e-8, inner_rtol=1e-3, use_graphs=1,
                max_iters=3000, newton_tol=1e-8)
    g.hf_set_state(*state)
    rng = np.random.default_rng(2024)
    m = wl.mesh
    nl_faces = np.nonzero(m.face_crackable & ((o.alpha > 0) | (o.beta > 0)))[0]
    crack_elems = np.unique(m.face_elems[nl_faces].ravel())
    elems = np.unique(np.concatenate([crack_elems[:24], rng.choice(o.ne, 40, replace=False)]))
    # every active pressure row (the injection row among them: its size sets
    # the scale of the pressure block, as in the small-mesh comparisons) and
    # a few inactive ones
    act = np.nonzero(o.active_pdofs())[0]
    pd = np.unique(np.concatenate([act, rng.choice(o.Np, 8, replace=False)]))
    rows = np.concatenate([np.concatenate([o.udofs(e) for e in elems]), o.Nu + pd])
    yield wl, o, g, elems, pd, rows
    g.close()


def _block_err(a, b, rows, nu):
    out = []
    for sel in (rows < nu, rows >= nu):
        r = rows[sel]
        scale = np.abs(b[r]).max()
        out.append(np.abs(a[r] - b[r]).max() / (scale if scale > 0 else 1.0))
    return out


def test_fullsize_residual_rows(full):
    wl, o, g, elems, pd, rows = full
    Rg = g.hf_eval_residual()
    Ro, _ = o.assemble(with_jacobian=False, elems=elems, pdofs=pd)
    eu, ep = _block_err(Rg, Ro, rows, o.Nu)
    assert eu < 1e-12 and ep < 1e-12


def test_fullsize_jacobian_rows(full):
    wl, o, g, elems, pd, rows = full
    rng = np.random.default_rng(7)
    x = rng.standard_normal(o.N)
    x[o.Nu:] *= 1e6
    yg = g.hf_apply_jacobian(x)
    _, Js = o.assemble(elems=elems, pdofs=pd)
    yo = Js @ x
    eu, ep = _block_err(yg, yo, rows, o.Nu)
    assert eu < 1e-12 and ep < 1e-12


def test_fullsize_criterion_traction_sampled(full):
    wl, o, g, elems, pd, rows = full
    m = wl.mesh
    tg = g.hf_get_criterion_traction()
    cand = np.nonzero(m.face_crackable & (o.alpha == 0))[0]
    rng = np.random.default_rng(3)
    pick = rng.choice(cand, size=min(24, cand.size), replace=False)
    to = np.array([o.dg_normal_traction(f).max() for f in pick])
    assert np.abs(tg[pick] - to).max() <= 1e-10 * np.abs(to).max()


def test_fullsize_newton_increment_satisfies_linearised_rows(full):
    """One Newton step in the bench's configuration: GMRES reports a relative
    residual <= 1e-8, and the oracle's own sampled rows of J d + R agree."""
    wl, o, g, elems, pd, rows = full
    U0, P0 = g.hf_get_state()[:2]
    R0, J0 = o.assemble(elems=elems, pdofs=pd)
    rep = g.hf_newton_step()
    assert rep["lin_converged"] and rep["lin_res"] <= 1e-8
    U1, P1 = g.hf_get_state()[:2]
    d = np.concatenate([U1 - U0, P1 - P0])
    r = (J0 @ d + R0)[rows]
    assert np.abs(r).max() <= 1e-7 * rep["res_norm"]
