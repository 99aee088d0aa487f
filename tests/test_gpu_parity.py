"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU
oracle on the same seeded inputs.  Small meshes spanning several subdomains
and ragged tails, in 2D and 3D, in all three facet states.

Tolerances: the residual and J x are sums of the same terms in a different
order and blocking, so they agree to a few hundred ulps of the largest term
(1e-12 relative to the block maximum).  A Newton step additionally goes
through GMRES solved to 1e-13 against the oracle's direct LU: 1e-10 relative
(FP64) and 1e-8 (mixed: FP32 inner solves inside FP64 refinement)."""
import numpy as np
import pytest

from hf_inputs import kgd_2d, penny_3d
from _setup import oracle_for, gpu_for, with_extra_cohesive, rel_err

pytestmark = pytest.mark.gpu


def cases():
    return {
        "2d_midline": kgd_2d(n=6, length=12.0, steps=1, seed_cells=2),
        "2d_all": kgd_2d(n=6, length=12.0, crackable="all", steps=1, seed_cells=2),
        "3d_plane": penny_3d(n=2, length=8.0, crackable="plane", steps=1, seed_cells=1),
        "3d_all": penny_3d(n=4, length=8.0, crackable="all", steps=1, seed_cells=1),
    }


def _pair(wl, extra=1, **solver):
    state, picked = with_extra_cohesive(wl, wl.seed(), count=extra)
    o = oracle_for(wl)
    o.set_state(*state)
    g = gpu_for(wl, **solver)
    g.hf_set_state(*state)
    return o, g, state


@pytest.mark.parametrize("name", ["2d_midline", "2d_all", "3d_plane", "3d_all"])
def test_residual_parity(name):
    wl = cases()[name]
    o, g, _ = _pair(wl)
    Ro, _ = o.assemble(with_jacobian=False)
    Rg = g.hf_eval_residual()
    nu = o.Nu
    assert rel_err(Rg[:nu], Ro[:nu]) < 1e-12
    assert rel_err(Rg[nu:], Ro[nu:]) < 1e-12
    g.close()


@pytest.mark.parametrize("name", ["2d_midline", "2d_all", "3d_plane", "3d_all"])
def test_jacobian_apply_parity(name):
    wl = cases()[name]
    o, g, _ = _pair(wl)
    _, J = o.assemble()
    rng = np.random.default_rng(3)
    for _ in range(2):
        x = rng.standard_normal(o.N)
        x[o.Nu:] *= 1e6          # pressures are O(MPa), displacements O(1)
        yo = J @ x
        yg = g.hf_apply_jacobian(x)
        assert rel_err(yg[: o.Nu], yo[: o.Nu]) < 1e-12
        assert rel_err(yg[o.Nu:], yo[o.Nu:]) < 1e-12
    g.close()


@pytest.mark.parametrize("name", ["2d_all", "3d_all"])
def test_criterion_traction_parity(name):
    wl = cases()[name]
    o, g, _ = _pair(wl)
    # a state with real stresses: one Newton step of the oracle
    o.newton_step()
    g.hf_set_state(o.U, o.P, o.alpha, o.beta, w_old=o.w_old)
    tg = g.hf_get_criterion_traction()
    cr = np.nonzero(wl.mesh.face_crackable & (o.alpha == 0))[0]
    to = np.array([o.dg_normal_traction(f).max() for f in cr])
    assert rel_err(tg[cr], to) < 1e-10
    g.close()


@pytest.mark.parametrize("name,prec,tol,graphs", [("2d_midline", "fp64", 1e-10, 0), ("2d_all", "fp64", 1e-10, 0),
                                                  ("3d_plane", "fp64", 1e-10, 0), ("3d_all", "fp64", 1e-10, 0),
                                                  ("2d_midline", "mixed", 1e-8, 0), ("3d_all", "mixed", 1e-8, 0),
                                                  ("3d_all", "fp64", 1e-10, 1), ("3d_all", "mixed", 1e-8, 1)])
def test_newton_step_parity(name, prec, tol, graphs):
    wl = cases()[name]
    o, g, _ = _pair(wl, precision=prec, rtol=1e-13 if prec == "fp64" else 1e-11, use_graphs=graphs)
    rep = g.hf_newton_step()
    o.newton_step()
    Ug, Pg = g.hf_get_state()[:2]
    assert rep["lin_converged"], rep
    assert rel_err(Ug, o.U) < tol
    assert rel_err(Pg, o.P) < tol
    g.close()


def test_time_step_parity_2d():
    """Newton to convergence, criterion, end of step: openings, pressures and
    facet states agree with the oracle after two time steps."""
    wl = kgd_2d(n=8, length=16.0, steps=2, seed_cells=2)
    state = wl.seed()
    o = oracle_for(wl)
    o.set_state(*state)
    g = gpu_for(wl)
    g.hf_set_state(*state)
    for step in range(2):
        for it in range(10):
            rg = g.hf_newton_step()
            ro = o.newton_step()
            if ro["converged"]:
                break
        assert rg["converged"]
        ng = g.hf_check_fracture_criterion()
        no, _ = o.check_fracture_criterion()
        assert ng == no
        bg = g.hf_accept_step()
        bo = o.accept_step()
        assert bg == bo
        w, p, a, b = g.hf_get_opening_pressure()
        assert np.array_equal(a, o.alpha) and np.array_equal(b, o.beta)
        assert rel_err(w, o.opening_at_face_nodes(o.U)) < 1e-9
        assert rel_err(p, o.P) < 1e-9
    g.close()


@pytest.mark.parametrize("name", ["2d_all", "3d_all"])
def test_block_diagonal_preconditioner_is_exact_on_its_blocks(name):
    """With one element per subdomain the preconditioner is the inverse of the
    element diagonal blocks: for x supported on non-adjacent elements,
    M^-1 (J x) returns x on those elements."""
    wl = cases()[name]
    o, g, _ = _pair(wl, jacobi_block=1, coarse=0)
    m = wl.mesh
    nen, d = m.n_en, m.dim
    ned = nen * d
    # greedy independent set of elements
    nb = {e: set() for e in range(m.n_elems)}
    for em, ep in m.face_elems:
        if ep >= 0:
            nb[int(em)].add(int(ep))
            nb[int(ep)].add(int(em))
    chosen, blocked = [], set()
    for e in range(m.n_elems):
        if e not in blocked:
            chosen.append(e)
            blocked |= nb[e] | {e}
    rng = np.random.default_rng(5)
    x = np.zeros(o.N)
    for e in chosen:
        x[e * ned:(e + 1) * ned] = rng.standard_normal(ned)
    z = g.hf_apply_preconditioner(g.hf_apply_jacobian(x))
    idx = np.concatenate([np.arange(e * ned, (e + 1) * ned) for e in chosen])
    assert rel_err(z[idx], x[idx]) < 1e-9
    g.close()


@pytest.mark.parametrize("block", [1, 4, 64])
def test_linear_solve_independent_of_subdomain_size(block):
    wl = cases()["3d_all"]
    o, g, _ = _pair(wl, jacobi_block=block)
    R, J = o.assemble()
    xo = o.solve_linear(J, -R)
    xg, rep = g.hf_solve_linear(-R)
    assert rep["lin_converged"]
    assert rel_err(xg[: o.Nu], xo[: o.Nu]) < 1e-9
    assert rel_err(xg[o.Nu:], xo[o.Nu:]) < 1e-9
    g.close()
