"""The coarse level of the preconditioner against its definition: the
difference between the two-level and the one-level preconditioner applied to
the same vector is the Galerkin correction Phi (Phi^T J Phi)^-1 Phi^T r, with
Phi the rigid-body modes of each aggregate (zero on Dirichlet rows), built
here in numpy from the mesh, the aggregate map and the oracle's tangent.  On
an uncracked state the oracle's displacement block is the linear part the
coarse level projects.  The correction does not depend on the basis chosen
for each aggregate's modes, so any centre and scale will do."""
import numpy as np
import pytest

from hf_inputs import kgd_2d, penny_3d
from _setup import oracle_for, gpu_for

pytestmark = pytest.mark.gpu


def _rbm_basis(mesh, agg):
    """Columns: per aggregate, translations and infinitesimal rotations about
    its centroid, on the displacement unknowns of its elements."""
    d, nen = mesh.dim, mesh.n_en
    ne = mesh.n_elems
    nm = 3 if d == 2 else 6
    nagg = agg.max() + 1
    Phi = np.zeros((ne * nen * d, nagg * nm))
    for g in range(nagg):
        els = np.nonzero(agg == g)[0]
        X = mesh.xyz[mesh.elem_nodes[els]]              # (k, nen, d)
        X = X - X.reshape(-1, d).mean(axis=0)
        rows = els[:, None] * nen * d + np.arange(nen)[None, :] * d   # first component of each node
        for k in range(d):
            Phi[(rows + k).ravel(), g * nm + k] = 1.0
        planes = [(0, 1)] if d == 2 else [(0, 1), (1, 2), (2, 0)]
        for q, (a, b) in enumerate(planes):
            c = g * nm + d + q
            Phi[(rows + a).ravel(), c] = -X[:, :, b].ravel()
            Phi[(rows + b).ravel(), c] = X[:, :, a].ravel()
    Phi[mesh.dir_dof] = 0.0
    return Phi


def _gpu_basis(mesh, agg, geo):
    """The library's own basis: modes about each aggregate's centre, scaled
    by its size (the layout hf_get_coarse_operator documents)."""
    d, nen = mesh.dim, mesh.n_en
    nm = 3 if d == 2 else 6
    Phi = np.zeros((mesh.n_elems * nen * d, geo.shape[0] * nm))
    e = np.arange(mesh.n_elems)
    X = (mesh.xyz[mesh.elem_nodes] - geo[agg][:, None, :d]) / geo[agg][:, None, 3:4]
    rows = e[:, None] * nen * d + np.arange(nen)[None, :] * d
    cols = agg[:, None] * nm + np.zeros((1, nen), dtype=int)
    for k in range(d):
        Phi[(rows + k).ravel(), (cols + k).ravel()] = 1.0
    planes = [(0, 1)] if d == 2 else [(0, 1), (1, 2), (2, 0)]
    for q, (a, b) in enumerate(planes):
        Phi[(rows + a).ravel(), (cols + d + q).ravel()] = -X[:, :, b].ravel()
        Phi[(rows + b).ravel(), (cols + d + q).ravel()] = X[:, :, a].ravel()
    Phi[mesh.dir_dof] = 0.0
    return Phi


CASES = [lambda: kgd_2d(n=10, length=20.0), lambda: penny_3d(n=4, crackable="plane")]


@pytest.mark.parametrize("make,coarse_max", [(CASES[0], 64), (CASES[1], 64), (CASES[1], 260)])
def test_coarse_operator_is_phi_t_j_phi(make, coarse_max):
    """A0 as built on the GPU equals Phi^T J Phi in the library's basis, and
    the stored inverse inverts it (258 coarse unknowns at 260: several pivot
    blocks of the blocked inversion, a ragged last block and several tiles)."""
    wl = make()
    m = wl.mesh
    U, P, al, be = wl.seed()
    state = (np.zeros_like(U), np.zeros_like(P), np.zeros_like(al), np.zeros_like(be))
    o = oracle_for(wl)
    o.set_state(*state)
    _, J = o.assemble()
    Juu = J.tocsr()[:o.Nu, :o.Nu]
    g = gpu_for(wl, precision="fp64", jacobi_block=8, coarse=1, coarse_max=coarse_max)
    g.hf_set_state(*state)
    agg = g.hf_get_aggregates()
    A0g, invg, geo = g.hf_get_coarse_operator()
    g.close()
    Phi = _gpu_basis(m, agg, geo)
    A0 = Phi.T @ (Juu @ Phi)
    if coarse_max > 64:
        assert A0.shape[0] > 2 * 64 and A0.shape[0] % 32 != 0, A0.shape
    assert np.abs(A0g - A0).max() <= 1e-12 * np.abs(A0).max()
    assert np.abs(invg @ A0 - np.eye(A0.shape[0])).max() <= 1e-9


@pytest.mark.parametrize("make", CASES)
def test_coarse_correction_is_the_galerkin_projection(make):
    wl = make()
    m = wl.mesh
    U, P, al, be = wl.seed()
    state = (np.zeros_like(U), np.zeros_like(P), np.zeros_like(al), np.zeros_like(be))
    o = oracle_for(wl)
    o.set_state(*state)
    _, J = o.assemble()
    nu = o.Nu
    Juu = J.tocsr()[:nu, :nu]
    g = gpu_for(wl, precision="fp64", jacobi_block=8, coarse=1, coarse_max=64)
    g.hf_set_state(*state)
    agg = g.hf_get_aggregates()
    assert g.hf_get_stats()["coarse_unknowns"] == (agg.max() + 1) * (3 if m.dim == 2 else 6)
    rng = np.random.default_rng(11)
    r = np.zeros(o.N)
    r[:nu] = rng.standard_normal(nu)
    # Dirichlet rows are identity rows whose columns stay in J: an O(1) entry
    # there gives O(1) preconditioner output in its element, and the O(1e-11)
    # coarse part would drown in its rounding.  Newton residuals vanish there.
    r[m.dir_dof] = 0.0
    z2 = g.hf_apply_preconditioner(r)
    g.hf_set_solver(precision="fp64", jacobi_block=8, coarse=0, coarse_max=64, rtol=1e-13, max_iters=20000)
    z1 = g.hf_apply_preconditioner(r)
    g.close()
    Phi = _rbm_basis(m, agg)
    A0 = Phi.T @ (Juu @ Phi)
    want = Phi @ np.linalg.solve(A0, Phi.T @ r[:nu])
    got = (z2 - z1)[:nu]
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_coarse_level_cuts_gmres_iterations():
    """Same Newton iteration, same tolerance, one- and two-level: the answer
    agrees to the tolerance and the two-level solve takes fewer iterations."""
    wl = kgd_2d(n=24, length=100.0)
    state = wl.seed()
    reps, states = [], []
    for coarse in (0, 1):
        g = gpu_for(wl, precision="mixed", rtol=1e-8, inner_rtol=1e-3, max_iters=20000, jacobi_block=16,
                    coarse=coarse, restart=30)
        g.hf_set_state(*state)
        reps.append(g.hf_newton_step())
        states.append(g.hf_get_state())
        g.close()
    assert all(r["lin_converged"] for r in reps)
    assert reps[1]["gmres_iters"] < reps[0]["gmres_iters"]
    # a relative residual of 1e-8 bounds the error only through the condition
    # number of J (force, flux and identity rows together): two solves that
    # both meet it agree to ~1e-5 in the displacements here
    U0, U1 = states[0][0], states[1][0]
    assert np.abs(U1 - U0).max() <= 1e-4 * np.abs(U0).max()
