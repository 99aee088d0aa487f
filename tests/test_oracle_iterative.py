"""Pins of the oracle's iterative solve (oracle/krylov.c via
oracle/iterative.py) against definitions and independent routes:

* ILU(0) reproduces A on its own sparsity pattern ((LU)_ij = a_ij there), the
  defining property of the incomplete factorisation, and is the exact LU when
  the pattern admits no fill (tridiagonal) or is dense;
* GMRES returns the solution numpy's dense solve gives;
* on the Newton systems of small KGD and penny meshes the iterative route and
  the oracle's direct LU agree to 1e-12, and both agree with an extended
  precision (40-digit) LU solve of the raw system."""
import numpy as np
import pytest
import scipy.sparse as sp

from hf_inputs import kgd_2d, penny_3d
from oracle.iterative import CSR, ILU0, gmres, solve_linear_iterative

from _setup import oracle_for, with_extra_cohesive, rel_err


def _factors(A):
    M = ILU0(CSR(A))
    Ac = CSR(A)
    F = sp.csr_matrix((M.lu, Ac.col, Ac.ptr), shape=A.shape)
    L = sp.tril(F, -1) + sp.eye(A.shape[0])
    U = sp.triu(F)
    return M, L, U


def test_ilu0_matches_matrix_on_its_pattern():
    rng = np.random.default_rng(4)
    n = 60
    A = sp.random(n, n, density=0.08, random_state=5, format="csr") + sp.diags(4.0 + rng.random(n))
    A = sp.csr_matrix(A)
    M, L, U = _factors(A)
    LU = (L @ U).tocsr()
    r, c = A.nonzero()
    assert np.allclose(np.asarray(LU[r, c]).ravel(), np.asarray(A[r, c]).ravel(), rtol=1e-13, atol=1e-13)
    # outside the pattern L U carries the dropped fill, so it is not A there
    assert abs(LU - A).max() > 1e-6


def test_ilu0_is_exact_lu_without_fill():
    rng = np.random.default_rng(6)
    n = 50
    T = sp.diags([rng.random(n - 1), 3.0 + rng.random(n), rng.random(n - 1)], [-1, 0, 1], format="csr")
    D = sp.csr_matrix(rng.random((12, 12)) + 12 * np.eye(12))
    for A in (T, D):
        M = ILU0(CSR(A))
        b = rng.standard_normal(A.shape[0])
        assert np.allclose(M.solve(b), np.linalg.solve(A.toarray(), b), rtol=1e-12, atol=1e-12)


def test_gmres_equals_dense_solve():
    rng = np.random.default_rng(8)
    n = 200
    A = sp.csr_matrix(sp.random(n, n, density=0.05, random_state=9) + sp.diags(2.0 + rng.random(n)))
    b = rng.standard_normal(n)
    x, its, res = gmres(CSR(A), ILU0(CSR(A)), b, restart=20, tol_abs=1e-14 * np.linalg.norm(b))
    assert res <= 1e-14 * np.linalg.norm(b)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-11, atol=1e-12)


CASES = {
    "kgd_all": lambda: kgd_2d(n=6, length=12.0, crackable="all", steps=1, seed_cells=2),
    "penny_all": lambda: penny_3d(n=4, length=8.0, crackable="all", steps=1, seed_cells=1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_iterative_solve_equals_direct_solve(name):
    wl = CASES[name]()
    state, _ = with_extra_cohesive(wl, wl.seed(), count=2)
    o = oracle_for(wl)
    o.set_state(*state)
    R, J = o.assemble()
    xd = o.solve_linear(J, -R)
    info = {}
    xi = solve_linear_iterative(J, -R, rtol=1e-13, info=info)
    assert info["rel_res"] <= 1e-13
    assert rel_err(xi[: o.Nu], xd[: o.Nu]) <= 1e-12
    assert rel_err(xi[o.Nu:], xd[o.Nu:]) <= 1e-12


def test_direct_and_iterative_solves_match_extended_precision():
    """Independent reference: a 40-digit LU solve (mpmath) of the raw,
    unequilibrated Newton system of a small KGD mesh."""
    mpmath = pytest.importorskip("mpmath")
    wl = kgd_2d(n=2, length=4.0, steps=1, seed_cells=1)
    o = oracle_for(wl)
    o.set_state(*wl.seed())
    assert o.beta.sum() >= 1
    R, J = o.assemble()
    mpmath.mp.dps = 40
    Ad = J.toarray()
    xm = mpmath.lu_solve(mpmath.matrix(Ad.tolist()), mpmath.matrix((-R).tolist()))
    xe = np.array([float(v) for v in xm])
    xo = o.solve_linear(J, -R)
    xi = solve_linear_iterative(J, -R, rtol=1e-14)
    for x in (xo, xi):
        assert rel_err(x[: o.Nu], xe[: o.Nu]) <= 1e-12
        assert rel_err(x[o.Nu:], xe[o.Nu:]) <= 1e-12
