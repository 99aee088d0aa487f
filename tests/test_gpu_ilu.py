"""The block-Jacobi preconditioner as block ILU(0), checked against the
definition: per subdomain, the element blocks of the displacement block A of
the Newton system (the oracle's, cohesive tangents included), eliminated in
the library's order (hf_get_subdomains),
    L_ik = A_ik D_k^-1 for earlier neighbours k,  D_i = A_ii - sum_k L_ik A_ki,
then z = (L D)^-1 ... by the forward and backward block substitutions.  The
structured meshes have no element-graph triangles inside a subdomain, so no
fill between neighbours arises and this recurrence is the whole of block
ILU(0).  Coarse level off; subdomains of 4 and 32 elements, 2D and 3D, one
cohesive facet in the softening branch."""
import numpy as np
import pytest

from hf_inputs import kgd_2d, penny_3d
from _setup import oracle_for, gpu_for, with_extra_cohesive, rel_err

pytestmark = pytest.mark.gpu


def block_ilu0_apply(A, ned, face_elems, sd_of, order, r):
    """z = M^-1 r for the block-Jacobi block ILU(0) of the sparse matrix A
    (element blocks of ned unknowns; neighbours = elements sharing a facet)."""
    ne = sd_of.size
    z = np.zeros(ne * ned)
    A = A.tocsr()
    cache = {}

    def blk(i, k):
        if (i, k) not in cache:
            cache[(i, k)] = A[i * ned:(i + 1) * ned, k * ned:(k + 1) * ned].toarray()
        return cache[(i, k)]

    nbrs = {e: [] for e in range(ne)}
    for em, ep in face_elems:
        if ep >= 0 and sd_of[em] == sd_of[ep]:
            nbrs[int(em)].append(int(ep))
            nbrs[int(ep)].append(int(em))
    for s in np.unique(sd_of):
        elems = [int(e) for e in np.nonzero(sd_of == s)[0]]
        elems.sort(key=lambda e: order[e])
        D, L = {}, {}
        for i in elems:
            Dii = blk(i, i).copy()
            for k in nbrs[i]:
                if order[k] < order[i]:
                    L[(i, k)] = blk(i, k) @ np.linalg.inv(D[k])
                    Dii -= L[(i, k)] @ blk(k, i)
            D[i] = Dii
        y = {}
        for i in elems:
            yi = r[i * ned:(i + 1) * ned].copy()
            for k in nbrs[i]:
                if order[k] < order[i]:
                    yi -= L[(i, k)] @ y[k]
            y[i] = yi
        for i in elems[::-1]:
            t = y[i].copy()
            for k in nbrs[i]:
                if order[k] > order[i]:
                    t -= blk(i, k) @ z[k * ned:(k + 1) * ned]
            z[i * ned:(i + 1) * ned] = np.linalg.solve(D[i], t)
    return z


CASES = {
    "2d": lambda: kgd_2d(n=6, length=12.0, crackable="all", steps=1, seed_cells=2),
    "3d": lambda: penny_3d(n=4, length=8.0, crackable="all", steps=1, seed_cells=1),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("G", [4, 32])
def test_preconditioner_is_block_ilu0(name, G):
    wl = CASES[name]()
    state, _ = with_extra_cohesive(wl, wl.seed(), count=1)
    o = oracle_for(wl)
    o.set_state(*state)
    g = gpu_for(wl, jacobi_block=G, coarse=0, precision="fp64")
    g.hf_set_state(*state)
    _, J = o.assemble()
    A = J[: o.Nu, : o.Nu]
    sd_of, order = g.hf_get_subdomains()
    assert sd_of.max() + 1 == -(-wl.mesh.n_elems // G)
    rng = np.random.default_rng(13)
    for _ in range(2):
        x = np.zeros(o.N)
        x[: o.Nu] = rng.standard_normal(o.Nu)
        zg = g.hf_apply_preconditioner(x)
        zr = block_ilu0_apply(A, o.ned, wl.mesh.face_elems, sd_of, order, x[: o.Nu])
        assert rel_err(zg[: o.Nu], zr) <= 1e-10
    g.close()
