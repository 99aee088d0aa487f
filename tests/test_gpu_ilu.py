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
import dataclasses

import numpy as np
import pytest

from hf_inputs import kgd_2d, penny_3d, split_triangles
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


def block_ilu0_full_apply(A, ned, face_elems, sd_of, order, r):
    """z = M^-1 r for the complete block ILU(0) of each subdomain's element
    blocks: row by row in the elimination order, A_ij -= L_ik U_kj for every
    earlier neighbour k of i and every block j of row i that row k also has,
    which includes the updates between neighbours through a common earlier
    neighbour (element-graph triangles)."""
    ne = sd_of.size
    z = np.zeros(ne * ned)
    A = A.tocsr()

    def blk(i, k):
        return A[i * ned:(i + 1) * ned, k * ned:(k + 1) * ned].toarray()

    nbrs = {e: [] for e in range(ne)}
    for em, ep in face_elems:
        if ep >= 0 and sd_of[em] == sd_of[ep]:
            nbrs[int(em)].append(int(ep))
            nbrs[int(ep)].append(int(em))
    for s in np.unique(sd_of):
        elems = sorted((int(e) for e in np.nonzero(sd_of == s)[0]), key=lambda e: order[e])
        U, L = {}, {}
        for i in elems:
            W = {i: blk(i, i)}
            for j in nbrs[i]:
                W[j] = blk(i, j)
            for k in sorted((k for k in nbrs[i] if order[k] < order[i]), key=lambda e: order[e]):
                L[(i, k)] = W[k] @ np.linalg.inv(U[(k, k)])
                for j in W:
                    if order[j] > order[k] and (k, j) in U:
                        W[j] = W[j] - L[(i, k)] @ U[(k, j)]
            for j, wj in W.items():
                if order[j] >= order[i]:
                    U[(i, j)] = wj
        y = {}
        for i in elems:
            yi = r[i * ned:(i + 1) * ned].copy()
            for k in nbrs[i]:
                if order[k] < order[i]:
                    yi -= L[(i, k)] @ y[k]
            y[i] = yi
        for i in elems[::-1]:
            t = y[i].copy()
            for j in nbrs[i]:
                if order[j] > order[i]:
                    t -= U[(i, j)] @ z[j * ned:(j + 1) * ned]
            z[i * ned:(i + 1) * ned] = np.linalg.solve(U[(i, i)], t)
    return z


@pytest.mark.parametrize("G", [4, 32])
def test_preconditioner_drops_the_fill_through_element_triangles(G):
    """On a mesh whose element graph has triangles inside subdomains (every
    triangle of the 6 x 6 KGD square split into three at its centroid), the
    preconditioner is the block ILU(0) recurrence without the updates of
    off-diagonal blocks through a common earlier neighbour, as the library
    documents: equal to that recurrence, and measurably different from the
    complete block ILU(0) (so the test sees the dropped fill)."""
    wl = kgd_2d(n=6, length=12.0, crackable="all", steps=1, seed_cells=2)
    wl = dataclasses.replace(wl, mesh=split_triangles(wl.mesh, range(wl.mesh.n_elems)))
    state, _ = with_extra_cohesive(wl, wl.seed(), count=1)
    o = oracle_for(wl)
    o.set_state(*state)
    g = gpu_for(wl, jacobi_block=G, coarse=0, precision="fp64")
    g.hf_set_state(*state)
    _, J = o.assemble()
    A = J[: o.Nu, : o.Nu]
    sd_of, order = g.hf_get_subdomains()
    m = wl.mesh
    adj = {e: set() for e in range(m.n_elems)}
    for em, ep in m.face_elems:
        if ep >= 0 and sd_of[em] == sd_of[ep]:
            adj[int(em)].add(int(ep))
            adj[int(ep)].add(int(em))
    triangles = sum(1 for i in adj for j in adj[i] for k in adj[j] if i < j < k and k in adj[i])
    assert triangles > 0
    rng = np.random.default_rng(17)
    x = np.zeros(o.N)
    x[: o.Nu] = rng.standard_normal(o.Nu)
    zg = g.hf_apply_preconditioner(x)[: o.Nu]
    g.close()
    z_drop = block_ilu0_apply(A, o.ned, m.face_elems, sd_of, order, x[: o.Nu])
    z_full = block_ilu0_full_apply(A, o.ned, m.face_elems, sd_of, order, x[: o.Nu])
    assert rel_err(zg, z_drop) <= 1e-10
    assert rel_err(zg, z_full) >= 1e-6
