"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module holds input data only: structured P2 simplex meshes, their face
topology, boundary-condition lists, crackable-face sets and a kinematic seed
state.  It contains none of the method's arithmetic (no basis functions, no
quadrature, no weak-form terms); both the CUDA library and the CPU oracle
receive the arrays built here and discretise them independently.

Conventions (the interface contract of ``include/hf.h``):

* 2D elements are 6-node triangles: vertices 0,1,2 counter-clockwise, then the
  edge mid-nodes 3=(0,1), 4=(1,2), 5=(2,0).
* 3D elements are 10-node tetrahedra with positive volume: vertices 0..3, then
  mid-nodes 4=(0,1), 5=(1,2), 6=(0,2), 7=(0,3), 8=(1,3), 9=(2,3).
* Local face i of an element is the facet opposite vertex i.
* ``face_elems[f] = (e_minus, e_plus)``; ``e_plus = -1`` marks a boundary facet.
  The opening normal of a facet is the outward normal of ``e_minus``.
* Displacement DOF of (element e, local node a, component k) is
  ``e*n_nodes_per_elem*dim + a*dim + k``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TRI_EDGES = ((0, 1), (1, 2), (2, 0))          # mid-nodes 3,4,5
TET_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))  # mid-nodes 4..9


@dataclasses.dataclass
class Mesh:
    dim: int
    xyz: np.ndarray            # (n_nodes, dim) float64
    elem_nodes: np.ndarray     # (n_elems, 6|10) int32
    face_elems: np.ndarray     # (n_faces, 2) int32
    face_local: np.ndarray     # (n_faces, 2) int8
    face_crackable: np.ndarray  # (n_faces,) int8
    dir_dof: np.ndarray        # (n_dir,) int64
    dir_val: np.ndarray        # (n_dir,) float64
    length: float              # domain side length L
    n: int                     # cells per side
    center_node: int           # global node id of the domain centre
    crack_normal_axis: int     # axis normal to the preferred crack plane

    @property
    def n_elems(self) -> int:
        return int(self.elem_nodes.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.face_elems.shape[0])

    @property
    def n_en(self) -> int:
        return int(self.elem_nodes.shape[1])

    @property
    def n_u(self) -> int:
        return self.n_elems * self.n_en * self.dim


def _local_face_vertices(dim: int, i: int) -> tuple:
    """Vertices of local face i (opposite vertex i), ascending local index."""
    return tuple(v for v in range(dim + 1) if v != i)


def _build_faces(dim: int, elem_nodes: np.ndarray):
    """Face list from element vertex sets: interior facets carry two elements."""
    nv = dim + 1
    ne = elem_nodes.shape[0]
    keys = []
    for i in range(nv):
        fv = _local_face_vertices(dim, i)
        keys.append(np.sort(elem_nodes[:, list(fv)], axis=1))
    keys = np.stack(keys, axis=1).reshape(ne * nv, dim)   # (ne*nv, dim)
    owner = np.repeat(np.arange(ne, dtype=np.int64), nv)
    local = np.tile(np.arange(nv, dtype=np.int64), ne)
    order = np.lexsort(keys.T[::-1])
    ks = keys[order]
    same_as_next = np.all(ks[:-1] == ks[1:], axis=1)
    faces_e = []
    faces_l = []
    i = 0
    m = ks.shape[0]
    idx_first = []
    while i < m:
        if i + 1 < m and same_as_next[i]:
            a, b = order[i], order[i + 1]
            ea, eb = owner[a], owner[b]
            if ea > eb:
                a, b = b, a
                ea, eb = eb, ea
            faces_e.append((ea, eb))
            faces_l.append((local[a], local[b]))
            idx_first.append(min(ea, eb))
            i += 2
        else:
            a = order[i]
            faces_e.append((owner[a], -1))
            faces_l.append((local[a], -1))
            idx_first.append(owner[a])
            i += 1
    fe = np.asarray(faces_e, dtype=np.int64)
    fl = np.asarray(faces_l, dtype=np.int64)
    # deterministic order: by e_minus, then local face id
    o = np.lexsort((fl[:, 0], fe[:, 0]))
    return fe[o].astype(np.int32), fl[o].astype(np.int8)


def _rollers(dim, xyz, elem_nodes, face_elems, face_local, half):
    """Zero normal displacement on every outer facet (strong, nodal)."""
    n_en = elem_nodes.shape[1]
    edges = TRI_EDGES if dim == 2 else TET_EDGES
    dofs = set()
    bnd = np.nonzero(face_elems[:, 1] < 0)[0]
    for f in bnd:
        e = int(face_elems[f, 0])
        i = int(face_local[f, 0])
        fv = _local_face_vertices(dim, i)
        loc = list(fv) + [dim + 1 + k for k, (a, b) in enumerate(edges)
                          if a in fv and b in fv]
        vx = xyz[elem_nodes[e, list(fv)]]
        # the facet lies on the plane where one coordinate is +-half
        for axis in range(dim):
            if np.all(np.abs(np.abs(vx[:, axis]) - half) < 1e-9 * half) and \
               np.all(np.abs(vx[:, axis] - vx[0, axis]) < 1e-9 * half):
                for a in loc:
                    dofs.add(e * n_en * dim + a * dim + axis)
    d = np.asarray(sorted(dofs), dtype=np.int64)
    return d, np.zeros(d.shape[0], dtype=np.float64)


def square_p2(n: int, length: float = 100.0, crackable: str = "midline",
              jitter: float = 0.0, seed: int = 191110275) -> Mesh:
    """[-L/2, L/2]^2 split into n x n squares, two P2 triangles per square.

    n must be even so that the midline y=0 and the centre node exist.
    ``crackable``: "midline" (edges on y=0) or "all" (every interior edge).
    ``jitter`` moves interior vertices by up to jitter*h (seeded), mid-nodes
    stay at edge midpoints.
    """
    if n % 2:
        raise ValueError("n must be even")
    g = 2 * n + 1
    h = length / n
    ii, jj = np.meshgrid(np.arange(g), np.arange(g), indexing="xy")
    xyz = np.stack([-length / 2 + ii.ravel() * (length / (2 * n)),
                    -length / 2 + jj.ravel() * (length / (2 * n))], axis=1)

    def nid(i, j):
        return j * g + i

    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    I = I.ravel()
    J = J.ravel()
    i0, j0 = 2 * I, 2 * J
    t1 = np.stack([nid(i0, j0), nid(i0 + 2, j0), nid(i0 + 2, j0 + 2),
                   nid(i0 + 1, j0), nid(i0 + 2, j0 + 1), nid(i0 + 1, j0 + 1)], axis=1)
    t2 = np.stack([nid(i0, j0), nid(i0 + 2, j0 + 2), nid(i0, j0 + 2),
                   nid(i0 + 1, j0 + 1), nid(i0 + 1, j0 + 2), nid(i0, j0 + 1)], axis=1)
    elem = np.empty((2 * n * n, 6), dtype=np.int64)
    elem[0::2] = t1
    elem[1::2] = t2
    if jitter > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        vi = (ii.ravel() % 2 == 0) & (jj.ravel() % 2 == 0)
        inner = vi & (ii.ravel() > 0) & (ii.ravel() < g - 1) & (jj.ravel() > 0) & (jj.ravel() < g - 1)
        # keep the crack line and the centre straight
        inner &= np.abs(xyz[:, 1]) > 1e-9 * length
        d = rng.uniform(-jitter * h, jitter * h, size=(int(inner.sum()), 2))
        xyz[inner] += d
        for (a, b), m in zip(TRI_EDGES, (3, 4, 5)):
            xyz[elem[:, m]] = 0.5 * (xyz[elem[:, a]] + xyz[elem[:, b]])
    fe, fl = _build_faces(2, elem)
    crack = np.zeros(fe.shape[0], dtype=np.int8)
    interior = fe[:, 1] >= 0
    if crackable == "all":
        crack[interior] = 1
    elif crackable == "midline":
        for f in np.nonzero(interior)[0]:
            fv = _local_face_vertices(2, int(fl[f, 0]))
            y = xyz[elem[fe[f, 0], list(fv)], 1]
            if np.all(np.abs(y) < 1e-9 * length):
                crack[f] = 1
    else:
        raise ValueError(crackable)
    dd, dv = _rollers(2, xyz, elem, fe, fl, length / 2)
    return Mesh(2, xyz, elem.astype(np.int32), fe, fl, crack, dd, dv, length, n,
                int(nid(n, n)), 1)


def split_triangles(mesh: Mesh, elems, crackable: str = "all") -> Mesh:
    """The 2D P2 mesh with each listed triangle split at its centroid into
    three (new vertex and the three new edge mid-nodes appended, the edges
    of the old triangle and their mid-nodes kept).  The three children share
    edges pairwise, so the element graph gains triangles: block ILU(0) then
    has fill between neighbours through a common earlier neighbour.
    ``crackable`` as in square_p2 ("all" or "midline")."""
    if mesh.dim != 2:
        raise ValueError("triangles only")
    xyz = [tuple(p) for p in mesh.xyz]
    out = [list(e) for e in mesh.elem_nodes]

    def add(p):
        xyz.append((float(p[0]), float(p[1])))
        return len(xyz) - 1
    for e in sorted(set(int(x) for x in elems)):
        v = [int(mesh.elem_nodes[e, k]) for k in range(3)]
        mid = {TRI_EDGES[k]: int(mesh.elem_nodes[e, 3 + k]) for k in range(3)}
        pv = [np.asarray(mesh.xyz[x]) for x in v]
        c = add((pv[0] + pv[1] + pv[2]) / 3.0)
        mc = [add((pv[k] + np.asarray(xyz[c])) / 2.0) for k in range(3)]
        kids = []
        for a, b in TRI_EDGES:   # child (v_a, v_b, c), counter-clockwise as its parent
            m_ab = mid[(a, b)]
            kids.append([v[a], v[b], c, m_ab, mc[b], mc[a]])
        out[e] = kids[0]
        out.extend(kids[1:])
    elem = np.asarray(out, dtype=np.int64)
    xyz = np.asarray(xyz, dtype=np.float64)
    fe, fl = _build_faces(2, elem)
    crack = np.zeros(fe.shape[0], dtype=np.int8)
    interior = fe[:, 1] >= 0
    if crackable == "all":
        crack[interior] = 1
    elif crackable == "midline":
        for f in np.nonzero(interior)[0]:
            fv = _local_face_vertices(2, int(fl[f, 0]))
            y = xyz[elem[fe[f, 0], list(fv)], 1]
            if np.all(np.abs(y) < 1e-9 * mesh.length):
                crack[f] = 1
    else:
        raise ValueError(crackable)
    dd, dv = _rollers(2, xyz, elem, fe, fl, mesh.length / 2)
    return Mesh(2, xyz, elem.astype(np.int32), fe, fl, crack, dd, dv, mesh.length, mesh.n,
                mesh.center_node, mesh.crack_normal_axis)


def cube_p2(n: int, length: float = 50.0, crackable: str = "plane") -> Mesh:
    """[-L/2, L/2]^3 split into n^3 cubes, six Kuhn P2 tetrahedra per cube.

    ``crackable``: "plane" (facets on z=0) or "all" (every interior facet).
    """
    if n % 2:
        raise ValueError("n must be even")
    g = 2 * n + 1
    h2 = length / (2 * n)
    ii, jj, kk = np.meshgrid(np.arange(g), np.arange(g), np.arange(g), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    order = np.lexsort((ii, jj, kk))    # node id = (k*g + j)*g + i
    ii, jj, kk = ii[order], jj[order], kk[order]
    xyz = np.stack([-length / 2 + ii * h2, -length / 2 + jj * h2, -length / 2 + kk * h2], axis=1)

    def nid(i, j, k):
        return (k * g + j) * g + i

    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    o = np.lexsort((I, J, K))
    I, J, K = I[o], J[o], K[o]
    perms = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
    tets = []
    for p in perms:
        pts = [np.zeros(3, dtype=np.int64)]
        for ax in p:
            q = pts[-1].copy()
            q[ax] += 1
            pts.append(q)
        pts = np.array(pts)
        vol = np.linalg.det((pts[1:] - pts[0]).astype(float))
        if vol < 0:
            pts = pts[[0, 1, 3, 2]]
        tets.append(pts)
    nc = I.shape[0]
    elem = np.empty((nc, 6, 10), dtype=np.int64)
    base = np.stack([2 * I, 2 * J, 2 * K], axis=1)
    for t, pts in enumerate(tets):
        vg = base[:, None, :] + 2 * pts[None, :, :]        # (nc, 4, 3) grid coords
        for a in range(4):
            elem[:, t, a] = nid(vg[:, a, 0], vg[:, a, 1], vg[:, a, 2])
        for m, (a, b) in enumerate(TET_EDGES):
            mg = (vg[:, a] + vg[:, b]) // 2
            elem[:, t, 4 + m] = nid(mg[:, 0], mg[:, 1], mg[:, 2])
    elem = elem.reshape(nc * 6, 10)
    fe, fl = _build_faces(3, elem)
    crack = np.zeros(fe.shape[0], dtype=np.int8)
    interior = fe[:, 1] >= 0
    if crackable == "all":
        crack[interior] = 1
    elif crackable == "plane":
        for f in np.nonzero(interior)[0]:
            fv = _local_face_vertices(3, int(fl[f, 0]))
            z = xyz[elem[fe[f, 0], list(fv)], 2]
            if np.all(np.abs(z) < 1e-9 * length):
                crack[f] = 1
    else:
        raise ValueError(crackable)
    dd, dv = _rollers(3, xyz, elem, fe, fl, length / 2)
    return Mesh(3, xyz, elem.astype(np.int32), fe, fl, crack, dd, dv, length, n,
                int(nid(n, n, n)), 2)


def pressure_nodes(mesh: Mesh) -> np.ndarray:
    """Global node ids carrying a pressure unknown: every node of a crackable
    facet, ascending.  Position in this array is the pressure DOF index."""
    edges = TRI_EDGES if mesh.dim == 2 else TET_EDGES
    nodes = set()
    for f in np.nonzero(mesh.face_crackable)[0]:
        e = int(mesh.face_elems[f, 0])
        fv = _local_face_vertices(mesh.dim, int(mesh.face_local[f, 0]))
        loc = list(fv) + [mesh.dim + 1 + k for k, (a, b) in enumerate(edges) if a in fv and b in fv]
        nodes.update(int(x) for x in mesh.elem_nodes[e, loc])
    return np.asarray(sorted(nodes), dtype=np.int64)


def face_vertex_coords(mesh: Mesh, f: int) -> np.ndarray:
    e = int(mesh.face_elems[f, 0])
    fv = _local_face_vertices(mesh.dim, int(mesh.face_local[f, 0]))
    return mesh.xyz[mesh.elem_nodes[e, list(fv)]]


def seed_faces(mesh: Mesh, radius: float) -> np.ndarray:
    """Crackable facets on the preferred crack plane whose vertices all lie
    within ``radius`` of the domain centre (the pre-existing seed crack)."""
    ax = mesh.crack_normal_axis
    c = mesh.xyz[mesh.center_node]
    out = np.zeros(mesh.n_faces, dtype=np.int8)
    for f in np.nonzero(mesh.face_crackable)[0]:
        v = face_vertex_coords(mesh, f)
        if np.all(np.abs(v[:, ax] - c[ax]) < 1e-9 * mesh.length) and \
           np.all(np.linalg.norm(v - c, axis=1) <= radius * (1 + 1e-12)):
            out[f] = 1
    return out


def seed_state(mesh: Mesh, radius: float, w0: float, p0: float):
    """Kinematic seed: elements above the crack plane move by +w/2 along the
    plane normal and those below by -w/2, with w = w0*sqrt(1-(r/R)^2) tapering
    to zero at the seed rim and decaying linearly away from the plane.  The
    seed facets are cohesive-failed and fluid-filled (alpha = beta = 1) and the
    pressure is p0 on their nodes.  Returns (U, P, alpha, beta)."""
    ax = mesh.crack_normal_axis
    c = mesh.xyz[mesh.center_node]
    n_en, d = mesh.n_en, mesh.dim
    X = mesh.xyz[mesh.elem_nodes]                     # (ne, n_en, d)
    cen = X[:, :d + 1].mean(axis=1)
    side = np.sign(cen[:, ax] - c[ax])
    rel = X - c
    r_in = np.sqrt(np.maximum(np.sum(rel ** 2, axis=2) - rel[:, :, ax] ** 2, 0.0))
    g_in = np.sqrt(np.maximum(0.0, 1.0 - (r_in / radius) ** 2))
    g_out = np.maximum(0.0, 1.0 - np.abs(rel[:, :, ax]) / radius)
    U = np.zeros((mesh.n_elems, n_en, d))
    U[:, :, ax] = side[:, None] * 0.5 * w0 * g_in * g_out
    sf = seed_faces(mesh, radius)
    pn = pressure_nodes(mesh)
    pos = {int(g): i for i, g in enumerate(pn)}
    P = np.zeros(pn.shape[0])
    edges = TRI_EDGES if d == 2 else TET_EDGES
    for f in np.nonzero(sf)[0]:
        e = int(mesh.face_elems[f, 0])
        fv = _local_face_vertices(d, int(mesh.face_local[f, 0]))
        loc = list(fv) + [d + 1 + k for k, (a, b) in enumerate(edges) if a in fv and b in fv]
        for gnode in mesh.elem_nodes[e, loc]:
            P[pos[int(gnode)]] = p0
    U = U.reshape(-1)
    U[mesh.dir_dof] = mesh.dir_val
    return U, P, sf.copy(), sf.copy()


def round_even(x: float) -> int:
    return max(2, 2 * int(round(x / 2.0)))


def batch_instances(count: int, seed: int = 191110275, ne_range=(1000, 50000)):
    """Parameter draws for a sweep of independent 2D instances: element count,
    E, K_Ic, mu, Q0 all log-uniform in their ranges (seeded PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def lu(lo, hi, size):
        return np.exp(rng.uniform(math.log(lo), math.log(hi), size))
    ne = lu(*ne_range, count)
    out = []
    E = lu(5e9, 50e9, count)
    K = lu(0.1e6, 3e6, count)
    mu = lu(1e-3, 1.0, count)
    Q0 = lu(1e-4, 1e-2, count)
    for i in range(count):
        out.append(dict(n=round_even(math.sqrt(ne[i] / 2.0)), E=float(E[i]), K_Ic=float(K[i]),
                        mu=float(mu[i]), Q0=float(Q0[i])))
    return out


def far_field_load(mesh: Mesh, sigma0: float):
    """A far-field stress sigma0 normal to the crack plane (compressive for
    sigma0 > 0), as the outer load of the propagation test of the paper:
    the rollers normal to the crack plane are removed from the face at
    +L/2 along the crack normal, and that face carries the traction
    -sigma0 n (n its outward normal); the opposite face keeps its rollers.
    Returns (mesh with the reduced Dirichlet list, Neumann facets, their
    tractions (n_neumann, dim))."""
    ax, half, d = mesh.crack_normal_axis, mesh.length / 2, mesh.dim
    edges = TRI_EDGES if d == 2 else TET_EDGES
    n_en = mesh.n_en
    top, drop = [], set()
    for f in np.nonzero(mesh.face_elems[:, 1] < 0)[0]:
        e = int(mesh.face_elems[f, 0])
        fv = _local_face_vertices(d, int(mesh.face_local[f, 0]))
        vx = mesh.xyz[mesh.elem_nodes[e, list(fv)]]
        if np.all(np.abs(vx[:, ax] - half) < 1e-9 * half):
            top.append(int(f))
            loc = list(fv) + [d + 1 + k for k, (a, b) in enumerate(edges) if a in fv and b in fv]
            for a in loc:
                drop.add(e * n_en * d + a * d + ax)
    keep = np.array([k not in drop for k in mesh.dir_dof.tolist()], dtype=bool)
    m2 = dataclasses.replace(mesh, dir_dof=mesh.dir_dof[keep], dir_val=mesh.dir_val[keep])
    trac = np.zeros((len(top), d))
    trac[:, ax] = -sigma0
    return m2, np.asarray(top, dtype=np.int32), trac
