"""Plain FP64 CPU oracle of the fully-coupled DG/CZM + lubrication step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code with
the CUDA library; both read the same seeded inputs from ``hf_inputs``.

Everything here follows the paper's statement of the method (Giovanardi,
Serebrinsky, Radovitzky, arXiv 1911.10275), written as directly as possible:

* Spaces (Sec. 3): discontinuous P2 vector displacement per element,
  continuous P2 pressure on the interface skeleton.
* Residual (Eq. discreteElastoStatics, Eq. discreteLubrication): bulk
  elasticity, IIPG-type DG consistency + stability on intact facets weighted
  by (1 - alpha), cohesive traction alpha*t(w), fluid pressure -beta*p*n,
  lubrication with cubic-law conductivity and backward-Euler storage term,
  point injection Q0.
* Jacobian (Eq. fully-coupled-fully-discrete): exact derivative of the
  residual, i.e. the blocks A, B, C, D of the linearised system.
* Newton (Sec. 3, after Eq. fully-coupled-fully-discrete): solve J d = -R,
  stop on relative increments of both nodal arrays.
* Activation: alpha from the DG traction exceeding sigma_c at any facet
  quadrature point (Sec. 3, activation of the TSL); beta at the end of the
  step from the opening exceeding delta_f (Remark in Sec. 3).
* Pre-existing dry crack (Sec. 4.5), as an option: facets whose cohesive
  law is spent (no strength in opening, contact penalty in closure) and,
  with Params.beta_connected, fluid entering a failed facet only from a
  fluid-filled neighbour.

Readings where the paper is silent are named in the docstrings below.
Quadrature rules come from library routines (numpy Gauss-Legendre, scipy
Gauss-Jacobi) combined as conical products; the sparse linear solve is
scipy's direct LU, or, where its fill-in does not fit in memory, the plain
ILU(0)-preconditioned GMRES of oracle/iterative.py.  There is no blocking,
fusion or reordering beyond what the definitions state.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special

TRI_EDGES = ((0, 1), (1, 2), (2, 0))
TET_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))


# --------------------------------------------------------------------------
# quadrature: Gauss rules from library routines, conical products on simplices
# --------------------------------------------------------------------------
def gauss_legendre01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_jacobi01(n, a):
    """Nodes/weights on [0,1] for the weight (1-t)^a."""
    x, w = scipy.special.roots_jacobi(n, a, 0.0)
    return 0.5 * (x + 1.0), w / 2.0 ** (a + 1)


def simplex_rule(s, n):
    """Rule on the reference s-simplex as (barycentric coords (nq, s+1),
    weights (nq,) summing to 1).  s=1: Gauss-Legendre; s=2,3: conical product
    (collapsed coordinates) of Gauss-Jacobi and Gauss-Legendre rules, exact for
    polynomials of degree 2n-1.  Points are listed with the first collapsed
    coordinate outermost."""
    if s == 1:
        t, w = gauss_legendre01(n)
        lam = np.stack([1.0 - t, t], axis=1)
        return lam, w / w.sum()
    if s == 2:
        u, wu = gauss_jacobi01(n, 1.0)
        v, wv = gauss_legendre01(n)
        pts, ws = [], []
        for i in range(n):
            for j in range(n):
                x1 = u[i]
                x2 = v[j] * (1.0 - u[i])
                pts.append((1.0 - x1 - x2, x1, x2))
                ws.append(wu[i] * wv[j])
        ws = np.asarray(ws)
        return np.asarray(pts), ws / ws.sum()
    if s == 3:
        u, wu = gauss_jacobi01(n, 2.0)
        v, wv = gauss_jacobi01(n, 1.0)
        t, wt = gauss_legendre01(n)
        pts, ws = [], []
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    x1 = u[i]
                    x2 = v[j] * (1.0 - u[i])
                    x3 = t[k] * (1.0 - u[i]) * (1.0 - v[j])
                    pts.append((1.0 - x1 - x2 - x3, x1, x2, x3))
                    ws.append(wu[i] * wv[j] * wt[k])
        ws = np.asarray(ws)
        return np.asarray(pts), ws / ws.sum()
    raise ValueError(s)


# --------------------------------------------------------------------------
# P2 Lagrange basis on a simplex, in barycentric coordinates
# --------------------------------------------------------------------------
def p2_values(lam, edges):
    """N (..., nn): vertex functions l_i(2 l_i - 1), edge functions 4 l_a l_b."""
    nv = lam.shape[-1]
    out = [lam[..., i] * (2.0 * lam[..., i] - 1.0) for i in range(nv)]
    out += [4.0 * lam[..., a] * lam[..., b] for a, b in edges]
    return np.stack(out, axis=-1)


def p2_dlam(lam, edges):
    """dN/dlambda (..., nn, nv)."""
    nv = lam.shape[-1]
    nn = nv + len(edges)
    out = np.zeros(lam.shape[:-1] + (nn, nv))
    for i in range(nv):
        out[..., i, i] = 4.0 * lam[..., i] - 1.0
    for m, (a, b) in enumerate(edges):
        out[..., nv + m, a] = 4.0 * lam[..., b]
        out[..., nv + m, b] = 4.0 * lam[..., a]
    return out


def face_local_nodes(dim, i):
    """Face-node order of local facet i: its vertices ascending, then the
    mid-nodes of its edges ascending (the convention of include/hf.h)."""
    edges = TRI_EDGES if dim == 2 else TET_EDGES
    fv = [v for v in range(dim + 1) if v != i]
    mids = sorted(dim + 1 + k for k, (a, b) in enumerate(edges) if a in fv and b in fv)
    return fv + mids


# --------------------------------------------------------------------------
# linear elasticity (Voigt form: the textbook B^T D B)
# --------------------------------------------------------------------------
def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def voigt_D(E, nu, dim):
    """Isotropic elasticity matrix; in 2D the plane-strain one."""
    lam, mu = lame(E, nu)
    if dim == 2:
        return np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def stiffness_tensor(E, nu, dim):
    lam, mu = lame(E, nu)
    I = np.eye(dim)
    return (lam * np.einsum("ij,kl->ijkl", I, I)
            + mu * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I)))


def voigt_B(grads, dim):
    """Strain-displacement matrix (..., nvoigt, nn*dim), engineering shear."""
    sh = grads.shape[:-2]
    nn = grads.shape[-2]
    nv = 3 if dim == 2 else 6
    B = np.zeros(sh + (nv, nn * dim))
    gx = grads[..., 0]
    gy = grads[..., 1]
    if dim == 2:
        B[..., 0, 0::2] = gx
        B[..., 1, 1::2] = gy
        B[..., 2, 0::2] = gy
        B[..., 2, 1::2] = gx
    else:
        gz = grads[..., 2]
        B[..., 0, 0::3] = gx
        B[..., 1, 1::3] = gy
        B[..., 2, 2::3] = gz
        B[..., 3, 1::3] = gz
        B[..., 3, 2::3] = gy
        B[..., 4, 0::3] = gz
        B[..., 4, 2::3] = gx
        B[..., 5, 0::3] = gy
        B[..., 5, 1::3] = gx
    return B


def voigt_to_tensor(s, dim):
    if dim == 2:
        out = np.zeros(s.shape[:-1] + (2, 2))
        out[..., 0, 0] = s[..., 0]
        out[..., 1, 1] = s[..., 1]
        out[..., 0, 1] = out[..., 1, 0] = s[..., 2]
        return out
    out = np.zeros(s.shape[:-1] + (3, 3))
    out[..., 0, 0] = s[..., 0]
    out[..., 1, 1] = s[..., 1]
    out[..., 2, 2] = s[..., 2]
    out[..., 1, 2] = out[..., 2, 1] = s[..., 3]
    out[..., 0, 2] = out[..., 2, 0] = s[..., 4]
    out[..., 0, 1] = out[..., 1, 0] = s[..., 5]
    return out


@dataclasses.dataclass
class Params:
    E: float = 20e9
    nu: float = 0.2
    sigma_c: float = 1e6
    delta_c: float = 96e-6
    b_stab: float = 10.0
    mu: float = 1e-3
    Q0: float = 1e-3
    inj_pdofs: tuple = ()          # pressure DOF indices receiving injection
    inj_weights: tuple = ()        # share of Q0 each (sum 1 for a point source)
    delta_f: float = 96e-6
    dt: float = 1.0
    p_vapor: float = 0.0
    cutoff_on: bool = False
    fluid_scaling: bool = True
    L_ref: float = 100.0
    newton_tol: float = 1e-10
    newton_maxit: int = 25
    fixed_pdofs: tuple = ()        # pressure DOFs held at fixed_pvals (an essential condition)
    fixed_pvals: tuple = ()
    beta_connected: bool = False   # fluid enters a failed facet only from a fluid-filled neighbour


class Oracle:
    """The discrete problem on one mesh; state (U, P, alpha, beta, w_old, t)."""

    FACE_ORDER = {2: 5, 3: 5}    # Gauss points per direction on facets
    VOL_ORDER = {2: 3, 3: 3}
    _consistency_sign = 1.0      # tests plant a sign error here to show the pins bite

    def __init__(self, mesh, params: Params, neu_faces=None, neu_traction=None):
        self.m = mesh
        self.prm = params
        d = mesh.dim
        self.dim = d
        self.edges = TRI_EDGES if d == 2 else TET_EDGES
        self.nn = mesh.elem_nodes.shape[1]
        self.ned = self.nn * d
        self.ne = mesh.elem_nodes.shape[0]
        self.nf = mesh.face_elems.shape[0]
        self.Nu = self.ne * self.ned
        # pressure DOFs: every node of a crackable facet, ascending global id
        pn = set()
        for f in np.nonzero(mesh.face_crackable)[0]:
            e = mesh.face_elems[f, 0]
            loc = face_local_nodes(d, int(mesh.face_local[f, 0]))
            pn.update(int(g) for g in mesh.elem_nodes[e, loc])
        self.pnodes = np.asarray(sorted(pn), dtype=np.int64)
        self.pindex = {int(g): i for i, g in enumerate(self.pnodes)}
        self.Np = self.pnodes.shape[0]
        self.N = self.Nu + self.Np
        self.nfn = len(face_local_nodes(d, 0))
        self._geometry()
        self.neu_faces = np.asarray(neu_faces if neu_faces is not None else [], dtype=np.int64)
        self.neu_traction = np.asarray(neu_traction if neu_traction is not None else
                                       np.zeros((0, d)), dtype=np.float64).reshape(-1, d)
        # state
        self.U = np.zeros(self.Nu)
        self.P = np.zeros(self.Np)
        self.alpha = np.zeros(self.nf, dtype=np.int8)
        self.beta = np.zeros(self.nf, dtype=np.int8)
        self.spent = np.zeros(self.nf, dtype=np.int8)   # 1: a crack whose cohesive law is spent (dry crack)
        self.w_old = np.zeros((self.nf, self.nfn))
        self.t = 0.0
        self.c_scale = 1.0

    # ---------------------------------------------------------------- geometry
    def _geometry(self):
        m, d = self.m, self.dim
        X = m.xyz[m.elem_nodes[:, : d + 1]]                    # (ne, d+1, d)
        T = np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1))      # (ne, d, d)
        self.vol = np.abs(np.linalg.det(T)) / math.factorial(d)
        Tinv = np.linalg.inv(T)                                # rows = grad lambda_1..d
        gl = np.zeros((self.ne, d + 1, d))
        gl[:, 1:] = Tinv
        gl[:, 0] = -Tinv.sum(axis=1)
        self.grad_lam = gl
        self.X0 = X[:, 0]
        self.Tinv = Tinv
        # facets: vertices in e_minus's local order, outward normal of e_minus
        nf = self.nf
        self.fvx = np.zeros((nf, d, d))
        self.normal = np.zeros((nf, d))
        self.area = np.zeros(nf)
        self.hf = np.zeros(nf)
        self.fnodes = np.zeros((nf, self.nfn), dtype=np.int64)   # global ids, face-node order
        for f in range(nf):
            e = m.face_elems[f, 0]
            i = int(m.face_local[f, 0])
            loc = face_local_nodes(d, i)
            self.fnodes[f] = m.elem_nodes[e, loc]
            V = m.xyz[m.elem_nodes[e, loc[:d]]]
            self.fvx[f] = V
            # outward normal of e_minus: opposite to grad lambda_i
            g = gl[e, i]
            self.normal[f] = -g / np.linalg.norm(g)
            if d == 2:
                self.area[f] = np.linalg.norm(V[1] - V[0])
            else:
                self.area[f] = 0.5 * np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0]))
            ep = m.face_elems[f, 1]
            vm = self.vol[e]
            self.hf[f] = (min(vm, self.vol[ep]) if ep >= 0 else vm) / self.area[f]
        self.face_rule = simplex_rule(d - 1, self.FACE_ORDER[d])
        self.vol_rule = simplex_rule(d, self.VOL_ORDER[d])

    def face_points(self, f):
        lam, w = self.face_rule
        return lam @ self.fvx[f], w * self.area[f]

    def elem_basis_at(self, e, x):
        """Basis values (nq, nn) and gradients (nq, nn, d) of element e at
        physical points x (nq, d) via its affine map."""
        xi = (x - self.X0[e]) @ self.Tinv[e].T
        lam = np.concatenate([1.0 - xi.sum(axis=1, keepdims=True), xi], axis=1)
        N = p2_values(lam, self.edges)
        G = np.einsum("qav,vd->qad", p2_dlam(lam, self.edges), self.grad_lam[e])
        return N, G

    def udofs(self, e):
        return e * self.ned + np.arange(self.ned)

    # ---------------------------------------------------------------- pieces
    def element_stiffness(self, e):
        """K_e = sum_q B^T D B |J| w_q (bulk term of Eq. discreteElastoStatics)."""
        lam, w = self.vol_rule
        N = p2_dlam(lam, self.edges)                                  # (nq, nn, nv)
        G = np.einsum("qav,vd->qad", N, self.grad_lam[e])
        B = voigt_B(G, self.dim)
        D = voigt_D(self.prm.E, self.prm.nu, self.dim)
        return np.einsum("q,qia,ij,qjb->ab", w * self.vol[e], B, D, B)

    def _side(self, f):
        m = self.m
        return [(int(m.face_elems[f, 0]), -1.0), (int(m.face_elems[f, 1]), +1.0)]

    def intact_blocks(self, f):
        """DG consistency + stability blocks of an interior facet (second line
        of Eq. discreteElastoStatics, without the (1 - alpha) factor), IIPG as
        written.  Returns {(s, t): (ned x ned)} for sides s, t in {0: -, 1: +};
        rows are test DOFs of side s, columns trial DOFs of side t."""
        d = self.dim
        x, wq = self.face_points(f)
        n = self.normal[f]
        Cten = stiffness_tensor(self.prm.E, self.prm.nu, d)
        Dv = voigt_D(self.prm.E, self.prm.nu, d)
        pen = self.prm.b_stab / self.hf[f]
        sides = self._side(f)
        basis = [self.elem_basis_at(e, x) for e, _ in sides]
        # traction of each trial DOF: sigma(N_b e_l) n  -> (nq, ned, d)
        trac = []
        for (N, G) in basis:
            B = voigt_B(G, d)                                   # (nq, nv, ned)
            S = voigt_to_tensor(np.einsum("ij,qjb->qbi", Dv, B), d)   # (nq, ned, d, d)
            trac.append(np.einsum("qbij,j->qbi", S, n))
        # (e_k x n) : C : (e_l x n)
        CC = np.einsum("j,ijkl,l->ik", n, Cten, n)
        out = {}
        for s in range(2):
            Ns, _ = basis[s]
            sig_s = sides[s][1]
            vjump = np.zeros((len(wq), self.ned, d))            # [[v]] for test DOF (a,k)
            for a in range(self.nn):
                for k in range(d):
                    vjump[:, a * d + k, k] = sig_s * Ns[:, a]
            for t in range(2):
                Nt, _ = basis[t]
                sig_t = sides[t][1]
                ujump = np.zeros((len(wq), self.ned, d))
                for b in range(self.nn):
                    for l in range(d):
                        ujump[:, b * d + l, l] = sig_t * Nt[:, b]
                cons = self._consistency_sign * 0.5 * np.einsum("q,qai,qbi->ab", wq, vjump, trac[t])
                stab = pen * np.einsum("q,qai,ik,qbk->ab", wq, vjump, CC, ujump)
                out[(s, t)] = cons + stab
        return out

    def tsl(self, w, f):
        """Traction-separation law (Eq. tsl) with the readings: zero traction
        beyond delta_c, contact penalty (b/h)(lambda+2mu) for w < 0.  On a
        spent facet (a pre-existing dry crack, Sec. 4.5) the law has no
        strength left: zero traction in opening, the same contact penalty in
        closure (continuous at w = 0)."""
        p = self.prm
        lam, mu = lame(p.E, p.nu)
        kp = p.b_stab / self.hf[f] * (lam + 2 * mu)
        if self.spent[f]:
            return np.where(w < 0.0, kp * w, 0.0), np.where(w < 0.0, kp, 0.0)
        T = np.where(w < 0.0, p.sigma_c + kp * w,
                     np.where(w < p.delta_c, p.sigma_c * (1.0 - w / p.delta_c), 0.0))
        dT = np.where(w < 0.0, kp, np.where(w < p.delta_c, -p.sigma_c / p.delta_c, 0.0))
        return T, dT

    def face_kinematics(self, f, U):
        """At facet quadrature points: basis of both sides, jump, opening."""
        x, wq = self.face_points(f)
        n = self.normal[f]
        sides = self._side(f)
        basis = [self.elem_basis_at(e, x) for e, _ in sides]
        jump = np.zeros((len(wq), self.dim))
        for (e, sg), (N, _) in zip(sides, basis):
            ue = U[self.udofs(e)].reshape(self.nn, self.dim)
            jump += sg * N @ ue
        return x, wq, n, sides, basis, jump, jump @ n

    def opening_at_face_nodes(self, U):
        """w = [[u]].n at the face nodes of every interior facet (Eq.
        displacementJump), face-node order; boundary facets get 0."""
        w = np.zeros((self.nf, self.nfn))
        m, d = self.m, self.dim
        for f in range(self.nf):
            ep = int(m.face_elems[f, 1])
            if ep < 0:
                continue
            em = int(m.face_elems[f, 0])
            um = U[self.udofs(em)].reshape(self.nn, d)
            up = U[self.udofs(ep)].reshape(self.nn, d)
            for a, g in enumerate(self.fnodes[f]):
                am = int(np.nonzero(m.elem_nodes[em] == g)[0][0])
                ap = int(np.nonzero(m.elem_nodes[ep] == g)[0][0])
                w[f, a] = (up[ap] - um[am]) @ self.normal[f]
        return w

    def pressure_trace(self, f, x):
        """eta_g and surface gradients at points x for the face nodes of f:
        the trace of e_minus's P2 basis, gradient projected on the facet."""
        m = self.m
        e = int(m.face_elems[f, 0])
        N, G = self.elem_basis_at(e, x)
        loc = face_local_nodes(self.dim, int(m.face_local[f, 0]))
        n = self.normal[f]
        Pn = np.eye(self.dim) - np.outer(n, n)
        eta = N[:, loc]
        geta = G[:, loc, :] @ Pn
        pd = np.array([self.pindex[int(g)] for g in self.fnodes[f]])
        return eta, geta, pd

    def active_pdofs(self):
        act = np.zeros(self.Np, dtype=bool)
        for f in np.nonzero(self.beta)[0]:
            act[[self.pindex[int(g)] for g in self.fnodes[f]]] = True
        return act

    def update_scaling(self):
        """c^n = (1/(12 mu) (max w^n / L)^3)^-1 applied to the fluid rows."""
        p = self.prm
        wmax = self.w_old[self.m.face_crackable.astype(bool)].max(initial=0.0)
        if p.fluid_scaling and wmax > 0.0:
            self.c_scale = 12.0 * p.mu / (wmax / p.L_ref) ** 3
        else:
            self.c_scale = 1.0

    # ---------------------------------------------------------------- assembly
    def assemble(self, U=None, P=None, with_jacobian=True, elems=None, pdofs=None):
        """Residual R(U, P) and Jacobian J = dR/d(U, P) in natural DOF order
        (displacements element-major, then pressures).

        With ``elems`` / ``pdofs`` given, only those elements and the facets
        touching them or those pressure DOFs are visited: the rows of the
        listed elements and pressure DOFs are then exact and every other row
        is partial (used to check sampled rows of a large problem)."""
        U = self.U if U is None else U
        P = self.P if P is None else P
        sample = elems is not None or pdofs is not None
        if sample:
            elem_list = np.asarray(elems if elems is not None else [], dtype=np.int64)
            want_p = set(int(g) for g in (pdofs if pdofs is not None else []))
            touch = set(int(e) for e in elem_list)
            face_list = [f for f in range(self.nf)
                         if int(self.m.face_elems[f, 0]) in touch or int(self.m.face_elems[f, 1]) in touch
                         or (self.m.face_crackable[f] and
                             any(self.pindex[int(g)] in want_p for g in self.fnodes[f]))]
            neu = [(f, tb) for f, tb in zip(self.neu_faces, self.neu_traction)
                   if int(self.m.face_elems[f, 0]) in touch]
        else:
            elem_list = range(self.ne)
            face_list = range(self.nf)
            neu = list(zip(self.neu_faces, self.neu_traction))
        R, coo = self.assemble_terms(U, P, elem_list, face_list, neu, with_jacobian)
        J = None
        if with_jacobian:
            J = sp.coo_matrix((coo[2], (coo[0], coo[1])), shape=(self.N, self.N)).tocsr()
        return self.finish_assembly(R, J, U, P)

    def assemble_terms(self, U, P, elem_list, face_list, neu, with_jacobian=True):
        """The sums of Eq. discreteElastoStatics and Eq. discreteLubrication
        over the listed elements (bulk term), interior facets (DG, cohesive
        and fluid terms) and Neumann facets ``neu`` = [(facet, traction)]:
        R and the Jacobian entries as COO arrays (rows, cols, vals), without
        the injection and the identity rows (``finish_assembly``).  Assembly
        is a sum over elements and facets, so partial sums over a partition of
        them add up to the whole."""
        p = self.prm
        d, ned = self.dim, self.ned
        R = np.zeros(self.N)
        rows, cols, vals = [], [], []

        def add(r, c, v):
            rr, cc = np.meshgrid(r, c, indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(v.ravel())

        # bulk elasticity
        for e in elem_list:
            Ke = self.element_stiffness(e)
            dofs = self.udofs(e)
            R[dofs] += Ke @ U[dofs]
            if with_jacobian:
                add(dofs, dofs, Ke)
        # interior facets
        act = self.active_pdofs()
        c = self.c_scale
        for f in face_list:
            if self.m.face_elems[f, 1] < 0:
                continue
            sides = self._side(f)
            dofs = [self.udofs(e) for e, _ in sides]
            a_f = int(self.alpha[f])
            b_f = int(self.beta[f])
            if a_f == 0:
                blk = self.intact_blocks(f)
                for s in range(2):
                    for t in range(2):
                        R[dofs[s]] += blk[(s, t)] @ U[dofs[t]]
                        if with_jacobian:
                            add(dofs[s], dofs[t], blk[(s, t)])
            if a_f == 0 and b_f == 0:
                continue
            x, wq, n, sides, basis, jump, w = self.face_kinematics(f, U)
            # test-jump normal component: sigma_s N_a n_k, per side (nq, ned)
            njump = [sg * np.einsum("qa,k->qak", N, n).reshape(len(wq), ned)
                     for (e, sg), (N, _) in zip(sides, basis)]
            if a_f:
                T, dT = self.tsl(w, f)
                for s in range(2):
                    R[dofs[s]] += np.einsum("q,q,qa->a", wq, T, njump[s])
                    if with_jacobian:
                        for t in range(2):
                            add(dofs[s], dofs[t],
                                np.einsum("q,q,qa,qb->ab", wq, dT, njump[s], njump[t]))
            if b_f:
                eta, geta, pd = self.pressure_trace(f, x)
                ph = eta @ P[pd]
                gp = np.einsum("qgi,g->qi", geta, P[pd])
                wp = np.maximum(w, 0.0)
                k3 = wp ** 3 / (12.0 * p.mu)
                dk3 = 3.0 * wp ** 2 / (12.0 * p.mu)
                wn = eta @ self.w_old[f]
                pdofs = self.Nu + pd
                for s in range(2):
                    R[dofs[s]] += -np.einsum("q,q,qa->a", wq, ph, njump[s])
                    if with_jacobian:
                        add(dofs[s], pdofs, -np.einsum("q,qa,qg->ag", wq, njump[s], eta))
                gg = np.einsum("qgi,qi->qg", geta, gp)
                R[pdofs] += c * (np.einsum("q,q,qg->g", wq, k3, gg)
                                 + np.einsum("q,q,qg->g", wq, (w - wn) / p.dt, eta))
                if with_jacobian:
                    for s in range(2):
                        add(pdofs, dofs[s], c * (np.einsum("q,q,qg,qb->gb", wq, dk3, gg, njump[s])
                                                 + np.einsum("q,qg,qb->gb", wq, eta, njump[s]) / p.dt))
                    add(pdofs, pdofs, c * np.einsum("q,q,qgi,qhi->gh", wq, k3, geta, geta))
        # Neumann traction on outer facets
        for f, tb in neu:
            e = int(self.m.face_elems[f, 0])
            x, wq = self.face_points(f)
            N, _ = self.elem_basis_at(e, x)
            R[self.udofs(e)] -= np.einsum("q,qa,k->ak", wq, N, tb).ravel()
        if with_jacobian and rows:
            coo = (np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
        else:
            coo = (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0))
        return R, coo

    def finish_assembly(self, R, J, U=None, P=None):
        """Adds the point injection to the summed terms and imposes the
        identity rows (inactive pressures p = p_v, Dirichlet displacements)."""
        U = self.U if U is None else U
        P = self.P if P is None else P
        p = self.prm
        act = self.active_pdofs()
        c = self.c_scale
        # injection (point source Q0 split by weights)
        for g, wgt in zip(p.inj_pdofs, p.inj_weights):
            R[self.Nu + g] -= c * p.Q0 * wgt
        # identity rows: inactive pressures (p = p_v), fixed pressures and
        # Dirichlet displacements
        fixed = np.zeros(self.Np, dtype=bool)
        fixed[list(p.fixed_pdofs)] = True
        fval = np.full(self.Np, p.p_vapor)
        fval[list(p.fixed_pdofs)] = p.fixed_pvals
        free = ~act & ~fixed
        ident = list(self.Nu + np.nonzero(free)[0]) + list(self.Nu + np.nonzero(fixed)[0]) + list(self.m.dir_dof)
        ident = np.asarray(ident, dtype=np.int64)
        target = np.concatenate([np.full(int(free.sum()), p.p_vapor), fval[fixed], self.m.dir_val])
        cur = np.concatenate([P[free], P[fixed], U[self.m.dir_dof]])
        R[ident] = cur - target
        if J is not None and ident.size:
            # row r of J becomes e_r^T: keep the other rows, add the unit diagonal
            is_id = np.zeros(self.N)
            is_id[ident] = 1.0
            J = (sp.diags(1.0 - is_id) @ J.tocsr() + sp.diags(is_id)).tocsr()
            J.eliminate_zeros()
        return R, J

    # ---------------------------------------------------------------- steps
    @staticmethod
    def solve_linear(J, b, refinements=3):
        """Exact solution of the linearised system J d = b (Eq.
        fully-coupled-fully-discrete).  The raw matrix mixes force rows
        (~E h), identity rows and scaled flux rows; its condition number is
        ~1e21, so the direct solve runs on the row- then column-equilibrated
        matrix (max-abs scaling, an exact change of rows and unknowns), by a
        library sparse LU, followed by iterative refinement on the original
        system with the same factors."""
        J = J.tocsr()
        r = 1.0 / abs(J).max(axis=1).toarray().ravel()
        J1 = sp.diags(r) @ J
        c = 1.0 / abs(J1).max(axis=0).toarray().ravel()
        A = (J1 @ sp.diags(c)).tocsc()
        lu = spla.splu(A)
        x = c * lu.solve(r * b)
        for _ in range(refinements):
            x = x + c * lu.solve(r * (b - J @ x))
        return x

    def newton_step(self, solve=None, assemble=None):
        """One Newton iteration: J d = -R, update, relative increments.
        ``solve(J, b)`` replaces the direct solve and ``assemble()`` the
        serial assembly (same definitions, other routes to them)."""
        R, J = self.assemble() if assemble is None else assemble()
        d = self.solve_linear(J, -R) if solve is None else solve(J, -R)
        dU, dP = d[: self.Nu], d[self.Nu:]
        P_old = self.P
        self.U = self.U + dU
        self.P = self.P + dP
        if self.prm.cutoff_on:
            act = self.active_pdofs()
            self.P[act] = np.maximum(self.P[act], self.prm.p_vapor)
            # the increment of the nodal pressure array is the change applied,
            # cut-off included
            dP = self.P - P_old
        du = np.linalg.norm(dU) / max(np.linalg.norm(self.U), 1e-300)
        dp = np.linalg.norm(dP) / max(np.linalg.norm(self.P), 1e-300)
        return dict(du_rel=du, dp_rel=dp, res_norm=float(np.linalg.norm(R)),
                    converged=bool(du <= self.prm.newton_tol and dp <= self.prm.newton_tol))

    def staggered_step(self, solve=None):
        """One iteration of the staggered scheme of Sec. 4.3 ("Fully-coupled
        vs. staggered"): the two equations solved in turn for their own
        unknown with the other taken from the previous iteration, i.e. the
        linear system of Eq. fully-coupled-fully-discrete decoupled into
        A dU = -R_u(U, P) and then, at the updated opening,
        D dP = -R_p(U + dU, P).  The decoupled fluid problem is elliptic and
        needs an essential pressure somewhere (Params.fixed_pdofs).  Reports
        the relative increments as newton_step does."""
        solve = solve or self.solve_linear
        Nu = self.Nu
        R, J = self.assemble()
        dU = solve(J[:Nu, :Nu].tocsr(), -R[:Nu])
        self.U = self.U + dU
        R2, J2 = self.assemble()
        D = J2[Nu:, Nu:].tocsr()
        if np.any(abs(D).max(axis=1).toarray().ravel() == 0.0):
            # a pressure row with no conductivity left (the opening closed on
            # every facet around it): the decoupled fluid problem is singular
            nan = float("nan")
            return dict(du_rel=nan, dp_rel=nan, res_norm=float(np.linalg.norm(R)), converged=False)
        dP = solve(D, -R2[Nu:])
        P_old = self.P
        self.P = self.P + dP
        if self.prm.cutoff_on:
            act = self.active_pdofs()
            self.P[act] = np.maximum(self.P[act], self.prm.p_vapor)
            dP = self.P - P_old
        du = np.linalg.norm(dU) / max(np.linalg.norm(self.U), 1e-300)
        dp = np.linalg.norm(dP) / max(np.linalg.norm(self.P), 1e-300)
        return dict(du_rel=du, dp_rel=dp, res_norm=float(np.linalg.norm(R)),
                    converged=bool(du <= self.prm.newton_tol and dp <= self.prm.newton_tol))

    def dg_normal_traction(self, f, U=None):
        """Normal DG traction n.<sigma(u)>n + (b/h) n.(C:([[u]] x n)) n at the
        facet quadrature points (the traction exchanged on an intact facet)."""
        U = self.U if U is None else U
        d = self.dim
        x, wq, n, sides, basis, jump, w = self.face_kinematics(f, U)
        Dv = voigt_D(self.prm.E, self.prm.nu, d)
        Cten = stiffness_tensor(self.prm.E, self.prm.nu, d)
        savg = np.zeros((len(wq), d, d))
        for (e, sg), (N, G) in zip(sides, basis):
            B = voigt_B(G, d)
            eps = np.einsum("qvb,b->qv", B, U[self.udofs(e)])
            savg += 0.5 * voigt_to_tensor(eps @ Dv.T, d)
        cons = np.einsum("i,qij,j->q", n, savg, n)
        stab = self.prm.b_stab / self.hf[f] * np.einsum("i,ijkl,qk,l,j->q", n, Cten, jump, n, n)
        return cons + stab

    def check_fracture_criterion(self):
        """alpha = 1 (irreversibly) on crackable intact facets where the DG
        normal traction exceeds sigma_c at any quadrature point."""
        new = 0
        tmax = np.full(self.nf, -np.inf)
        for f in np.nonzero(self.m.face_crackable)[0]:
            if self.alpha[f]:
                continue
            tdg = self.dg_normal_traction(f)
            tmax[f] = tdg.max()
            if tmax[f] > self.prm.sigma_c:
                new += 1
        flip = (tmax > self.prm.sigma_c) & (self.alpha == 0)
        self.alpha[flip] = 1
        return new, tmax

    def accept_step(self):
        """End of step: beta = 1 where alpha = 1 and the opening exceeds
        delta_f at a quadrature point; w^n <- w^{n+1}; t += dt; rescale.
        With prm.beta_connected such a facet takes fluid only when it shares
        a node with a fluid-filled facet (one wetted in this step counts), so
        a dry crack not reached by the fluid stays dry."""
        new = 0
        cand = []
        for f in np.nonzero(self.m.face_crackable)[0]:
            if self.alpha[f] and not self.beta[f]:
                w = self.face_kinematics(f, self.U)[-1]
                if w.max() > self.prm.delta_f:
                    cand.append(int(f))
        if not self.prm.beta_connected:
            for f in cand:
                self.beta[f] = 1
                new += 1
        else:
            wet = set()
            for f in np.nonzero(self.beta)[0]:
                wet.update(self.face_nodes(int(f)))
            grew = True
            while grew:
                grew = False
                for f in cand:
                    if not self.beta[f] and wet.intersection(self.face_nodes(f)):
                        self.beta[f] = 1
                        wet.update(self.face_nodes(f))
                        new += 1
                        grew = True
        self.w_old = self.opening_at_face_nodes(self.U)
        self.t += self.prm.dt
        self.update_scaling()
        return new

    def face_nodes(self, f):
        """Global node ids of facet f (its minus side's face nodes)."""
        e = self.m.face_elems[f, 0]
        loc = face_local_nodes(self.dim, int(self.m.face_local[f, 0]))
        return set(int(g) for g in self.m.elem_nodes[e, loc])

    def set_state(self, U, P, alpha, beta, w_old=None, t=0.0, spent=None):
        """spent: facets of a pre-existing dry crack (cohesive law spent;
        they must have alpha = 1), zeros when not given."""
        self.U = np.array(U, dtype=np.float64)
        self.P = np.array(P, dtype=np.float64)
        self.alpha = np.array(alpha, dtype=np.int8)
        self.beta = np.array(beta, dtype=np.int8)
        self.spent = np.zeros(self.nf, dtype=np.int8) if spent is None else np.array(spent, dtype=np.int8)
        if np.any(self.spent & (self.alpha == 0)):
            raise ValueError("a spent facet must have alpha = 1")
        self.w_old = self.opening_at_face_nodes(self.U) if w_old is None else \
            np.array(w_old, dtype=np.float64).reshape(self.nf, self.nfn)
        self.t = float(t)
        self.update_scaling()
