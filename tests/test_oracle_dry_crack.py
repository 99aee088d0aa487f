"""Oracle pins for a pre-existing dry crack (Sec. 4.5: a fluid-driven crack
meeting a natural crack), the first of the two NEXT-4 extensions not yet on
the GPU.  Readings, as the oracle implements them: a dry crack is a set of
facets with alpha = 1, beta = 0 and a spent cohesive law (`spent`): zero
traction in opening, the contact penalty (b/h)(lambda + 2 mu) in closure;
with `beta_connected` the end of the step wets a failed facet only when it
shares a node with a fluid-filled one.

Pins: (i) the spent law's values and slopes; (ii) a dry crack cutting the
whole square, closed by a uniform far-field compression sigma0, transmits
the load through contact alone: the exact discrete solution is the uniform
stress with the crack closed by sigma0 / k_p; (iii) a dry crack under remote
tension opens exactly as the same crack held at that pressure with no far
field (superposition, exact for the linear problem); (iv) the tangent
against central differences with spent facets open and closed; (v) the
connectivity rule of the end of step."""
import numpy as np
import pytest

from hf_inputs import kgd_2d, far_field_load, pressure_nodes
from oracle import Oracle, Params, fem


def _oracle(m, wl, **kw):
    inj, wts = wl.injection()
    prm = dict(E=wl.E, nu=wl.nu, sigma_c=1e6, delta_c=1e-4, b_stab=10.0, mu=wl.mu, Q0=0.0,
               inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=1e-6, dt=1.0, L_ref=wl.fluid_length,
               newton_tol=1e-11)
    prm.update(kw.pop("prm", {}))
    return Oracle(m, Params(**prm), **kw)


def _midline(m):
    return np.nonzero(m.face_crackable)[0]


def _facet_x(m, f):
    e, j = m.face_elems[f, 0], m.face_local[f, 0]
    vs = [v for v in range(3) if v != j]
    return m.xyz[m.elem_nodes[e, vs], 0].mean()


def _newton(o, its=8):
    for _ in range(its):
        r = o.newton_step()
        if r["converged"]:
            return r
    raise AssertionError(r)


def test_spent_law_values_and_slopes():
    wl = kgd_2d(n=8, length=16.0, crackable="midline")
    o = _oracle(wl.mesh, wl)
    f = int(_midline(wl.mesh)[0])
    al = np.zeros(o.nf, np.int8)
    al[f] = 1
    sp = al.copy()
    o.set_state(np.zeros(o.Nu), np.zeros(o.Np), al, np.zeros(o.nf, np.int8), spent=sp)
    lam, mu = fem.lame(o.prm.E, o.prm.nu)
    kp = o.prm.b_stab / o.hf[f] * (lam + 2 * mu)
    w = np.array([-2e-5, -1e-9, 0.0, 1e-9, 5e-5, 3e-4])
    T, dT = o.tsl(w, f)
    assert np.allclose(T, [-2e-5 * kp, -1e-9 * kp, 0, 0, 0, 0], rtol=1e-14, atol=0)
    assert np.array_equal(dT, [kp, kp, 0, 0, 0, 0])
    # the intact-strength law differs by sigma_c in closure, and only there below delta_c
    o.spent[f] = 0
    T2, _ = o.tsl(w, f)
    assert np.allclose(T2[:2] - T[:2], o.prm.sigma_c, rtol=1e-12)
    # a spent facet must have been activated
    with pytest.raises(ValueError):
        o.set_state(np.zeros(o.Nu), np.zeros(o.Np), np.zeros(o.nf, np.int8), np.zeros(o.nf, np.int8), spent=sp)


def test_closed_dry_crack_transmits_uniform_compression():
    """A dry crack along the whole midline under the far-field compression
    sigma0: the exact discrete solution is the uniform stress, the crack
    closed by sigma0 / k_p at every face node (P2 reproduces the piecewise
    linear field with that jump)."""
    wl = kgd_2d(n=8, length=16.0, crackable="midline")
    sigma0 = 3e6
    m, nf, tr = far_field_load(wl.mesh, sigma0)
    o = _oracle(m, wl, neu_faces=nf, neu_traction=tr)
    cr = _midline(m)
    al = np.zeros(o.nf, np.int8)
    al[cr] = 1
    U = np.zeros(o.Nu)
    ax = m.crack_normal_axis
    for e in range(o.ne):     # start with the crack slightly closed (contact branch active)
        if m.xyz[m.elem_nodes[e, :3], ax].mean() > 0:
            U[o.udofs(e)[ax::2]] -= 1e-7
    o.set_state(U, np.zeros(o.Np), al, np.zeros(o.nf, np.int8), spent=al)
    _newton(o)
    lam, mu = fem.lame(o.prm.E, o.prm.nu)
    kp = o.prm.b_stab / o.hf[cr[0]] * (lam + 2 * mu)
    assert np.allclose(o.hf[cr], o.hf[cr[0]])
    w = o.opening_at_face_nodes(o.U)[cr]
    assert np.abs(w + sigma0 / kp).max() <= 1e-9 * sigma0 / kp
    # the stress is uniform: on the crack plane the average normal stress is -sigma0, and the
    # criterion's DG traction adds the penalty on the jump, k_p w = -sigma0: -2 sigma0 in all
    t = np.array([o.dg_normal_traction(int(f)) for f in cr])
    assert np.abs(t + 2 * sigma0).max() <= 1e-6 * sigma0


def test_open_dry_crack_under_tension_equals_the_pressurised_crack():
    """Superposition: a dry crack under the remote tension s opens exactly as
    the same crack, fluid-filled and held at pressure s, with no far field."""
    wl = kgd_2d(n=12, length=24.0, crackable="midline")
    s = 2e6
    m, nf, tr = far_field_load(wl.mesh, -s)            # a negative far-field stress pulls
    cr = _midline(m)
    crack = np.array([f for f in cr if abs(_facet_x(m, f)) < 3.0])
    al = np.zeros(m.n_faces, np.int8)
    al[crack] = 1
    # (a) dry, under tension
    oa = _oracle(m, wl, neu_faces=nf, neu_traction=tr)
    oa.set_state(np.zeros(oa.Nu), np.zeros(oa.Np), al, np.zeros(oa.nf, np.int8), spent=al)
    _newton(oa)
    wa = oa.opening_at_face_nodes(oa.U)[crack]
    # (b) the same facets fluid-filled at pressure s, no far field
    m0, nf0, tr0 = far_field_load(wl.mesh, 0.0)
    pn = pressure_nodes(m0)
    ob = _oracle(m0, wl, neu_faces=nf0, neu_traction=tr0,
                 prm=dict(fixed_pdofs=tuple(range(pn.size)), fixed_pvals=tuple([s] * pn.size)))
    ob.set_state(np.zeros(ob.Nu), np.full(ob.Np, s), al, al, spent=al)
    _newton(ob)
    wb = ob.opening_at_face_nodes(ob.U)[crack]
    assert wa.min() >= 0.0 and wa.max() > 0.0
    assert np.abs(wa - wb).max() <= 1e-9 * np.abs(wb).max()


def test_tangent_with_spent_facets_open_and_closed():
    wl = kgd_2d(n=6, length=12.0, crackable="midline")
    m = wl.mesh
    o = _oracle(m, wl)
    cr = _midline(m)
    al = np.zeros(o.nf, np.int8)
    al[cr] = 1
    U = np.zeros(o.Nu)
    ax = m.crack_normal_axis
    rng = np.random.default_rng(3)
    for e in range(o.ne):      # some crack facets opened, some closed
        c = m.xyz[m.elem_nodes[e, :3]].mean(axis=0)
        if c[ax] > 0:
            U[o.udofs(e)[ax::2]] += 2e-5 if c[0] > 0 else -2e-5
    U += 1e-7 * rng.standard_normal(o.Nu)
    o.set_state(U, np.zeros(o.Np), al, np.zeros(o.nf, np.int8), spent=al)
    w = o.opening_at_face_nodes(U)[cr]
    assert w.min() < 0 < w.max()
    R, J = o.assemble()
    cols = []
    for f in cr[:4]:
        for e in m.face_elems[f]:
            cols += list(o.udofs(int(e))[ax::2][:3])
    for j in cols:
        h = 1e-10
        xp = U.copy()
        xp[j] += h
        xm = U.copy()
        xm[j] -= h
        Rp, _ = o.assemble(xp, o.P, False)
        Rm, _ = o.assemble(xm, o.P, False)
        fd = (Rp - Rm) / (2 * h)
        col = J[:, j].toarray().ravel()
        assert np.abs(fd - col).max() <= 1e-6 * np.abs(col).max(), j


def test_fluid_enters_only_connected_failed_facets():
    """End of step with beta_connected: of the failed facets opened past
    delta_f, those sharing a node with the fluid (directly or through facets
    wetted in the same step) take fluid; a dry crack separated from it by an
    intact facet stays dry.  Without the option every such facet is wetted."""
    wl = kgd_2d(n=12, length=24.0, crackable="midline")
    m = wl.mesh
    cr = sorted(_midline(m), key=lambda f: _facet_x(m, f))
    x = np.array([_facet_x(m, f) for f in cr])
    wet = [f for f, xi in zip(cr, x) if abs(xi) < 2.0]             # the fluid-filled crack
    near = [f for f, xi in zip(cr, x) if 2.0 < abs(xi) < 4.0]      # failed, connected to it
    far = [f for f, xi in zip(cr, x) if 6.0 < abs(xi) < 8.0]       # failed, behind an intact gap
    al = np.zeros(m.n_faces, np.int8)
    be = np.zeros(m.n_faces, np.int8)
    al[wet + near + far] = 1
    be[wet] = 1
    sp = np.zeros(m.n_faces, np.int8)
    sp[far] = 1
    for connected, expect in ((True, set(near)), (False, set(near) | set(far))):
        o = _oracle(m, wl, prm=dict(beta_connected=connected))
        U = np.zeros(o.Nu)
        for e in range(o.ne):   # the upper half lifted: every midline facet opens by 1e-4
            if m.xyz[m.elem_nodes[e, :3], 1].mean() > 0:
                U[o.udofs(e)[1::2]] += 1e-4
        o.set_state(U, np.zeros(o.Np), al, be, spent=sp)
        n = o.accept_step()
        got = set(int(f) for f in np.nonzero(o.beta & (be == 0))[0])
        assert got == expect and n == len(expect)
