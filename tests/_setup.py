"""Shared set-up for parity tests: the same seeded workload and state fed to
the CUDA library (through the C ABI) and to the FP64 oracle."""
import numpy as np

from oracle import Oracle, Params


def oracle_for(wl, fluid_scaling=True, cutoff=False):
    inj, wts = wl.injection()
    prm = Params(E=wl.E, nu=wl.nu, sigma_c=wl.sigma_c, delta_c=wl.delta_c, b_stab=wl.b_stab, mu=wl.mu,
                 Q0=wl.Q0, inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=wl.delta_f, dt=wl.dt,
                 L_ref=wl.fluid_length, fluid_scaling=fluid_scaling, cutoff_on=cutoff)
    return Oracle(wl.mesh, prm)


def gpu_for(wl, fluid_scaling=True, cutoff=False, **solver):
    from paper_1911_10275_gb300 import HFMesh
    inj, wts = wl.injection()
    g = HFMesh.from_mesh(wl.mesh)
    g.hf_set_material(wl.E, wl.nu, wl.sigma_c, wl.delta_c, wl.b_stab)
    g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, wl.dt, 0.0, cutoff, wl.fluid_length)
    opts = dict(rtol=1e-13, max_iters=20000, jacobi_block=16, fluid_scaling=int(fluid_scaling))
    opts.update(solver)
    g.hf_set_solver(**opts)
    return g


def with_extra_cohesive(wl, state, count=1, opening=3e-5):
    """Seed state plus `count` cohesive-only facets (alpha=1, beta=0) next to
    the seed, opened by `opening` (inside the softening branch)."""
    U, P, al, be = (np.array(x, copy=True) for x in state)
    m = wl.mesh
    cr = np.nonzero(m.face_crackable & (al == 0))[0]
    c = m.xyz[m.center_node]
    # nearest crackable intact facets to the seed
    d = []
    for f in cr:
        e = m.face_elems[f, 0]
        d.append(np.linalg.norm(m.xyz[m.elem_nodes[e, : m.dim + 1]].mean(axis=0) - c))
    pick = cr[np.argsort(d)[:count]]
    nen, dim = m.n_en, m.dim
    for f in pick:
        al[f] = 1
        ep = m.face_elems[f, 1]
        U[ep * nen * dim + np.arange(nen) * dim + m.crack_normal_axis] += opening
    return (U, P, al, be), pick


def rel_err(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def oracle_advance_step(o, newton_max=8, rounds_max=4, max_cutbacks=10, newton=None, log=None, max_new_facets=0):
    """One time step of Sec. 3 on the oracle, with the driver rules of
    hf_advance_step: Newton until converged, the criterion, Newton again if it
    switched facets (at most rounds_max rounds), end of step; an attempt that
    does not converge within newton_max iterations (or turns non-finite) is
    undone and retried with half the sub-step, which grows back by 1.5 after
    each accepted sub-step until t + dt is reached; at most max_cutbacks
    failures in a row, 256 attempts in all.  Past newton_max an attempt goes
    on while the increments at least halve every iteration (at most
    4 newton_max iterations); with max_new_facets > 0 an attempt whose
    criterion switches more facets than that in one round fails too.
    ``newton()`` replaces ``o.newton_step()``
    (the same iteration with pooled assembly, say).  With ``log`` a list, one
    record per attempt is appended: its sub-step, the Newton iterations of
    each Newton round (a round ends with the fracture criterion), the facets
    each criterion switched, and whether the attempt was accepted."""
    newton = newton or o.newton_step
    dt0 = o.prm.dt
    target = o.t + dt0
    sub = dt0
    rep = {"newton_iters": 0, "cutbacks": 0, "substeps": 0}

    def snap():
        return (o.U.copy(), o.P.copy(), o.alpha.copy(), o.beta.copy(), o.w_old.copy(), o.t)

    saved = snap()
    cuts = attempts = 0
    while target - o.t > 1e-12 * dt0:
        sub = min(sub, target - o.t)
        o.prm.dt = sub
        ok, rounds, it, prev = False, 0, 0, np.inf
        rec = {"dt": sub, "rounds": [], "switched": [], "accepted": False}
        while True:
            r = newton()
            rep["newton_iters"] += 1
            it += 1
            if not (np.isfinite(r["du_rel"]) and np.isfinite(r["dp_rel"])):
                break
            if r["converged"]:
                n_new, _ = o.check_fracture_criterion()
                rounds += 1
                rec["rounds"].append(it)
                rec["switched"].append(int(n_new))
                if max_new_facets > 0 and n_new > max_new_facets:
                    it = None      # its Newton count is in rec["rounds"] already
                    break
                if n_new == 0 or rounds >= rounds_max:
                    ok = True
                    break
                it, prev = 0, np.inf
                continue
            inc = max(r["du_rel"], r["dp_rel"])
            if it >= newton_max and (it >= 4 * newton_max or not inc <= 0.5 * prev):
                break
            prev = inc
        attempts += 1
        if not ok and it is not None:
            rec["rounds"].append(it)
        rec["accepted"] = ok
        if log is not None:
            log.append(rec)
        if ok:
            o.accept_step()
            rep["substeps"] += 1
            cuts = 0
            saved = snap()
            sub = min(dt0, 1.5 * sub)
        else:
            o.set_state(*saved)
            cuts += 1
            assert cuts <= max_cutbacks and attempts < 256
            rep["cutbacks"] += 1
            sub *= 0.5
    o.t = target
    o.prm.dt = dt0
    return rep
