"""Shared set-up for parity tests: the same seeded workload and state fed to
the CUDA library (through the C ABI) and to the FP64 oracle."""
import numpy as np

from oracle import Oracle, Params


def oracle_for(wl, fluid_scaling=True, cutoff=False):
    inj, wts = wl.injection()
    prm = Params(E=wl.E, nu=wl.nu, sigma_c=wl.sigma_c, delta_c=wl.delta_c, b_stab=wl.b_stab, mu=wl.mu,
                 Q0=wl.Q0, inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=wl.delta_f, dt=wl.dt,
                 L_ref=wl.mesh.length, fluid_scaling=fluid_scaling, cutoff_on=cutoff)
    return Oracle(wl.mesh, prm)


def gpu_for(wl, fluid_scaling=True, cutoff=False, **solver):
    from paper_1911_10275_gb300 import HFMesh
    inj, wts = wl.injection()
    g = HFMesh.from_mesh(wl.mesh)
    g.hf_set_material(wl.E, wl.nu, wl.sigma_c, wl.delta_c, wl.b_stab)
    g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, wl.dt, 0.0, cutoff, wl.mesh.length)
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
