"""Writes c1_steps_oracle.json: the FP64 oracle's first time steps of the 2D
KGD workload c1 (square of 100 m, 44 x 44 squares of two P2 triangles:
3,872 elements, 46,553 unknowns; crack on the midline; E = 20 GPa,
nu = 0.2, K_Ic = 1 MPa sqrt(m), sigma_c = 1 MPa, mu = 1e-3 Pa s,
Q0 = 1e-3 m^2/s, dt = 1 s; pressure cut-off on; Newton to 1e-10) from its
seed state, each step driven by the rules of hf_advance_step (Newton until
the relative increments of U and P are at most 1e-10, the fracture
criterion of Sec. 3, Newton again while it switches facets, the end of the
step; failed attempts undone and retried with half the sub-step).  The
Newton systems are solved by the oracle's direct LU; the assembly is summed
over a process pool.  Only oracle/, the oracle's driver in tests/_setup.py
and the seeded input generator are used.

Stored per step: the step report (Newton iterations, cutbacks, sub-steps),
the attempt log (sub-step, Newton iterations per round, facets switched by
each criterion, accepted or undone) from which a caller can replay the
oracle's decisions,
facet-state counts and lists, U at a fixed sample of unknowns, every
non-zero pressure, the openings at the face nodes of every cohesive or fluid
facet, and the infinity norms of the full fields.

    python tests/golden/make_c1_steps.py [--steps 10] [--workers 8]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    ap.add_argument("--out", default=os.path.join(HERE, "c1_steps_oracle.json"))
    args = ap.parse_args()
    from hf_inputs import c1_kgd_toughness
    from oracle import Oracle, Params, parallel
    from _setup import oracle_advance_step

    wl = c1_kgd_toughness()
    inj, wts = wl.injection()
    prm = Params(E=wl.E, nu=wl.nu, sigma_c=wl.sigma_c, delta_c=wl.delta_c, b_stab=wl.b_stab, mu=wl.mu,
                 Q0=wl.Q0, inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=wl.delta_f, dt=wl.dt,
                 p_vapor=0.0, cutoff_on=True, fluid_scaling=True, L_ref=wl.fluid_length, newton_tol=1e-10)
    o = Oracle(wl.mesh, prm)
    o.set_state(*wl.seed())
    m = wl.mesh
    rng = np.random.default_rng(191110275)
    crack_faces = np.nonzero(m.face_crackable)[0]
    near = np.unique(m.face_elems[crack_faces].ravel())
    near = near[near >= 0]
    u_idx = np.unique(np.concatenate([
        rng.choice(o.Nu, 128, replace=False),
        (rng.choice(near, 32, replace=False)[:, None] * o.ned + rng.integers(0, o.ned, (32, 4))).ravel()]))
    out = {"workload": wl.name, "unknowns": int(o.N), "elements": int(o.ne), "u_index": u_idx.tolist(),
           "rules": "hf_advance_step: Newton tol 1e-10, newton_max 8 (continuing while increments halve, "
                    "at most 32), criterion rounds 4, cutbacks halve the sub-step, growth 1.5; cut-off on",
           "linear_solve": "oracle direct LU (equilibrated, 3 refinement steps)", "steps": []}

    def newton():
        return o.newton_step(assemble=lambda: parallel.assemble(o, workers=args.workers))

    for k in range(1, args.steps + 1):
        t0 = time.time()
        log = []
        rep = oracle_advance_step(o, newton=newton, log=log)
        wf = o.opening_at_face_nodes(o.U)
        faces = np.nonzero(m.face_crackable & ((o.alpha > 0) | (o.beta > 0)))[0]
        p_idx = np.nonzero(o.P != 0.0)[0]
        out["steps"].append({"k": k, "t": o.t, **{key: int(v) for key, v in rep.items()}, "attempts": log,
                             "alpha_faces": np.nonzero(o.alpha)[0].tolist(),
                             "beta_faces": np.nonzero(o.beta)[0].tolist(),
                             "U": o.U[u_idx].tolist(), "P_index": p_idx.tolist(), "P": o.P[p_idx].tolist(),
                             "w_faces": faces.tolist(), "w": wf[faces].tolist(),
                             "U_inf": float(np.abs(o.U).max()), "P_inf": float(np.abs(o.P).max()),
                             "w_inf": float(np.abs(wf[crack_faces]).max())})
        print(f"step {k}: t={o.t:.3f} {rep} alpha={int(o.alpha.sum())} beta={int(o.beta.sum())} "
              f"{time.time() - t0:.0f}s", flush=True)
        with open(args.out + ".tmp", "w") as f:
            json.dump(out, f)
        os.replace(args.out + ".tmp", args.out)


if __name__ == "__main__":
    main()
