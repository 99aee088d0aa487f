"""Writes c3_newton_oracle.json: the FP64 oracle's trajectory over the first
Newton iterations of the 3D penny workload (cube of 50 m, 18^3 cubes of six
P2 tetrahedra: 34,992 elements, 1,051,129 unknowns; crack plane z = 0) from
its seed state.  The driving rules are the ones bench.py applies to the CUDA
library: the Newton iteration of Sec. 3 (after Eq.
fully-coupled-fully-discrete) until the relative increments of U and P are
both at most 1e-8; then the fracture criterion (Sec. 3, activation of the
TSL), Newton again if it switched facets (at most 4 rounds), then the end of
the step (beta and w^n, Remark in Sec. 3); an attempt that has not converged
after 8 iterations restarts the step from its initial state with half the
time step, and accepted steps grow it back by 1.5 up to dt.  Pressure cut-off
at p_v = 0 on, fluid-row scaling on.

Each linear system is solved by the oracle's own ILU(0)-preconditioned GMRES
(oracle/iterative.py) to a relative residual of 1e-13 on the equilibrated
system; the assembly is the oracle's, summed over a process pool.  Only
oracle/ and the seeded input generator hf_inputs/ are used.

Stored per iteration (sampled, to keep the file small): the relative
increments, the facet-state counts, U at a fixed sample of unknowns, every
non-zero pressure, the opening at the face nodes of every cohesive or
fluid-filled facet, and the infinity norms of the full U, P and opening
fields (the denominators of the relative errors).

    python tests/golden/make_c3_newton.py [--iters 20] [--n 18] [--workers 8]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--n", type=int, default=18)
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "c3_newton_oracle.json"))
    args = ap.parse_args()
    from hf_inputs import c3_penny, penny_3d
    from oracle import Oracle, Params
    from oracle import parallel
    from oracle.iterative import solve_linear_iterative

    wl = c3_penny() if args.n == 18 else penny_3d(n=args.n, crackable="plane", name=f"penny3d_n{args.n}_plane")
    inj, wts = wl.injection()
    prm = Params(E=wl.E, nu=wl.nu, sigma_c=wl.sigma_c, delta_c=wl.delta_c, b_stab=wl.b_stab, mu=wl.mu,
                 Q0=wl.Q0, inj_pdofs=tuple(inj), inj_weights=tuple(wts), delta_f=wl.delta_f, dt=wl.dt,
                 p_vapor=0.0, cutoff_on=True, fluid_scaling=True, L_ref=wl.fluid_length, newton_tol=1e-8)
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

    def solve(J, b):
        info = {}
        x = solve_linear_iterative(J, b, rtol=1e-13, restart=100, info=info)
        solve.last = info
        return x

    def assemble():
        return parallel.assemble(o, workers=args.workers)

    dt0 = wl.dt
    dt = dt0
    saved = (o.U.copy(), o.P.copy(), o.alpha.copy(), o.beta.copy(), o.w_old.copy(), o.t)
    it_in_step = rounds = 0
    out = {"workload": wl.name, "unknowns": int(o.N), "elements": int(o.ne), "u_index": u_idx.tolist(),
           "rules": "Newton tol 1e-8 on both relative increments; criterion rounds <= 4; cap 8 iterations "
                    "then restart with dt/2; growth 1.5 back to dt; cut-off p >= 0; fluid scaling on",
           "linear_solve": "oracle ILU(0) + GMRES(100), refinement to relative residual 1e-13 (equilibrated)",
           "iters": []}
    for k in range(1, args.iters + 1):
        t0 = time.time()
        rep = o.newton_step(solve=solve, assemble=assemble)
        it_in_step += 1
        events = []
        if rep["converged"]:
            n_new, _ = o.check_fracture_criterion()
            rounds += 1
            events.append(f"criterion:{n_new}")
            if n_new == 0 or rounds >= 4:
                nb = o.accept_step()
                events.append(f"accept:{nb}")
                it_in_step = rounds = 0
                saved = (o.U.copy(), o.P.copy(), o.alpha.copy(), o.beta.copy(), o.w_old.copy(), o.t)
                if dt < dt0:
                    dt = min(dt0, dt * 1.5)
                    o.prm.dt = dt
            else:
                it_in_step = 0
        elif it_in_step >= 8:
            U, P, a, b, w, t = saved
            dt = max(dt / 2, dt0 / 1024)
            o.prm.dt = dt
            o.set_state(U, P, a, b, w, t)
            it_in_step = rounds = 0
            events.append("restart")
        wf = o.opening_at_face_nodes(o.U)
        faces = np.nonzero(m.face_crackable & ((o.alpha > 0) | (o.beta > 0)))[0]
        p_idx = np.nonzero(o.P != 0.0)[0]
        rec = {"k": k, "du_rel": rep["du_rel"], "dp_rel": rep["dp_rel"], "converged": bool(rep["converged"]),
               "events": events, "n_alpha": int(o.alpha.sum()), "n_beta": int(o.beta.sum()), "dt": dt,
               "t": o.t, "gmres_iters": solve.last["iters"], "lin_rel_res": solve.last["rel_res"],
               "U": o.U[u_idx].tolist(), "P_index": p_idx.tolist(), "P": o.P[p_idx].tolist(),
               "w_faces": faces.tolist(), "w": wf[faces].tolist(),
               "U_inf": float(np.abs(o.U).max()), "P_inf": float(np.abs(o.P).max()),
               "w_inf": float(np.abs(wf[crack_faces]).max())}
        out["iters"].append(rec)
        print(f"iter {k}: du={rep['du_rel']:.3e} dp={rep['dp_rel']:.3e} conv={rep['converged']} {events} "
              f"gmres={solve.last['iters']} res={solve.last['rel_res']:.1e} {time.time() - t0:.0f}s", flush=True)
        with open(args.out + ".tmp", "w") as f:
            json.dump(out, f)
        os.replace(args.out + ".tmp", args.out)


if __name__ == "__main__":
    main()
