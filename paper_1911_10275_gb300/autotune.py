"""Measured choice of the solver's shape knobs per problem class: the
block-Jacobi subdomain size G (elements per ILU(0) block: larger blocks cut
GMRES iterations but deepen the level schedule of the triangular solves) and
the GMRES restart length m (longer cycles cut iterations but lengthen the
Gram-Schmidt sweeps).  Each candidate runs the same Newton iterations from the
same state on the GPU; the fastest wins.  Classes are (dimension, precision,
log2 of the unknown count), so one tuning run covers every instance of
similar size in a sweep or a request stream."""
from __future__ import annotations

import math
import time

CANDIDATES = tuple((G, m) for G in (8, 16, 32) for m in (60, 90))


def size_class(wl, precision):
    from . import hf_mesh_sizes
    nu, np_ = hf_mesh_sizes(wl.mesh)
    return (wl.mesh.dim, precision, int(round(math.log2(max(nu + np_, 2)))))


def measure(wl, precision, G, m, base, newton_iters=2, stream=None):
    """Seconds per Newton iteration with (G, m), after one untimed iteration;
    the state is reset to the seed before each candidate."""
    from . import HFMesh
    g = HFMesh.from_mesh(wl.mesh, stream=stream)
    try:
        inj, wts = wl.injection()
        g.hf_set_material(wl.E, wl.nu, wl.sigma_c, wl.delta_c, wl.b_stab)
        g.hf_set_injection(wl.mu, wl.Q0, inj, wts, wl.delta_f, wl.dt, 0.0, True, wl.fluid_length)
        g.hf_set_solver(**{**base, "precision": precision, "jacobi_block": G, "restart": m})
        g.hf_set_state(*wl.seed())
        g.hf_newton_step()
        t0 = time.perf_counter()
        its = 0
        for _ in range(newton_iters):
            r = g.hf_newton_step()
            its += 1
            if not r["lin_converged"]:
                return math.inf
        return (time.perf_counter() - t0) / its
    finally:
        g.close()


class Tuner:
    """Caches the fastest (G, m) per size class; tune() measures a class the
    first time one of its workloads is seen."""

    def __init__(self, base=None, candidates=CANDIDATES, newton_iters=2):
        self.base = dict(base or {"rtol": 1e-8, "inner_rtol": 1e-3, "max_iters": 3000, "newton_tol": 1e-8,
                                  "use_graphs": 1, "reorth": 1, "coarse": 1})
        self.candidates = tuple(candidates)
        self.newton_iters = newton_iters
        self.best = {}
        self.timings = {}

    def tune(self, wl, precision="mixed"):
        key = size_class(wl, precision)
        if key not in self.best:
            t = {c: measure(wl, precision, c[0], c[1], self.base, self.newton_iters) for c in self.candidates}
            self.timings[key] = t
            self.best[key] = min(t, key=lambda c: (t[c], c))
        return self.best[key]

    def solver_for(self, wl, precision="mixed"):
        G, m = self.tune(wl, precision)
        return {**self.base, "precision": precision, "jacobi_block": G, "restart": m}

    def report(self):
        return {f"{k[0]}d/{k[1]}/2^{k[2]}": {"G": v[0], "restart": v[1],
                                              "ms_per_newton": round(1000 * self.timings[k][v], 3)}
                for k, v in self.best.items()}
