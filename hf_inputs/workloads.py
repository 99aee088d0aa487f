"""Workload definitions: the synthetic stand-ins for the paper's KGD and
penny-shaped fracture tests (meshes from hf_inputs.mesh plus physical
parameters).  Input data only: both the CUDA library and the oracle receive
these numbers.  The cohesive length delta_c follows from G_c = sigma_c
delta_c / 2 (the relation stated beside Eq. tsl) with G_c = K_Ic^2 / E'."""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .mesh import Mesh, square_p2, cube_p2, pressure_nodes, seed_state, batch_instances


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    E: float
    nu: float
    K_Ic: float
    sigma_c: float
    mu: float
    Q0: float
    dt: float
    b_stab: float = 10.0
    steps: int = 10
    seed_radius: float = 0.0
    w0: float = 1e-3
    p0: float = 1e6
    L_ref: float = 0.0      # length L of the fluid-row scaling c = 12 mu (L / max w)^3; 0: the domain side

    @property
    def fluid_length(self):
        return self.L_ref if self.L_ref > 0 else self.mesh.length

    @property
    def G_c(self):
        return self.K_Ic ** 2 * (1.0 - self.nu ** 2) / self.E

    @property
    def delta_c(self):
        return 2.0 * self.G_c / self.sigma_c

    @property
    def delta_f(self):
        return self.delta_c      # fluid enters fully failed facets

    def injection(self):
        pn = pressure_nodes(self.mesh)
        i = int(np.nonzero(pn == self.mesh.center_node)[0][0])
        return [i], [1.0]

    def seed(self):
        return seed_state(self.mesh, self.seed_radius, self.w0, self.p0)


def kgd_2d(n=44, length=100.0, crackable="midline", E=20e9, nu=0.2, K_Ic=1e6, sigma_c=1e6, mu=1e-3,
           Q0=1e-3, dt=1.0, steps=10, seed_cells=2, jitter=0.0, name=None) -> Workload:
    """Plane-strain KGD: square of side `length`, n x n squares of two P2
    triangles, injection at the centre, crack on the midline (or anywhere)."""
    m = square_p2(n, length, crackable=crackable, jitter=jitter)
    h = length / n
    return Workload(name or f"kgd2d_n{n}", m, E, nu, K_Ic, sigma_c, mu, Q0, dt, steps=steps,
                    seed_radius=seed_cells * h * 1.0001, w0=1e-3, p0=1e6)


def penny_3d(n=18, length=50.0, crackable="all", E=10e9, nu=0.25, K_Ic=1e6, sigma_c=0.3e6, mu=1e-2,
             Q0=1e-2, dt=1.0, steps=20, seed_cells=2, name=None) -> Workload:
    """Penny-shaped fracture: cube of side `length`, n^3 cubes of six P2
    tetrahedra, point injection at the centre of the plane z = 0.  sigma_c
    defaults to 0.3 MPa so that the cohesive length E' G_c / sigma_c^2
    (~12 m) spans several elements of the n = 18 mesh (h = 2.8 m)."""
    m = cube_p2(n, length, crackable=crackable)
    h = length / n
    return Workload(name or f"penny3d_n{n}", m, E, nu, K_Ic, sigma_c, mu, Q0, dt, steps=steps,
                    seed_radius=seed_cells * h * 1.0001, w0=2e-3, p0=1e6)


# the configurations the library is measured and tested on
def c1_kgd_toughness():
    return kgd_2d(n=44, name="c1_kgd2d_n44_fp64")


def c2_kgd_viscosity():
    return kgd_2d(n=316, crackable="all", mu=1e-1, K_Ic=0.1e6, steps=50, name="c2_kgd2d_n316_all")


def c3_penny():
    """The penny crack lives in its plane z = 0, as the KGD crack lives on the
    midline: facets off the plane are intact DG interfaces."""
    return penny_3d(n=18, crackable="plane", name="c3_penny3d_n18_mixed")


# ---------------------------------------------------------------- many instances
def _even(x, lo, hi):
    """Even integer nearest x within [lo, hi] (bounds rounded inwards to even)."""
    lo = lo + (lo % 2)
    hi = hi - (hi % 2)
    n = int(round(x / 2.0)) * 2
    return max(lo, min(hi, n))


def _log_uniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def sample_parameters(rng):
    """E, K_Ic, mu, Q0 drawn log-uniformly over the ranges of the batched
    sweep: E in [5, 50] GPa, K_Ic in [0.1, 3] MPa m^1/2, mu in [1e-3, 1] Pa s,
    Q0 in [1e-4, 1e-2] (m^2/s in 2D, m^3/s in 3D)."""
    return {"E": _log_uniform(rng, 5e9, 50e9), "K_Ic": _log_uniform(rng, 0.1e6, 3e6),
            "mu": _log_uniform(rng, 1e-3, 1.0), "Q0": _log_uniform(rng, 1e-4, 1e-2)}


def balanced_fluid_length(wl: Workload, w=None) -> float:
    """Length L for which the fluid-row scaling c = 12 mu (L / w)^3 equals
    E dt / h at opening w (the seed opening by default): the factor that
    brings the pressure rows of the Newton system to the size of the
    displacement rows (force ~ E h^(d-2) w against flux ~ c w h^(d-1) / dt)."""
    h = wl.mesh.length / wl.mesh.n
    w = wl.w0 if w is None else w
    return w * (wl.E * wl.dt / (12.0 * wl.mu * h)) ** (1.0 / 3.0)


def toughness_consistent(wl: Workload, sigma_c_max=1e6, zone_elems=4.0) -> Workload:
    """The same instance with a seed and a cohesive strength that its
    parameters can support, for draws over wide parameter ranges:

    * the seed pressure p0 is the one at which the seed crack (half-length or
      radius a) is at its toughness: K_I = K_Ic with K_I = p sqrt(pi a) for the
      plane-strain crack and 2 p sqrt(a / pi) for the penny crack;
    * the seed opening is the static elastic opening of that pressure at the
      centre: 4 p0 a / E' in plane strain, 8 p0 a / (pi E') for the penny
      (E' = E / (1 - nu^2));
    * sigma_c is lowered below sigma_c_max where needed so that the cohesive
      length E' G_c / sigma_c^2 = K_Ic^2 / sigma_c^2 spans zone_elems elements;
    * the length L of the fluid-row scaling from balanced_fluid_length.
    """
    m = wl.mesh
    h = m.length / m.n
    a = wl.seed_radius
    Ep = wl.E / (1.0 - wl.nu ** 2)
    if m.dim == 2:
        p0 = wl.K_Ic / math.sqrt(math.pi * a)
        w0 = 4.0 * p0 * a / Ep
    else:
        p0 = wl.K_Ic * math.sqrt(math.pi) / (2.0 * math.sqrt(a))
        w0 = 8.0 * p0 * a / (math.pi * Ep)
    sigma_c = min(sigma_c_max, wl.K_Ic / math.sqrt(zone_elems * h))
    out = dataclasses.replace(wl, p0=p0, w0=w0, sigma_c=sigma_c)
    return dataclasses.replace(out, L_ref=balanced_fluid_length(out))


def toughness_vertex_size(wl: Workload, t: float) -> float:
    """Half-length (2D) or radius (3D) at time t of the seed crack grown as
    the toughness vertex with no leak-off: the volume V0 + Q0 t held at
    K_I = K_Ic (plane strain: V = 2 sqrt(pi) K_Ic l^(3/2) / E'; penny:
    V = 8 sqrt(pi) K_Ic R^(5/2) / (3 E')), V0 the seed's volume at its
    toughness.  For the same volume a viscous crack is shorter, so this
    bounds the crack's size from above."""
    Ep = wl.E / (1.0 - wl.nu ** 2)
    a = wl.seed_radius
    if wl.mesh.dim == 2:
        return (a ** 1.5 + Ep * wl.Q0 * t / (2.0 * math.sqrt(math.pi) * wl.K_Ic)) ** (2.0 / 3.0)
    return (a ** 2.5 + 3.0 * Ep * wl.Q0 * t / (8.0 * math.sqrt(math.pi) * wl.K_Ic)) ** 0.4


def crack_stays_inside(wl: Workload, steps: int, frac: float = 0.6) -> bool:
    """True when the crack's size bound after `steps` steps of dt stays
    within frac of the half-domain: the paper's tests keep the domain much
    larger than the crack, and a draw whose crack would reach the boundary
    within the run is not an instance of them."""
    return toughness_vertex_size(wl, steps * wl.dt) <= frac * 0.5 * wl.mesh.length


def sweep_instances(count=256, seed=191110275, ne_range=(1000, 50000), steps=10, mesh_cache=None):
    """Batched 2D KGD sweep: `count` independent plane-strain instances with
    the draws of batch_instances (element count, E, K_Ic, mu, Q0 log-uniform),
    nu = 0.2, sigma_c = 1 MPa at most, crack on the midline, seed and sigma_c
    from toughness_consistent; a draw whose crack could reach the boundary
    within the run (crack_stays_inside) is replaced by a fresh draw of E,
    K_Ic, mu and Q0.  Meshes of equal n are shared through mesh_cache (a
    dict)."""
    cache = {} if mesh_cache is None else mesh_cache
    out = []
    draws = batch_instances(count, seed, ne_range)
    rng = np.random.Generator(np.random.PCG64(seed + 1))   # redraws of E, K_Ic, mu, Q0
    for i, d in enumerate(draws):
        n = d["n"]
        key = ("kgd", n)
        if key not in cache:
            cache[key] = square_p2(n, 100.0, crackable="midline")
        h = 100.0 / n
        prm = {k: d[k] for k in ("E", "K_Ic", "mu", "Q0")}
        for _ in range(100):
            wl = toughness_consistent(
                Workload(f"sweep{i}_kgd2d_n{n}", cache[key], prm["E"], 0.2, prm["K_Ic"], 1e6, prm["mu"], prm["Q0"],
                         1.0, steps=steps, seed_radius=2 * h * 1.0001, w0=1e-3, p0=1e6))
            if crack_stays_inside(wl, steps):
                break
            prm = sample_parameters(rng)
        out.append(wl)
    return out


def serving_requests(count=2000, rate=200.0, seed=191110275, kgd_n=(50, 316), penny_n=(7, 22), steps=5,
                     mesh_cache=None):
    """Poisson stream of solve requests: exponential inter-arrival times of
    mean 1/rate, half plane-strain KGD (n x n squares of two P2 triangles,
    n in kgd_n), half penny-shaped (n^3 cubes of six P2 tetrahedra, n in
    penny_n, crack plane z = 0), parameters from sample_parameters (nu = 0.2
    for KGD, 0.25 for the penny), `steps` time steps each from the seed
    state; seed and sigma_c (at most 1 MPa for KGD, 0.3 MPa for the penny)
    from toughness_consistent; a draw whose crack could reach the boundary
    within the request (crack_stays_inside) is replaced by a fresh draw.
    Returns (arrival times in s, workloads)."""
    rng = np.random.default_rng(seed)
    cache = {} if mesh_cache is None else mesh_cache
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        prm = sample_parameters(rng)
        kgd = rng.uniform() < 0.5
        if kgd:
            n = _even(math.exp(rng.uniform(math.log(kgd_n[0]), math.log(kgd_n[1]))), kgd_n[0], kgd_n[1])
            key = ("kgd", n)
            if key not in cache:
                cache[key] = square_p2(n, 100.0, crackable="midline")
            h = 100.0 / n

            def make(prm):
                return toughness_consistent(
                    Workload(f"req{i}_kgd2d_n{n}", cache[key], prm["E"], 0.2, prm["K_Ic"], 1e6, prm["mu"], prm["Q0"],
                             1.0, steps=steps, seed_radius=2 * h * 1.0001, w0=1e-3, p0=1e6))
        else:
            n = _even(math.exp(rng.uniform(math.log(penny_n[0]), math.log(penny_n[1]))), penny_n[0] + 1, penny_n[1])
            key = ("penny", n)
            if key not in cache:
                cache[key] = cube_p2(n, 50.0, crackable="plane")
            h = 50.0 / n

            def make(prm):
                return toughness_consistent(
                    Workload(f"req{i}_penny3d_n{n}", cache[key], prm["E"], 0.25, prm["K_Ic"], 0.3e6, prm["mu"],
                             prm["Q0"], 1.0, steps=steps, seed_radius=2 * h * 1.0001, w0=2e-3, p0=1e6),
                    sigma_c_max=0.3e6)
        wl = make(prm)
        for _ in range(100):
            if crack_stays_inside(wl, steps):
                break
            wl = make(sample_parameters(rng))
        out.append(wl)
    return t, out
