"""Workload definitions: the synthetic stand-ins for the paper's KGD and
penny-shaped fracture tests (meshes from hf_inputs.mesh plus physical
parameters).  Input data only: both the CUDA library and the oracle receive
these numbers.  The cohesive length delta_c follows from G_c = sigma_c
delta_c / 2 (the relation stated beside Eq. tsl) with G_c = K_Ic^2 / E'."""
from __future__ import annotations

import dataclasses

import numpy as np

from .mesh import Mesh, square_p2, cube_p2, pressure_nodes, seed_state


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
