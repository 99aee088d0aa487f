"""Closed forms used to pin the oracle's physics (test infrastructure only).

* Nondimensional toughness and viscosity of the plane-strain (KGD) fracture,
  Sec. 4.1: K = (12 mu Q0 E'^3)^(-1/4) * 8/sqrt(2 pi) * K_Ic and
  M = 12 mu Q0 E'^3 (8/sqrt(2 pi) K_Ic)^(-4); K = M^(-1/4).
  Regimes: viscosity-dominated for K < 0.70, toughness-dominated for K > 4.13.
* Same numbers for the radial (penny) fracture, Sec. 4.4, which depend on t:
  K = (t^2 / ((12 mu)^5 Q0^3 E'^13))^(1/18) * 8/sqrt(2 pi) K_Ic,
  M = 12 mu (Q0^3 E'^13 / t^2)^(1/5) (8/sqrt(2 pi) K_Ic)^(-18/5); M = K^(-18/5).
  Regimes: K < 0.37 viscosity, K > 3.5 toughness.
* Zero-toughness (M-vertex) KGD scaling, Sec. 4 (analytic solution):
  l(t) = gamma0 Q0^(1/2) E'^(1/6) t^(2/3) / mu'^(1/6), mu' = 12 mu.
* Toughness-vertex KGD fracture, derived from Sneddon's opening of a
  pressurised crack, Irwin's K_I = p sqrt(pi l) and the global volume balance
  (Q0 total rate, l half-length, no leak-off):
  V = pi p l^2 / E' * 2 = Q0 t  ->  l(t) = (E' Q0 t / (2 sqrt(pi) K_Ic))^(2/3).
* Sneddon: opening of a crack of half-length l under uniform net pressure p in
  an infinite plane-strain body, w(x) = (4 p / E') sqrt(l^2 - x^2).
* Zero-toughness (M-vertex) radial fracture, Sec. 4.4 (analytic solution of
  the viscosity regime): R(t) = gamma_m0 (Q0^3 E' t^4 / mu')^(1/9), mu' = 12 mu.
"""
import math


def e_prime(E, nu):
    return E / (1.0 - nu * nu)


def kic_from_gc(Gc, E, nu):
    """Plane-strain mode-I toughness K_Ic = sqrt(G_c E') (Irwin)."""
    return math.sqrt(Gc * e_prime(E, nu))


def kgd_K(E, nu, mu, Q0, Kic):
    return (12.0 * mu * Q0 * e_prime(E, nu) ** 3) ** -0.25 * 8.0 / math.sqrt(2.0 * math.pi) * Kic


def kgd_M(E, nu, mu, Q0, Kic):
    return 12.0 * mu * Q0 * e_prime(E, nu) ** 3 * (8.0 / math.sqrt(2.0 * math.pi) * Kic) ** -4


def penny_K(E, nu, mu, Q0, Kic, t):
    Ep = e_prime(E, nu)
    return (t * t / ((12.0 * mu) ** 5 * Q0 ** 3 * Ep ** 13)) ** (1.0 / 18.0) \
        * 8.0 / math.sqrt(2.0 * math.pi) * Kic


def penny_M(E, nu, mu, Q0, Kic, t):
    Ep = e_prime(E, nu)
    return 12.0 * mu * (Q0 ** 3 * Ep ** 13 / (t * t)) ** 0.2 \
        * (8.0 / math.sqrt(2.0 * math.pi) * Kic) ** (-18.0 / 5.0)


def penny_time_for_K(E, nu, mu, Q0, Kic, K_target):
    """Time at which the radial-fracture toughness reaches K_target (K ~ t^(1/9))."""
    K1 = penny_K(E, nu, mu, Q0, Kic, 1.0)
    return (K_target / K1) ** 9


def m_vertex_length(E, nu, mu, Q0, t, gamma0):
    Ep = e_prime(E, nu)
    return gamma0 * Q0 ** 0.5 * Ep ** (1.0 / 6.0) * t ** (2.0 / 3.0) / (12.0 * mu) ** (1.0 / 6.0)


def m_vertex_gamma0(E, nu, mu, Q0, t, length):
    return length / m_vertex_length(E, nu, mu, Q0, t, 1.0)


def k_vertex_length(E, nu, Q0, Kic, t):
    return (e_prime(E, nu) * Q0 * t / (2.0 * math.sqrt(math.pi) * Kic)) ** (2.0 / 3.0)


def k_vertex_pressure(Kic, length):
    return Kic / math.sqrt(math.pi * length)


def sneddon_opening(E, nu, p, length, x):
    return 4.0 * p / e_prime(E, nu) * math.sqrt(max(length * length - x * x, 0.0))


def penny_m_vertex_radius(E, nu, mu, Q0, t, gamma_m0):
    return gamma_m0 * (Q0 ** 3 * e_prime(E, nu) * t ** 4 / (12.0 * mu)) ** (1.0 / 9.0)


def penny_m_vertex_gamma(E, nu, mu, Q0, t, radius):
    return radius / penny_m_vertex_radius(E, nu, mu, Q0, t, 1.0)
