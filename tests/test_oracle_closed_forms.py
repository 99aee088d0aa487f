"""Pins of the closed forms in oracle/kgd.py against numbers the paper prints
(tests/golden/paper_numbers.txt, each line cited to its section/table)."""
import math
import os

import pytest

from oracle import kgd

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")


def _gold():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


G = _gold()
E, NU, Q0_2D, GC_2D = 17e9, 0.2, 1e-3, 120.0


def test_kgd_table_viscosity_regime():
    kic = kgd.kic_from_gc(GC_2D, E, NU)
    K = kgd.kgd_K(E, NU, G["kgd_visc_mu"], Q0_2D, kic)
    M = kgd.kgd_M(E, NU, G["kgd_visc_mu"], Q0_2D, kic)
    assert K == pytest.approx(G["kgd_visc_K"], abs=0.006)
    assert M == pytest.approx(G["kgd_visc_M"], abs=0.5)
    assert K < 0.70   # viscosity-dominated threshold (Sec. 4.1)


def test_kgd_table_toughness_regime():
    kic = kgd.kic_from_gc(GC_2D, E, NU)
    K = kgd.kgd_K(E, NU, G["kgd_tough_mu"], Q0_2D, kic)
    M = kgd.kgd_M(E, NU, G["kgd_tough_mu"], Q0_2D, kic)
    assert K == pytest.approx(G["kgd_tough_K"], abs=0.06)
    assert M == pytest.approx(G["kgd_tough_M"], abs=0.00006)
    assert K > 4.13   # toughness-dominated threshold (Sec. 4.1)
    assert K == pytest.approx(M ** -0.25, rel=1e-12)


def test_penny_table_and_regime_times():
    mu, Q0, Gc = 0.15, 0.03, 100.0
    kic = kgd.kic_from_gc(Gc, E, NU)
    t0 = G["penny_t0"]
    K = kgd.penny_K(E, NU, mu, Q0, kic, t0)
    M = kgd.penny_M(E, NU, mu, Q0, kic, t0)
    assert K == pytest.approx(G["penny_K"], abs=0.006)
    assert M == pytest.approx(G["penny_M"], abs=0.06)
    assert M == pytest.approx(K ** (-18.0 / 5.0), rel=1e-12)
    t_v = kgd.penny_time_for_K(E, NU, mu, Q0, kic, 0.37)
    t_k = kgd.penny_time_for_K(E, NU, mu, Q0, kic, 3.5)
    assert t_v == pytest.approx(G["penny_visc_until"], rel=0.01)
    assert t_k == pytest.approx(G["penny_tough_after"], rel=0.05)


def test_m_vertex_scaling_consistent_with_propagation_numbers():
    """l = gamma0 Q0^1/2 E'^1/6 t^2/3 / mu'^1/6: the two (t, l) pairs of the
    propagation test imply the same gamma0 within the paper's 'approximately'."""
    mu = G["kgd_visc_mu"]
    g_a = kgd.m_vertex_gamma0(E, NU, mu, Q0_2D, G["prop_t0"], G["prop_l0"])
    g_b = kgd.m_vertex_gamma0(E, NU, mu, Q0_2D, G["prop_t_final"], G["prop_l_final"])
    assert 0.55 < g_a < 0.65 and 0.55 < g_b < 0.66
    assert g_a == pytest.approx(g_b, rel=0.08)


def test_k_vertex_closed_form_volume_balance():
    """Toughness vertex: Sneddon volume 2 pi p l^2/E' with p = K/sqrt(pi l)
    equals Q0 t (global balance, no leak-off) and K_I = p sqrt(pi l) = K_Ic."""
    kic = 1e6
    for t in (1.0, 10.0, 100.0):
        l = kgd.k_vertex_length(E, NU, Q0_2D, kic, t)
        p = kgd.k_vertex_pressure(kic, l)
        vol = 2.0 * math.pi * p * l * l / kgd.e_prime(E, NU)
        assert vol == pytest.approx(Q0_2D * t, rel=1e-12)
        assert p * math.sqrt(math.pi * l) == pytest.approx(kic, rel=1e-12)
        # Sneddon profile integrates to the same volume
        n = 20000
        xs = [(-l + (i + 0.5) * 2 * l / n) for i in range(n)]
        v2 = sum(kgd.sneddon_opening(E, NU, p, l, x) for x in xs) * 2 * l / n
        assert v2 == pytest.approx(vol, rel=1e-5)


def test_config_regime_labels():
    """The 2D KGD workload with E=20 GPa, nu=0.2, mu=1e-3, K_Ic=1 MPa sqrt(m),
    Q0=1e-3 falls in the transition band (0.70 < K < 4.13)."""
    K = kgd.kgd_K(20e9, 0.2, 1e-3, 1e-3, 1e6)
    assert 0.70 < K < 4.13
    assert K == pytest.approx(0.989, abs=0.002)


def test_penny_initial_radius_consistent_with_m_vertex():
    """Sec. 4.4 starts the penny crack from the viscosity-regime analytic
    solution with radius 10 m at 17.6 s: R = gamma_m0 (Q0^3 E' t^4/mu')^(1/9)
    then fixes gamma_m0 ~ 0.70, the constant of the zero-toughness radial
    similarity solution (0.6955 in the literature the paper cites)."""
    mu, Q0 = 0.15, 0.03
    g = kgd.penny_m_vertex_gamma(E, NU, mu, Q0, G["penny_t0"], G["penny_R0"])
    assert 0.69 < g < 0.705
    assert g == pytest.approx(0.6955, rel=0.01)
    # R grows as t^(4/9): doubling t multiplies R by 2^(4/9)
    r1 = kgd.penny_m_vertex_radius(E, NU, mu, Q0, 10.0, g)
    r2 = kgd.penny_m_vertex_radius(E, NU, mu, Q0, 20.0, g)
    assert r2 / r1 == pytest.approx(2.0 ** (4.0 / 9.0), rel=1e-12)
