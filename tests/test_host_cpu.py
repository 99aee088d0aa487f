"""Host-side logic without a GPU: unknown counts and the device-memory bound
computed by the library from a descriptor, the replica split of independent
instances (with a two-rank gloo group), the serving client's bookkeeping and
the request generators."""
import math
import os
import socket

import numpy as np
import pytest

from hf_inputs import kgd_2d, penny_3d, sweep_instances, serving_requests
from _setup import oracle_for


@pytest.mark.parametrize("make", [lambda: kgd_2d(n=8), lambda: kgd_2d(n=6, crackable="all"),
                                  lambda: penny_3d(n=4, crackable="plane"), lambda: penny_3d(n=2)])
def test_mesh_sizes_match_the_oracle(make):
    from paper_1911_10275_gb300 import hf_mesh_sizes
    wl = make()
    o = oracle_for(wl)
    assert hf_mesh_sizes(wl.mesh) == (o.Nu, o.Np)


def test_device_bound_grows_with_the_mesh_and_covers_the_matrices():
    from paper_1911_10275_gb300 import hf_estimate_device_bytes
    prev = 0
    for n in (8, 16, 32):
        m = kgd_2d(n=n).mesh
        b = hf_estimate_device_bytes(m, jacobi_block=32)
        ne = m.n_elems
        # J in FP64 and FP32 plus both ILU record sets: 4 (12x12 + 3 * 12x6) values per element
        assert b >= ne * (144 + 216) * (8 + 4) * 2
        assert b > prev
        prev = b
    m = penny_3d(n=4).mesh
    assert hf_estimate_device_bytes(m, jacobi_block=8) >= hf_estimate_device_bytes(m, jacobi_block=64)
    assert hf_estimate_device_bytes(m, restart=90) > hf_estimate_device_bytes(m, restart=30)


def test_partition_is_balanced_complete_and_deterministic():
    from paper_1911_10275_gb300.replicas import partition
    rng = np.random.default_rng(0)
    costs = rng.lognormal(size=101)
    for world in (1, 2, 3, 8):
        parts = partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(101))
        loads = [costs[p].sum() for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest item
        assert max(loads) <= np.mean(loads) + costs.max() + 1e-12
        assert parts == partition(list(costs), world)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, costs, q):
    import torch.distributed as dist
    from paper_1911_10275_gb300.replicas import my_share, max_over_ranks, sum_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = my_share(costs, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    slowest = max_over_ranks(10.0 + rank)
    total = sum_over_ranks(len(mine))
    dist.destroy_process_group()
    q.put((rank, got, slowest, total))


def test_replicas_on_two_gloo_ranks():
    """Each rank takes its own share of the instances with no exchange; the
    shares agree across ranks, cover every instance once, and the job time is
    the slowest rank's."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    costs = [float(c) for c in np.random.default_rng(1).uniform(1, 5, size=37)]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == out[1][1]
    shares = out[0][1]
    assert sorted(shares[0] + shares[1]) == list(range(37))
    assert out[0][2] == out[1][2] == 11.0
    assert out[0][3] == out[1][3] == 37.0


def test_latency_summary_percentiles():
    from paper_1911_10275_gb300.serving import latency_summary
    recs = [{"status": 0, "latency": (i + 1) / 1000.0, "t_submit": 0.0, "t_done": (i + 1) / 1000.0,
             "newton_iters": 3, "gmres_iters": 10, "cutbacks": 0} for i in range(100)]
    recs.append({"status": -4, "latency": 9.0, "t_submit": 0.0, "t_done": 0.05, "newton_iters": 0,
                 "gmres_iters": 0, "cutbacks": 10})
    s = latency_summary(recs)
    assert s["completed"] == 100 and s["failed"] == 1
    assert abs(s["p50_ms"] - 50.5) < 1e-9 and abs(s["p99_ms"] - 99.01) < 1e-9
    assert abs(s["throughput_req_s"] - 1000.0) < 1e-9


def test_generators_are_seeded_and_in_range():
    a = sweep_instances(16)
    b = sweep_instances(16)
    assert [w.name for w in a] == [w.name for w in b]
    for w in a:
        assert 1000 / 1.2 <= w.mesh.n_elems <= 50000 * 1.2
        assert 5e9 <= w.E <= 50e9 and 0.1e6 <= w.K_Ic <= 3e6 and 1e-3 <= w.mu <= 1.0 and 1e-4 <= w.Q0 <= 1e-2
    t, r = serving_requests(40, rate=200.0, kgd_n=(50, 60), penny_n=(7, 8))
    assert np.all(np.diff(t) > 0) and abs(np.mean(np.diff(t)) - 1 / 200.0) < 2.5e-3
    dims = {w.mesh.dim for w in r}
    assert dims == {2, 3}


def test_drawn_instances_are_toughness_consistent_and_balanced():
    """The seed of a drawn instance sits at its toughness (K_I = K_Ic from the
    plane-strain or penny formula), its opening is the elastic one of that
    pressure, the cohesive length spans four elements, and the fluid rows
    are scaled to c = E dt / h at the seed opening."""
    import math
    from hf_inputs import toughness_consistent, balanced_fluid_length
    for wl in (kgd_2d(n=20, K_Ic=0.3e6, E=9e9, mu=0.2), penny_3d(n=6, K_Ic=2e6, E=30e9, mu=1e-3)):
        t = toughness_consistent(wl, sigma_c_max=1e6)
        a, h = t.seed_radius, t.mesh.length / t.mesh.n
        Ep = t.E / (1 - t.nu ** 2)
        if t.mesh.dim == 2:
            assert abs(t.p0 * math.sqrt(math.pi * a) - t.K_Ic) < 1e-9 * t.K_Ic
            assert abs(t.w0 - 4 * t.p0 * a / Ep) < 1e-12 * t.w0
        else:
            assert abs(2 * t.p0 * math.sqrt(a / math.pi) - t.K_Ic) < 1e-9 * t.K_Ic
            assert abs(t.w0 - 8 * t.p0 * a / (math.pi * Ep)) < 1e-12 * t.w0
        assert t.sigma_c <= 1e6 and t.K_Ic ** 2 / t.sigma_c ** 2 >= 4 * h * (1 - 1e-12)
        c = 12 * t.mu * (t.fluid_length / t.w0) ** 3
        assert abs(c - t.E * t.dt / h) < 1e-9 * c
        assert t.fluid_length == balanced_fluid_length(t)
    assert kgd_2d(n=8).fluid_length == kgd_2d(n=8).mesh.length


def test_autotuner_picks_the_fastest_candidate_once_per_size_class(monkeypatch):
    """The tuner measures each candidate once per (dimension, precision,
    log2 unknowns) class and hands every workload of the class the fastest;
    a candidate whose solve did not converge (infinite time) never wins."""
    import math
    from paper_1911_10275_gb300 import autotune
    calls = []

    def fake_measure(wl, precision, G, m, base, newton_iters=2, stream=None):
        calls.append((wl.mesh.n, G, m))
        return math.inf if (G, m) == (8, 60) else 1.0 / G + m / 1000.0
    monkeypatch.setattr(autotune, "measure", fake_measure)
    t = autotune.Tuner()
    a, b, c = kgd_2d(n=18), kgd_2d(n=20), kgd_2d(n=40)
    assert autotune.size_class(a, "mixed") == autotune.size_class(b, "mixed") != autotune.size_class(c, "mixed")
    best = t.tune(a, "mixed")
    assert best == min((cand for cand in autotune.CANDIDATES if cand != (8, 60)), key=lambda q: 1.0 / q[0] + q[1] / 1000.0)
    n_first = len(calls)
    assert n_first == len(autotune.CANDIDATES)
    assert t.tune(b, "mixed") == best and len(calls) == n_first        # same class: cached
    t.tune(c, "mixed")
    assert len(calls) == 2 * n_first                                    # new class: measured
    opts = t.solver_for(a, "mixed")
    assert opts["jacobi_block"] == best[0] and opts["restart"] == best[1] and opts["precision"] == "mixed"
    assert set(t.report()) == {"2d/mixed/2^%d" % autotune.size_class(w, "mixed")[2] for w in (a, c)}


def test_toughness_vertex_size_bound_against_the_opening_profiles():
    """The size bound of the instance generators (hf_inputs.workloads):
    at t = 0 it returns the seed's size; for t > 0 the crack it returns,
    held at K_I = K_Ic, holds exactly V0 + Q0 t, with the volumes integrated
    numerically from Sneddon's plane-strain opening 4 p / E' sqrt(l^2 - x^2)
    and the penny's 8 p R / (pi E') sqrt(1 - r^2 / R^2), p from Irwin's
    K_I = p sqrt(pi l) and the penny's K_I = 2 p sqrt(R / pi)."""
    import dataclasses
    from hf_inputs.workloads import toughness_vertex_size, crack_stays_inside, toughness_consistent
    from scipy.integrate import quad

    def volume_2d(l, K, Ep):
        p = K / math.sqrt(math.pi * l)
        return quad(lambda x: 4 * p / Ep * math.sqrt(l * l - x * x), -l, l)[0]

    def volume_3d(R, K, Ep):
        p = K * math.sqrt(math.pi) / (2 * math.sqrt(R))
        return quad(lambda r: 2 * math.pi * r * 8 * p * R / (math.pi * Ep) * math.sqrt(1 - (r / R) ** 2), 0, R)[0]

    for wl, vol in ((toughness_consistent(kgd_2d(n=20, length=40.0, E=17e9, K_Ic=1.5e6, Q0=1e-3)), volume_2d),
                    (toughness_consistent(penny_3d(n=12, crackable="plane", E=10e9, K_Ic=1e6, Q0=1e-2)), volume_3d)):
        Ep = wl.E / (1 - wl.nu ** 2)
        a = wl.seed_radius
        assert toughness_vertex_size(wl, 0.0) == pytest.approx(a, rel=1e-12)
        v0 = vol(a, wl.K_Ic, Ep)
        for t in (0.5, 3.0, 20.0):
            size = toughness_vertex_size(wl, t)
            assert vol(size, wl.K_Ic, Ep) == pytest.approx(v0 + wl.Q0 * t, rel=1e-9)
        # the filter: inside for a short run, outside once the bound passes 0.6 of the half-domain
        assert crack_stays_inside(wl, 0)
        far = dataclasses.replace(wl, Q0=wl.Q0 * 1e6)
        assert not crack_stays_inside(far, 1)
