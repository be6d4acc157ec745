"""The paper's cost model (Sec. 4) against values worked out by hand and
against the bound the paper states (Omega <= A).  CPU only."""
import itertools
import math

import pytest

from paper_2206_02255_gb300 import costmodel as cm


def test_tau():
    assert cm.tau(1024, 16, 2, 32) == pytest.approx(1.0)
    assert cm.tau(1024, 16, 2, 8) == pytest.approx(3.0)
    assert cm.tau(65536, 16, 4, 16) == pytest.approx(4.0)


def test_work_p0_is_one_query_and_one_fill():
    # P = 0: level 0 only, every initial region queried (4nA/g each, G of
    # them) and filled (n^2/G each): W = 4 n A g + n^2
    n, g, r, B, A = 1024, 16, 2, 8, 512
    assert cm.work_ssd(n, g, r, B, 0.0, A, 10.0) == pytest.approx(4 * n * A * g + n * n)


def test_work_p1_is_the_full_tree():
    # P = 1, tau = 3: levels 0 and 1 query and split every region, then the
    # last level computes every pixel:
    #   (256A + lam A) 256 + (128A + lam A) 1024 + n^2 A
    n, g, r, B, A, lam = 1024, 16, 2, 8, 512, 10.0
    want = (256 * A + lam * A) * 256 + (128 * A + lam * A) * 1024 + n * n * A
    assert cm.work_ssd(n, g, r, B, 1.0, A, lam) == pytest.approx(want)


def test_omega_is_bounded_by_A():
    # the paper's bound: subdivision can save at most the dwell work A per pixel
    for n, g, r, k, P, A, lam in itertools.product([1024, 16384], [2, 16], [2, 4], [1, 2, 3],
                                                   [0.0, 0.3, 0.7, 1.0], [64, 2048],
                                                   [0.0, 100.0]):
        B = n // (g * r ** k)
        if B < 1 or g * B * r ** k != n:
            continue
        assert cm.omega(n, g, r, B, P, A, lam) <= A * (1 + 1e-12)


def test_time_exhaustive_by_hand():
    # ceil(1024^2 / (152 * 128)) = ceil(53.89...) = 54 rounds of A
    assert cm.time_exhaustive(1024, 512, 152, 128) == 54 * 512


def test_times_reduce_at_p1_and_p0():
    n, g, r, B, A, lam, q, c = 4096, 8, 2, 64, 256, 5.0, 16, 64
    # P = 0: SBR is level 0's query plus the fill, one region per block:
    # (ceil(4n/(g c)) A + ceil(n^2/(G c))) ceil(G/q)
    G = g * g
    want = (math.ceil(4 * n / (g * c)) * A + math.ceil(n * n / (G * c))) * math.ceil(G / q)
    assert cm.time_sbr(n, g, r, B, 0.0, A, lam, q, c) == pytest.approx(want)
    # MBR at P = 0 is the query by blocks plus the fill spread over q c cores
    want = math.ceil(4 * n / (g * c)) * math.ceil(G / q) * A + math.ceil(n * n / (q * c))
    assert cm.time_mbr(n, g, r, B, 0.0, A, lam, q, c) == pytest.approx(want)


def test_optimum_search_space_and_monotone_in_dwell():
    best = cm.optimum(16384, 2048, 0.5, 10.0, scheme="sbr")
    v, g, r, B = best
    assert g in cm.POW2 and r in cm.POW2 and B in cm.POW2 and g * B <= 16384
    # more dwell per pixel never makes the optimal time smaller
    assert cm.optimum(16384, 4096, 0.5, 10.0, scheme="sbr")[0] >= v


def test_estimate_p_from_counts():
    st = {"regions_per_level": [256, 2720, 27792], "subdivisions_per_level": [170, 1737, 0]}
    assert cm.estimate_p(st) == pytest.approx((170 + 1737) / (256 + 2720))


def test_level_terms_by_hand():
    # n = 64, g = 2, r = 2: level sides 32, 16; q = 4, c = 32, A = 10
    t = cm.level_terms(64, 2, 2, 10.0, 4, 32, regions=[4, 8], subdivs=[2, 0], leaves=3, levels=2)
    # level 0: s = 32, P = 1/2, waves = 1: ceil(128/32) 10 + 0.5 ceil(1024/32) = 40 + 16; b = 0.5 * 10
    assert t[0] == pytest.approx((56.0, 5.0))
    # level 1: s = 16, P = 0, waves = 2: (ceil(64/32) 10 + ceil(256/32)) 2 = (20 + 8) 2
    assert t[1] == pytest.approx((56.0, 0.0))
    # last pass: s_L = 16: 10 ceil(256/32) ceil(3/4) = 80
    assert t[2] == pytest.approx((80.0, 0.0))


def test_fit_lambda_recovers_planted_values():
    terms = [(56.0, 5.0), (120.0, 20.0), (300.0, 11.0), (80.0, 0.0)]
    kappa, lam = 0.002, 7.5
    ms = [kappa * (a + lam * b) for a, b in terms]
    k, l = cm.fit_lambda(ms, terms)
    assert k == pytest.approx(kappa) and l == pytest.approx(lam)


def test_fit_lambda_clamps_negative_lambda():
    terms = [(10.0, 5.0), (20.0, 5.0), (30.0, 0.0)]
    ms = [1.0, 2.0, 3.5]  # no subdivision cost at all: lambda must not go negative
    k, l = cm.fit_lambda(ms, terms)
    assert l >= 0.0 and k > 0.0
