"""Pins of the oracle's FMM bandwidth and spherical grid (Sec. II.A, after Eq. 4)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


@pytest.mark.parametrize("L", [1, 5, 13, 39])
def test_gauss_legendre_exact_for_polynomials(L):
    g = grid.make_grid(L)
    x = np.cos(g.theta)
    assert abs(g.w_theta.sum() - 2.0) < 1e-13
    for m in range(2 * L + 2):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(g.w_theta * x ** m) - exact) < 1e-12
    # theta ascending in (0, pi)
    assert np.all(np.diff(g.theta) > 0) and g.theta[0] > 0 and g.theta[-1] < math.pi


@pytest.mark.parametrize("rule", ["2L+1", "2L+2"])
def test_uniform_phi_exact_for_harmonics(rule):
    L = 9
    g = grid.make_grid(L, rule)
    for m in range(-(g.n_phi - 1), g.n_phi):
        s = np.sum(g.w_phi * np.exp(1j * m * g.phi))
        assert abs(s - (2 * math.pi if m == 0 else 0.0)) < 1e-12


def test_direction_triads_orthonormal_right_handed():
    g = grid.make_grid(7)
    for a, b in ((g.khat, g.khat), (g.theta_hat, g.theta_hat), (g.phi_hat, g.phi_hat)):
        assert np.allclose(np.einsum("ic,ic->i", a, b), 1.0, atol=1e-14)
    for a, b in ((g.khat, g.theta_hat), (g.khat, g.phi_hat), (g.theta_hat, g.phi_hat)):
        assert np.allclose(np.einsum("ic,ic->i", a, b), 0.0, atol=1e-14)
    assert np.allclose(np.cross(g.theta_hat, g.phi_hat), g.khat, atol=1e-14)
    # theta-fastest flattening, i = i_theta + n_theta i_phi
    i = 3 + g.n_theta * 5
    assert np.allclose(g.khat[i], [math.sin(g.theta[3]) * math.cos(g.phi[5]),
                                   math.sin(g.theta[3]) * math.sin(g.phi[5]),
                                   math.cos(g.theta[3])])


def test_sphere_rule_integrates_plane_wave():
    """int exp(j k khat.d) dOmega = 4 pi sin(k|d|)/(k|d|): band-limited, exact once L > k|d|."""
    g = grid.make_grid(30)
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.normal(size=3)
        d *= 2.0 / np.linalg.norm(d)
        kd = 2 * math.pi * 2.0
        s = np.sum(g.weights * np.exp(1j * 2 * math.pi * g.khat @ d))
        assert abs(s - 4 * math.pi * math.sin(kd) / kd) < 1e-12
    assert abs(g.weights.sum() - 4 * math.pi) < 1e-12


def test_bandwidth_matches_paper_tables():
    gold = json.load(open(GOLDEN))["bandwidth"]
    for row in gold:
        assert grid.bandwidth(2 * math.pi, row["box"], row["digits"]) == row["L"], row["cite"]


def test_bandwidth_is_monotone_and_exceeds_kd():
    k = 2 * math.pi
    prev = 0
    for a in (0.25, 0.5, 1.0, 2.0, 4.0):
        L = grid.bandwidth(k, a, 6)
        assert L > k * a * math.sqrt(3)
        assert L > prev
        prev = L
    assert grid.bandwidth(k, 1.0, 3) < grid.bandwidth(k, 1.0, 6)
