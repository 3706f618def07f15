"""FMM bandwidth and spherical k-space grid (Sec. II.A, text after Eq. 4).

* L = 2kR^s + (2kR^s)^(1/3) * 1.8 * (log10(1/accuracy))^(2/3) (ref. [25]),
  with 2R^s = a sqrt(3) the diameter of the sphere enclosing a box of edge a.
  Readings: d0 = log10(1/accuracy) is the number of accurate digits, and L is
  rounded up to the next integer.  ``L_override`` reproduces other roundings.
* n_theta = L + 1 Gauss-Legendre points in cos(theta), theta ascending.
* n_phi = 2L + 1 uniform points (the paper), or 2(L + 1) (the sphere
  workloads); phi_j = 2 pi j / n_phi, weight 2 pi / n_phi.
* Directions are flattened with theta fastest: i = i_theta + n_theta * i_phi
  (the n_theta x n_phi reshape of Fig. 3b).
* theta_hat = (cos t cos p, cos t sin p, -sin t), phi_hat = (-sin p, cos p, 0),
  so I - k k = theta_hat theta_hat + phi_hat phi_hat.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def bandwidth(k: float, box: float, digits: float) -> int:
    kd = k * box * math.sqrt(3.0)
    return int(math.ceil(kd + 1.8 * digits ** (2.0 / 3.0) * kd ** (1.0 / 3.0)))


def n_phi_of(L: int, rule: str) -> int:
    if rule == "2L+1":
        return 2 * L + 1
    if rule == "2L+2":
        return 2 * L + 2
    raise ValueError(rule)


@dataclasses.dataclass
class SphereGrid:
    L: int
    n_theta: int
    n_phi: int
    theta: np.ndarray      # (n_theta,)
    w_theta: np.ndarray    # (n_theta,) Gauss-Legendre weights in cos(theta), sum 2
    phi: np.ndarray        # (n_phi,)
    w_phi: float           # 2 pi / n_phi
    khat: np.ndarray       # (N_dir, 3)
    theta_hat: np.ndarray  # (N_dir, 3)
    phi_hat: np.ndarray    # (N_dir, 3)
    weights: np.ndarray    # (N_dir,) w_theta * w_phi

    @property
    def n_dir(self):
        return self.n_theta * self.n_phi


def make_grid(L: int, nphi_rule: str = "2L+2") -> SphereGrid:
    n_theta = L + 1
    n_phi = n_phi_of(L, nphi_rule)
    x, w = np.polynomial.legendre.leggauss(n_theta)
    # leggauss orders x = cos(theta) ascending, i.e. theta descending
    x = x[::-1]
    w = w[::-1]
    theta = np.arccos(x)
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    T, P = np.meshgrid(theta, phi, indexing="ij")  # (n_theta, n_phi)
    T = T.reshape(-1, order="F")
    P = P.reshape(-1, order="F")
    st, ct, sp, cp = np.sin(T), np.cos(T), np.sin(P), np.cos(P)
    khat = np.stack([st * cp, st * sp, ct], axis=1)
    th = np.stack([ct * cp, ct * sp, -st], axis=1)
    ph = np.stack([-sp, cp, np.zeros_like(sp)], axis=1)
    w_phi = 2.0 * math.pi / n_phi
    weights = np.outer(w, np.full(n_phi, w_phi)).reshape(-1, order="F")
    return SphereGrid(L, n_theta, n_phi, theta, w, phi, w_phi, khat, th, ph, weights)
