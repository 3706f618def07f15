"""Translation stage of the FMM-FFT (Sec. II.A, between Eqs. 3 and 5; refs. [7, 8], [25]).

For RWG m in observation box v and RWG n in source box v' with the boxes far
apart, the EFIE interaction is
    Z_mn ~= (-j k / (16 pi^2)) sum_alpha sum_i w_i conj(P^alpha_m(k_i)) T_L(k_i, X) P^alpha_n(k_i),
X = r_v - r_v' (box centres), with the translation operator of the addition theorem
    T_L(k_hat, X) = sum_{l=0}^{L} (-j)^l (2l + 1) h_l^(2)(k |X|) P_l(k_hat . X_hat).
The translation stage turns the outgoing spectra F_v' of aggregation (Eq. 3) into
the incoming spectra of every box,
    g_v(k_i) = (-j k / (16 pi^2)) sum_{v' far from v} T_L(k_i, r_v - r_v') F_v'(k_i),
and the weighted disaggregation of g (Eq. 5 with the quadrature weights) gives the
far part of Z x.  Readings: two boxes are far when their grid indices differ by 2
or more in some coordinate (the boxes do not touch); the constant -jk/(16 pi^2)
is carried by the translation.  Plain double loop over box pairs: the reference
the FFT-based GPU translation is checked against.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from . import apply


def translation_operator(L: int, k: float, X: np.ndarray, khat: np.ndarray) -> np.ndarray:
    """T_L(k_hat_i, X) for every direction i (khat: N_dir x 3)."""
    x = k * np.linalg.norm(X)
    c = khat @ (X / np.linalg.norm(X))
    T = np.zeros(len(khat), complex)
    for l in range(L + 1):
        h2 = special.spherical_jn(l, x) - 1j * special.spherical_yn(l, x)
        T += (-1j) ** l * (2 * l + 1) * h2 * special.eval_legendre(l, c)
    return T


def is_far(i1, i2) -> bool:
    return int(np.max(np.abs(np.asarray(i1) - np.asarray(i2)))) >= 2


def translate(spectra: np.ndarray, groups, grid, k: float) -> np.ndarray:
    """Incoming spectra (G, 2, N_dir[, R]) from outgoing ones, by the double sum over far box pairs."""
    G = groups.n_groups
    out = np.zeros_like(spectra, dtype=np.complex128)
    scale = -1j * k / (16 * math.pi ** 2)
    cache = {}
    for v in range(G):
        for w in range(G):
            d = tuple(int(t) for t in groups.box_index[v] - groups.box_index[w])
            if max(abs(t) for t in d) < 2:
                continue
            T = cache.get(d)
            if T is None:
                T = scale * translation_operator(grid.L, k, groups.centre[v] - groups.centre[w], grid.khat)
                cache[d] = T
            Tb = T.reshape((-1,) + (1,) * (spectra.ndim - 3))
            out[v] += Tb[None] * spectra[w]
    return out


def far_matvec(ops, groups, grid, x: np.ndarray, k: float, tucker=True) -> np.ndarray:
    """Far part of Z x: weighted disaggregation of the translated aggregation."""
    F = apply.aggregate_all(ops, groups.members, x, tucker=tucker)
    g = translate(F, groups, grid, k)
    return apply.disaggregate_all(ops, groups.members, g, len(x), grid.weights, tucker=tucker)
