"""Far-field storage of the dense and Tucker formats (Sec. II.C, Tables I, III).

Dense: every group keeps an N_dir x n_beta matrix per component alpha, so the
whole problem stores N_RWG * (L + 1) * n_phi * 2 complex numbers.
Tucker: per group and component, n_theta r_theta + n_phi r_phi + n_beta r_beta
+ r_theta r_phi r_beta complex numbers (factors and core of Eq. 6).
"""
from __future__ import annotations


def dense_bytes(n_rwg: int, L: int, n_phi: int, bytes_per_complex: int = 16) -> int:
    return n_rwg * (L + 1) * n_phi * 2 * bytes_per_complex


def tucker_bytes(shapes, bytes_per_complex: int = 16) -> int:
    """``shapes``: iterable of (n_theta, n_phi, n_beta, r_theta, r_phi, r_beta)."""
    total = 0
    for nt, npf, nb, rt, rp, rb in shapes:
        total += nt * rt + npf * rp + nb * rb + rt * rp * rb
    return total * bytes_per_complex
