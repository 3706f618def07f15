"""Truncated higher-order SVD (Eq. 6, Sec. II.B; De Lathauwer et al., ref. [26]).

For p = theta, phi, beta: U^p holds the leading left singular vectors of the
mode-p unfolding A_(p) (n_p x prod of the other sizes).  The core is
C = A x_1 U^theta^H x_2 U^phi^H x_3 U^beta^H.

Truncation (Sec. III.A, "Box size and ranks": Tucker truncates each mode at
gamma / sqrt(3)).  Reading of the tolerance: relative tail energy,
r_p = the smallest r >= 1 with  sqrt(sum_{i > r} sigma_i^2) <= gamma/sqrt(3) ||A||_F.
With this reading ||A - A_hat||_F <= gamma ||A||_F (ref. [26]).

The oracle is the plain T-HOSVD: every factor comes from the unfolding of the
uncompressed tensor.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Tucker:
    U_theta: np.ndarray  # n_theta x r_theta
    U_phi: np.ndarray    # n_phi x r_phi
    U_beta: np.ndarray   # n_beta x r_beta
    core: np.ndarray     # r_theta x r_phi x r_beta

    @property
    def ranks(self):
        return self.core.shape


def unfold(A: np.ndarray, mode: int) -> np.ndarray:
    """Mode-``mode`` unfolding: rows indexed by that mode, columns by the others."""
    return np.moveaxis(A, mode, 0).reshape(A.shape[mode], -1)


def truncation_rank(sigma: np.ndarray, threshold: float) -> int:
    """Smallest r >= 1 whose discarded tail energy is within ``threshold``."""
    tail = np.sqrt(np.cumsum((sigma ** 2)[::-1]))[::-1]  # tail[r] = ||sigma[r:]||
    tail = np.append(tail, 0.0)
    for r in range(1, len(sigma) + 1):
        if tail[r] <= threshold:
            return r
    return len(sigma)


def mode_product(A: np.ndarray, M: np.ndarray, mode: int) -> np.ndarray:
    """A x_mode M: contracts index ``mode`` of A with the columns of M (M is m x n_mode)."""
    out = np.tensordot(M, A, axes=(1, mode))
    return np.moveaxis(out, 0, mode)


def thosvd(A: np.ndarray, tol: float) -> Tucker:
    norm = np.linalg.norm(A)
    threshold = tol / math.sqrt(3.0) * norm
    factors = []
    for mode in range(3):
        U, s, _ = np.linalg.svd(unfold(A, mode), full_matrices=False)
        r = truncation_rank(s, threshold)
        factors.append(U[:, :r])
    core = A
    for mode in range(3):
        core = mode_product(core, factors[mode].conj().T, mode)
    return Tucker(factors[0], factors[1], factors[2], core)


def reconstruct(T: Tucker) -> np.ndarray:
    A = T.core
    A = mode_product(A, T.U_theta, 0)
    A = mode_product(A, T.U_phi, 1)
    A = mode_product(A, T.U_beta, 2)
    return A
