"""Truncated-SVD compression of the aggregation matrix (the comparator of Sec. II.C, ref. [11]).

The paper compares its Tucker format with the matrix-decomposition approach of
ref. [11]: the N_dir x n_beta aggregation matrix A_bar = P^{alpha,+} of a group
(Fig. 1a before tensorisation) is replaced by its truncated SVD

    A_bar ~= U_r Sigma_r V_r^H,

stored as B = U_r Sigma_r (N_dir x r) and V_r (n_beta x r).  Sec. II.C gives the
cost of both stages as O(n_beta r + n_theta n_phi r) per group:

    aggregation     F = B (V_r^H x)                       (Eq. 3 with A_bar replaced)
    disaggregation  y = V_r (B^H (W g))                   (Eq. 5, weighted as in apply.py)

Truncation.  The note under Table II says the SVD truncates at gamma while
Tucker truncates every mode at gamma / sqrt(3).  Read with the same relative
tail-energy rule as hosvd.py: r = the smallest r >= 1 with
sqrt(sum_{i > r} sigma_i^2) <= gamma ||A_bar||_F, so ||A_bar - B V_r^H||_F <= gamma ||A_bar||_F.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .apply import dense_matrix
from .hosvd import truncation_rank


@dataclasses.dataclass
class SVDFactors:
    B: np.ndarray  # N_dir x r, U_r Sigma_r
    V: np.ndarray  # n_beta x r, V_r

    @property
    def rank(self):
        return self.B.shape[1]


def truncated_svd(A: np.ndarray, tol: float) -> SVDFactors:
    """Truncated SVD of the aggregation matrix of an n_theta x n_phi x n_beta tensor."""
    M = dense_matrix(A)
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    r = truncation_rank(s, tol * np.linalg.norm(M))
    return SVDFactors(U[:, :r] * s[:r], Vh[:r].conj().T)


def reconstruct(S: SVDFactors) -> np.ndarray:
    """The N_dir x n_beta matrix B V^H."""
    return S.B @ S.V.conj().T


def svd_aggregate(S: SVDFactors, x: np.ndarray) -> np.ndarray:
    t = S.V.conj().T @ x          # r (x R)
    return S.B @ t                # N_dir (x R)


def svd_disaggregate(S: SVDFactors, g: np.ndarray, weights=None) -> np.ndarray:
    if weights is not None:
        g = weights.reshape((-1,) + (1,) * (g.ndim - 1)) * g
    s = S.B.conj().T @ g          # r (x R)
    return S.V @ s                # n_beta (x R)


def memory_bytes(shapes, bytes_per_complex: int = 16) -> int:
    """Storage of the SVD format, Sec. II.C: ``shapes`` = iterable of (N_dir, n_beta, r)."""
    return sum((nd + nb) * r for nd, nb, r in shapes) * bytes_per_complex
