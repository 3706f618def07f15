"""Aggregation and disaggregation, dense and Tucker (Sec. II.A Eqs. 3, 5; Sec. II.C).

Column-major (Matlab) conventions throughout, as the reshapes of Figs. 2b/3b
imply: a direction index is i = i_theta + n_theta i_phi, and the mode-3
matricised core C_(3) is r_beta x (r_theta r_phi) with column a + r_theta b.

Dense (Figs. 2a / 3a):
    F_alpha = A_alpha x                                        (Eq. 3)
    y       = sum_alpha A_alpha^H (W * g_alpha)                (Eq. 5 with P^- = conj(P^+))

Tucker aggregation, Fig. 2b, step by step:
    1. t = U_beta^T x (r_beta); u = t^T C_(3)  (1 x r_theta r_phi)
    2. reshape u to the r_theta x r_phi matrix M; V = U_phi M^T  (n_phi x r_theta)
    3. F = U_theta V^T  (n_theta x n_phi)
    4. vec(F) is the N_dir spectrum of the group.

Tucker disaggregation, Fig. 3b, step by step:
    1. G = conj(W * g) reshaped n_theta x n_phi; H = U_theta^T G U_phi
    2. s = C_(3) vec(H)
    3. y = conj(U_beta s).

W are the quadrature weights w_theta * 2 pi / n_phi.  ``apply_weights=False``
gives the paper's plain Eq. 5 (the conjugate transpose).  Reading: the
disaggregation the solver needs integrates over the unit sphere, so the
weights are applied to the incoming spectrum by default.

x / g may carry a trailing right-hand-side axis (columns).
"""
from __future__ import annotations

import numpy as np

from .hosvd import Tucker


def core_matricised(T: Tucker) -> np.ndarray:
    """C_(3): r_beta x (r_theta r_phi), column index a + r_theta b."""
    rt, rp, rb = T.core.shape
    return T.core.reshape(rt * rp, rb, order="F").T


def tucker_aggregate(T: Tucker, x: np.ndarray) -> np.ndarray:
    x2 = x.reshape(x.shape[0], -1)
    R = x2.shape[1]
    rt, rp, rb = T.core.shape
    nt, npf = T.U_theta.shape[0], T.U_phi.shape[0]
    C3 = core_matricised(T)
    out = np.empty((nt * npf, R), dtype=np.complex128)
    for r in range(R):
        t = T.U_beta.T @ x2[:, r]                    # step 1
        u = t @ C3                                   # 1 x (r_theta r_phi)
        M = u.reshape(rt, rp, order="F")             # step 2
        V = T.U_phi @ M.T                            # n_phi x r_theta
        F = T.U_theta @ V.T                          # step 3: n_theta x n_phi
        out[:, r] = F.reshape(-1, order="F")         # step 4
    return out.reshape((nt * npf,) + x.shape[1:])


def tucker_disaggregate(T: Tucker, g: np.ndarray, weights=None) -> np.ndarray:
    g2 = g.reshape(g.shape[0], -1)
    R = g2.shape[1]
    nt, npf = T.U_theta.shape[0], T.U_phi.shape[0]
    C3 = core_matricised(T)
    nb = T.U_beta.shape[0]
    out = np.empty((nb, R), dtype=np.complex128)
    for r in range(R):
        gr = g2[:, r] if weights is None else weights * g2[:, r]
        G = np.conj(gr).reshape(nt, npf, order="F")  # step 1
        H = T.U_theta.T @ G @ T.U_phi                # r_theta x r_phi
        s = C3 @ H.reshape(-1, order="F")            # step 2
        out[:, r] = np.conj(T.U_beta @ s)            # step 3
    return out.reshape((nb,) + g.shape[1:])


def dense_matrix(A: np.ndarray) -> np.ndarray:
    """Aggregation matrix (N_dir x n_beta) of an n_theta x n_phi x n_beta tensor (Fig. 1a)."""
    nt, npf, nb = A.shape
    return A.reshape(nt * npf, nb, order="F")


def dense_aggregate(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    return dense_matrix(A) @ x


def dense_disaggregate(A: np.ndarray, g: np.ndarray, weights=None) -> np.ndarray:
    P = dense_matrix(A)
    if weights is not None:
        g = (weights.reshape((-1,) + (1,) * (g.ndim - 1))) * g
    return P.conj().T @ g


# ---------------------------------------------------------------- whole problem
def aggregate_all(ops, members, x, tucker=True):
    """Spectra of every group: array (G, 2, N_dir[, R]).

    ``ops[g][alpha]`` is a Tucker (tucker=True) or a dense tensor; ``members[g]``
    the global RWG ids of group g; x is in global RWG order.
    """
    out = []
    for g, ids in enumerate(members):
        xg = x[ids]
        per = []
        for alpha in range(2):
            op = ops[g][alpha]
            per.append(tucker_aggregate(op, xg) if tucker else dense_aggregate(op, xg))
        out.append(np.stack(per))
    return np.stack(out)


def disaggregate_all(ops, members, spectra, n_rwg, weights=None, tucker=True, beta=0.0, y0=None):
    """y = beta y0 + sum over groups and alpha of the disaggregated spectra (global RWG order)."""
    tail = spectra.shape[3:]
    y = np.zeros((n_rwg,) + tail, dtype=np.complex128)
    if y0 is not None and beta != 0.0:
        y += beta * y0
    for g, ids in enumerate(members):
        acc = 0.0
        for alpha in range(2):
            op = ops[g][alpha]
            s = spectra[g, alpha]
            acc = acc + (tucker_disaggregate(op, s, weights) if tucker
                         else dense_disaggregate(op, s, weights))
        y[ids] += acc
    return y
