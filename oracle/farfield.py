"""Far-fields of RWG functions, Eq. 4 (Sec. II.A).

    P^{alpha,+}_{n,i} = alpha_i . int_{S_n} (I - k_i k_i) b_n(r) exp(+j k k_i.(r - r_v)) dr

alpha_i is theta_hat_i or phi_hat_i; both are orthogonal to k_i, so the
projector drops out and P^{alpha,+}_{n,i} = alpha_i . int b_n exp(...) dr.
The receiving pattern is P^{alpha,-} = conj(P^{alpha,+}) (free space, end of
Sec. II.A).

Quadrature (the paper does not say which rule it uses): a collapsed
(Duffy) tensor-product Gauss-Legendre rule of ``order`` x ``order`` points on
each triangle,  r(u, v) = p + u (q1 - p) + v (1 - u) (q2 - p),
dA = 2 A (1 - u) du dv on [0, 1]^2.

The aggregation tensor of one group and one component (Fig. 1a) is the
n_theta x n_phi x n_beta array A[i_theta, i_phi, n] = P^{alpha,+}_{n, i}.
"""
from __future__ import annotations

import numpy as np

from .rwg import RWG


def collapsed_rule(order: int):
    """Points (u, v) and weights on [0,1]^2 of the collapsed Gauss-Legendre rule.

    Returns ``(u, v, w)`` with w already multiplied by the Duffy factor (1 - u),
    so that  int_T f dA = 2 A sum_q w_q f(r(u_q, v_q))  and sum_q w_q = 1/2.
    """
    x, w = np.polynomial.legendre.leggauss(order)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    U, V = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    U = U.ravel()
    V = V.ravel()
    return U, V, (WU * WV).ravel() * (1.0 - U)


def rwg_quadrature(verts, rwg: RWG, ids, order: int):
    """Quadrature points and vector amplitudes of b_n for the RWGs ``ids``.

    Returns ``pts`` (n, 2Q, 3) and ``amp`` (n, 2Q, 3) such that for any f,
        int b_n(r) f(r) dr = sum_q amp[n, q] f(pts[n, q]).
    """
    verts = np.asarray(verts, dtype=np.float64)
    ids = np.asarray(ids, dtype=np.int64)
    u, v, w = collapsed_rule(order)
    pts = []
    amp = []
    for side, sign in ((0, 1.0), (1, -1.0)):
        p = verts[rwg.free[ids, side]]          # (n, 3) free vertex
        q1 = verts[rwg.edge[ids, 0]]
        q2 = verts[rwg.edge[ids, 1]]
        r = (p[:, None, :] + u[None, :, None] * (q1 - p)[:, None, :]
             + (v * (1.0 - u))[None, :, None] * (q2 - p)[:, None, :])
        # b = l/(2A) (r - p) on T+, l/(2A) (p - r) on T-; dA = 2A * w
        a = sign * rwg.length[ids][:, None, None] * w[None, :, None] * (r - p[:, None, :])
        pts.append(r)
        amp.append(a)
    return np.concatenate(pts, axis=1), np.concatenate(amp, axis=1)


def radiation_vectors(verts, rwg: RWG, ids, centre, k, khat, order=6, sign=+1.0, chunk=32):
    """J[n, :, i] = int b_n(r) exp(sign * j k khat_i . (r - centre)) dr, shape (n, 3, N_dir)."""
    ids = np.asarray(ids, dtype=np.int64)
    khat = np.asarray(khat, dtype=np.float64)
    out = np.empty((len(ids), 3, len(khat)), dtype=np.complex128)
    for s in range(0, len(ids), chunk):
        sub = ids[s:s + chunk]
        pts, amp = rwg_quadrature(verts, rwg, sub, order)
        phase = k * ((pts - np.asarray(centre)[None, None, :]) @ khat.T)   # (n, 2Q, N_dir)
        ampT = np.ascontiguousarray(amp.transpose(0, 2, 1))                 # (n, 3, 2Q)
        # exp(sign j phase) = cos(phase) + sign j sin(phase)
        out[s:s + len(sub)] = ampT @ np.cos(phase) + (sign * 1j) * (ampT @ np.sin(phase))
    return out


def group_tensors(verts, rwg: RWG, ids, centre, k, grid, order=6):
    """Aggregation tensors (A_theta, A_phi) of one group, each n_theta x n_phi x n_beta."""
    J = radiation_vectors(verts, rwg, ids, centre, k, grid.khat, order)
    out = []
    for ahat in (grid.theta_hat, grid.phi_hat):
        P = np.einsum("nci,ic->in", J, ahat)  # (N_dir, n_beta)
        out.append(P.reshape(grid.n_theta, grid.n_phi, len(ids), order="F"))
    return out
