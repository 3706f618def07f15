"""RWG-tested plane-wave excitation (Eq. 2, Sec. III.A).

V_m = <b_m, n x n x E^i> = -int b_m(r) . E^i(r) dr  (b_m is tangential, so
n x n x E^i = -E^i_tan on S), with E^i(r) = p_hat exp(-j k k_inc . r) for a
wave propagating along
k_inc = sin(t) cos(p) x + sin(t) sin(p) y + cos(t) z.
The inner product does not conjugate (Galerkin testing, Eq. 2).
"""
from __future__ import annotations

import numpy as np

from .farfield import rwg_quadrature


def planewave_rhs(verts, rwg, k, khat_inc, pol, order=6, chunk=4096):
    khat_inc = np.asarray(khat_inc, dtype=np.float64)
    pol = np.asarray(pol, dtype=np.float64)
    out = np.empty(rwg.n, dtype=np.complex128)
    ids = np.arange(rwg.n)
    for s in range(0, rwg.n, chunk):
        sub = ids[s:s + chunk]
        pts, amp = rwg_quadrature(verts, rwg, sub, order)
        E = np.exp(-1j * k * (pts @ khat_inc))             # (n, 2Q)
        out[s:s + len(sub)] = -np.einsum("nqc,c,nq->n", amp, pol, E)
    return out


def incidence(theta, phi):
    """(k_inc, theta_hat_inc, phi_hat_inc) for the incidence angles (theta, phi)."""
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    return (np.array([st * cp, st * sp, ct]),
            np.array([ct * cp, ct * sp, -st]),
            np.array([-sp, cp, 0.0]))
