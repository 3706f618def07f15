"""Pins of the oracle's far-field of Eq. 4 and of its use in the FMM (Sec. II.A).

* closed form: the Hermite-Genocchi formula gives int_T exp(sum lambda_k z_k) as a
  divided difference of exp, and the linear RWG factor as a confluent one;
* the plane-wave excitation at a grid direction equals the receiving pattern
  conj(P^{alpha,+}) of Eq. 4 up to the phase of the group centre;
* physics: aggregation -> textbook translation (ref. [25] addition theorem) ->
  disaggregation reproduces the direct EFIE interaction of two far RWGs with
  the Green's function exp(-jkR)/(4 pi R) of Eq. 1.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import farfield, grid, planewave, rwg, translation


def _divdiff_exp(nodes):
    """Divided difference exp[x0, ..., xm]; equal nodes must be adjacent (confluent)."""
    x = list(nodes)
    m = len(x)
    table = [np.exp(xi) for xi in x]
    for level in range(1, m):
        new = []
        for i in range(m - level):
            if x[i + level] == x[i]:  # only level-1 confluence (one repeated node) is needed here
                assert level == 1
                new.append(np.exp(x[i]))
            else:
                new.append((table[i + 1] - table[i]) / (x[i + level] - x[i]))
        table = new
    return table[0]


def _closed_form_rwg_vector(v0, v1, v2, p_side, l, sign_b, kvec):
    """int_T (sign_b) l/(2A) (r - p) exp(j kvec.r) dA, T = (v0, v1, v2), in closed form."""
    V = [v0, v1, v2]
    A = 0.5 * np.linalg.norm(np.cross(v1 - v0, v2 - v0))
    z = [1j * np.dot(kvec, vi) for vi in V]
    I0 = 2 * A * _divdiff_exp(z)
    Ii = []
    for i in range(3):
        others = [z[j] for j in range(3) if j != i]
        Ii.append(2 * A * _divdiff_exp([z[i], z[i]] + others))
    r_int = sum(V[i] * Ii[i] for i in range(3))
    return sign_b * l / (2 * A) * (r_int - p_side * I0)


@pytest.mark.parametrize("scale,order,tol", [(0.9, 16, 1e-11), (0.1, 6, 1e-10)])
def test_single_rwg_far_field_closed_form(scale, order, tol):
    rng = np.random.default_rng(7)
    base = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.3], [1.1, 1.0, -0.4]])
    verts = base * scale + rng.normal(scale=0.01, size=base.shape)
    tris = np.array([[0, 1, 2], [1, 3, 2]])
    r = rwg.build_rwg(verts, tris)
    assert r.n == 1
    k = 2 * math.pi
    centre = np.array([0.3, -0.2, 0.1]) * scale
    khat = rng.normal(size=(12, 3))
    khat /= np.linalg.norm(khat, axis=1, keepdims=True)
    J = farfield.radiation_vectors(verts, r, [0], centre, k, khat, order=order)[0]
    for i in range(len(khat)):
        kvec = k * khat[i]
        expect = np.zeros(3, complex)
        for side, sgn in ((0, 1.0), (1, -1.0)):
            t = tris[r.tri[0, side]]
            expect += _closed_form_rwg_vector(verts[t[0]], verts[t[1]], verts[t[2]],
                                              verts[r.free[0, side]], r.length[0], sgn, kvec)
        expect *= np.exp(-1j * np.dot(kvec, centre))
        assert np.linalg.norm(J[:, i] - expect) <= tol * np.linalg.norm(expect)


def test_group_tensor_layout_and_projection(sphere2_oracle):
    P = sphere2_oracle
    g = 3
    ids = P.groups.members[g]
    At, Ap = P.tensors[g]
    assert At.shape == (P.grid.n_theta, P.grid.n_phi, len(ids))
    J = farfield.radiation_vectors(P.verts, P.rwg, ids[:4], P.groups.centre[g], P.k, P.grid.khat)
    it, ip = 5, 7
    i = it + P.grid.n_theta * ip
    for n in range(4):
        assert abs(At[it, ip, n] - P.grid.theta_hat[i] @ J[n, :, i]) < 1e-14
        assert abs(Ap[it, ip, n] - P.grid.phi_hat[i] @ J[n, :, i]) < 1e-14


def test_planewave_at_grid_direction_is_receive_pattern(sphere2_oracle):
    """V_m = -exp(-j k k_i . r_v) conj(P^{alpha,+}_{m,i}) for k_inc = k_i, p = alpha_i."""
    P = sphere2_oracle
    g = 5
    ids = P.groups.members[g]
    At, Ap = P.tensors[g]
    for it, ip in ((2, 3), (9, 20)):
        i = it + P.grid.n_theta * ip
        kh = P.grid.khat[i]
        for A, ahat in ((At, P.grid.theta_hat[i]), (Ap, P.grid.phi_hat[i])):
            V = planewave.planewave_rhs(P.verts, P.rwg, P.k, kh, ahat)
            expect = -np.exp(-1j * P.k * kh @ P.groups.centre[g]) * np.conj(A[it, ip, :])
            assert np.max(np.abs(V[ids] - expect)) < 1e-12 * np.max(np.abs(expect))


def _tri_rule(order):
    """Collapsed Gauss-Legendre rule written independently of the oracle: (u, v, w), sum w = 1/2."""
    x, w = special.roots_legendre(order)
    x = (x + 1) / 2
    w = w / 2
    u = np.repeat(x, order)
    v = np.tile(x, order)
    ww = np.repeat(w, order) * np.tile(w, order) * (1 - u)
    return u, v, ww


def _direct_efie(verts, tris, r, m, n, k, order=7):
    """int int [b_m.b_n - div b_m div' b_n / k^2] exp(-jkR)/(4 pi R) over the supports."""
    u, v, w = _tri_rule(order)
    total = 0.0
    pts, vals, divs, wts = [], [], [], []
    for idx in (m, n):
        P_, V_, D_, W_ = [], [], [], []
        for side in range(2):
            t = tris[r.tri[idx, side]]
            a, b, c = verts[t[0]], verts[t[1]], verts[t[2]]
            A = r.area[idx, side]
            q = a[None] + u[:, None] * (b - a)[None] + (v * (1 - u))[:, None] * (c - a)[None]
            P_.append(q)
            V_.append(rwg.evaluate(verts, r, idx, side, q))
            D_.append(np.full(len(u), rwg.divergence(r, idx, side)))
            W_.append(2 * A * w)
        pts.append(np.concatenate(P_))
        vals.append(np.concatenate(V_))
        divs.append(np.concatenate(D_))
        wts.append(np.concatenate(W_))
    R = np.linalg.norm(pts[0][:, None, :] - pts[1][None, :, :], axis=2)
    G = np.exp(-1j * k * R) / (4 * math.pi * R)
    kern = vals[0] @ vals[1].T - np.outer(divs[0], divs[1]) / k ** 2
    total = np.sum(wts[0][:, None] * wts[1][None, :] * kern * G)
    return total


@pytest.mark.parametrize("digits", [4, 6])
def test_two_group_translation_matches_direct_interaction(digits):
    k = 2 * math.pi
    a = 0.5
    L = grid.bandwidth(k, a, digits)
    g = grid.make_grid(L, "2L+1")
    rng = np.random.default_rng(11)
    src_c = np.zeros(3)
    worst = 0.0
    for X in (np.array([2 * a, 0, 0]), np.array([2 * a, 2 * a, 0]), np.array([0, 2 * a, -2 * a])):
        obs_c = src_c + X
        # one random RWG (two triangles, edges ~ lambda/10) inside each box
        verts = []
        for c in (obs_c, src_c):
            p0 = c + rng.uniform(-0.3 * a, 0.3 * a, size=3)
            e1, e2, e3 = (rng.normal(scale=0.06, size=3) for _ in range(3))
            verts += [p0, p0 + e1, p0 + e2, p0 + e1 + e3]
        verts = np.array(verts)
        tris = np.array([[0, 1, 2], [1, 3, 2], [4, 5, 6], [5, 7, 6]])
        r = rwg.build_rwg(verts, tris)
        assert r.n == 2
        m, n = 0, 1  # RWG 0 is in the observer box (lower vertex ids)
        Jm = farfield.radiation_vectors(verts, r, [m], obs_c, k, g.khat, order=6)[0]
        Jn = farfield.radiation_vectors(verts, r, [n], src_c, k, g.khat, order=6)[0]
        Z_fmm = 0.0
        for ahat in (g.theta_hat, g.phi_hat):
            Pm = np.einsum("ci,ic->i", Jm, ahat)
            Pn = np.einsum("ci,ic->i", Jn, ahat)
            Z_fmm = Z_fmm + np.sum(g.weights * translation.translation_operator(L, k, X, g.khat) * np.conj(Pm) * Pn)
        Z_fmm *= -1j * k / (16 * math.pi ** 2)
        Z_dir = _direct_efie(verts, tris, r, m, n, k)
        worst = max(worst, abs(Z_fmm - Z_dir) / abs(Z_dir))
    print("translation worst rel err", digits, worst)
    assert worst <= 10.0 ** (-(digits - 1)), worst
