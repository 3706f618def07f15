"""Pins of the oracle's truncated HOSVD (Eq. 6, Sec. II.B; ref. [26])."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import hosvd, svd
from paper_2103_05822_gb300.inputs import icosphere

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _orth(n, r, seed):
    q, _ = np.linalg.qr(_rand((n, r), seed))
    return q


@pytest.mark.parametrize("ranks", [(1, 1, 1), (2, 3, 4), (5, 2, 7)])
def test_exact_low_rank_recovered(ranks):
    shape = (9, 14, 23)
    core = _rand(ranks, 1)
    A = core
    for mode, (n, r) in enumerate(zip(shape, ranks)):
        A = hosvd.mode_product(A, _orth(n, r, 10 + mode), mode)
    T = hosvd.thosvd(A, 1e-10)
    assert T.ranks == ranks
    assert np.linalg.norm(hosvd.reconstruct(T) - A) <= 1e-13 * np.linalg.norm(A)


def test_factors_orthonormal_and_core_all_orthogonal(sphere2_oracle):
    At, _ = sphere2_oracle.tensors[1]
    norm2 = np.linalg.norm(At) ** 2
    for tol in (0.0, 1e-4):
        T = hosvd.thosvd(At, tol)
        for U in (T.U_theta, T.U_phi, T.U_beta):
            assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-13)
        # all-orthogonality: core slices along each mode are mutually orthogonal, with
        # squared norms the mode's singular values squared, descending; truncation of the
        # other modes perturbs this by at most the discarded energy
        for mode in range(3):
            C = hosvd.unfold(T.core, mode)
            G = C @ C.conj().T
            off = G - np.diag(np.diag(G))
            slack = tol ** 2 * norm2 + 1e-13 * norm2
            assert np.max(np.abs(off)) <= slack
            assert np.all(np.diff(np.real(np.diag(G))) <= slack)
            if tol == 0.0:
                s = np.linalg.svd(hosvd.unfold(At, mode), compute_uv=False)
                assert np.allclose(np.sqrt(np.real(np.diag(G))), s[:len(G)], rtol=1e-10, atol=1e-12 * s[0])


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_error_bound_on_far_field_tensors(sphere2_oracle, tol):
    for g in (0, 7, 20):
        for A in sphere2_oracle.tensors[g]:
            T = hosvd.thosvd(A, tol)
            err = np.linalg.norm(hosvd.reconstruct(T) - A)
            assert err <= tol * np.linalg.norm(A)
            rt, rp, rb = T.ranks
            nt, npf, nb = A.shape
            assert 1 <= rt <= nt and 1 <= rp <= npf and 1 <= rb <= min(nb, nt * npf)


def test_zero_tolerance_reproduces_tensor(sphere2_oracle):
    A = sphere2_oracle.tensors[2][1]
    T = hosvd.thosvd(A, 0.0)
    assert T.ranks == (A.shape[0], A.shape[1], min(A.shape[2], A.shape[0] * A.shape[1]))
    assert np.linalg.norm(hosvd.reconstruct(T) - A) <= 1e-13 * np.linalg.norm(A)


def test_truncation_rank_rule():
    s = np.array([4.0, 3.0, 0.0])
    # tail after r=1 is 3 -> threshold 3 keeps r = 1 (inclusive), 2.999 needs r = 2
    assert hosvd.truncation_rank(s, 3.0) == 1
    assert hosvd.truncation_rank(s, 2.999) == 2
    assert hosvd.truncation_rank(s, 0.0) == 2
    assert hosvd.truncation_rank(np.zeros(4), 0.0) == 1
    assert hosvd.truncation_rank(s, 100.0) == 1


def test_tolerance_is_split_over_three_modes():
    """Per-mode threshold gamma/sqrt(3) (Sec. III.A): tails just inside it are cut."""
    n = 12
    sig = np.array([1.0] + [0.0] * (n - 1))
    tail_val = 0.999e-3 / math.sqrt(3.0)  # one discarded singular value per mode
    sig[1] = tail_val
    U1, U2, U3 = (_orth(n, n, s) for s in (1, 2, 3))
    # diagonal core with entries sigma: mode unfoldings then have singular values sigma
    core = np.zeros((n, n, n), complex)
    for i in range(n):
        core[i, i, i] = sig[i]
    A = hosvd.mode_product(hosvd.mode_product(hosvd.mode_product(core, U1, 0), U2, 1), U3, 2)
    norm = np.linalg.norm(A)
    assert abs(norm - np.linalg.norm(sig)) < 1e-14
    # threshold gamma/sqrt(3) ||A|| with gamma = 1e-3 / ||A||: the tail 0.999e-3/sqrt(3) is inside
    T = hosvd.thosvd(A, 1e-3 / norm)
    assert T.ranks == (1, 1, 1)
    assert np.linalg.norm(hosvd.reconstruct(T) - A) <= 1e-3
    # a threshold just below the tail keeps it
    T2 = hosvd.thosvd(A, 0.998e-3 / norm)
    assert T2.ranks == (2, 2, 2)


@pytest.mark.slow
def test_ranks_match_paper_table_iv_order_of_magnitude():
    """A 2-lambda box on a 30-lambda sphere at L = 37, gamma = 1e-6 (Table IV: Tucker 25, 29, 175; SVD 168)."""
    gold = json.load(open(GOLDEN))["sphere_ranks_2lambda"]
    v, f = icosphere(30.0, 180)
    # keep only triangles near one box (a patch around a point of the sphere)
    c = np.array([1.0, 0.6, 0.45])
    c = 15.0 * c / np.linalg.norm(c)
    cent = v[f].mean(axis=1)
    keep = np.all(np.abs(cent - c) < 3.5, axis=1)
    sub = f[keep]
    used, inv = np.unique(sub, return_inverse=True)
    vs, fs = v[used], inv.reshape(-1, 3)
    r = oracle.rwg.build_rwg(vs, fs)
    mp = oracle.rwg.midpoints(vs, r)
    box = 2.0
    # boxes of the global grid (anchored at the sphere's bounding box, -15) in the patch;
    # take the one whose RWG count is closest to the paper's 909
    best = None
    base = np.floor((c + 15.0) / box) * box - 15.0
    for off in np.ndindex(3, 3, 3):
        lo = base + (np.array(off) - 1) * box
        inside = np.all((mp >= lo) & (mp < lo + box), axis=1)
        if np.all(np.abs(lo + box / 2 - c) <= 3.5 - box / 2 - 0.2):  # box well inside the patch
            cnt = int(inside.sum())
            if best is None or abs(cnt - gold["n_beta"]) < abs(best[0] - gold["n_beta"]):
                best = (cnt, lo, np.nonzero(inside)[0])
    _, lo, ids = best
    assert 600 < len(ids) < 1300
    g = oracle.grid.make_grid(gold["L"], "2L+1")
    At, Ap = oracle.farfield.group_tensors(vs, r, ids, lo + box / 2, 2 * math.pi, g, order=5)
    for A in (At, Ap):
        T = hosvd.thosvd(A, gold["tol"])
        rt, rp, rb = T.ranks
        scale_b = len(ids) / gold["n_beta"]
        assert 0.7 * gold["r_theta"] <= rt <= 1.3 * gold["r_theta"], T.ranks
        assert 0.7 * gold["r_phi"] <= rp <= 1.4 * gold["r_phi"], T.ranks
        assert 0.6 * gold["r_beta"] <= rb <= 1.5 * gold["r_beta"] * max(1.0, scale_b), T.ranks
        # the SVD comparator of the same box (Table IV, SVD column): just below the Tucker r_beta
        rs = svd.truncated_svd(A, gold["tol"]).rank
        assert rs <= rb and 0.6 * gold["svd_r_beta"] <= rs <= 1.5 * gold["svd_r_beta"] * max(1.0, scale_b), rs
        print("ranks", len(ids), T.ranks, "svd", rs)
