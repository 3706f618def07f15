"""Pins of the oracle's truncated-SVD comparator (Sec. II.C, ref. [11]; Tables II-IV).

* exact low rank: a rank-3 aggregation matrix is recovered with rank 3;
* the gamma bound ||A_bar - B V^H||_F <= gamma ||A_bar||_F on real far-field
  matrices, with the smallest such rank (one less breaks the bound);
* gamma = 0 reproduces the matrix;
* the SVD and the Tucker beta mode truncate the same singular values: the
  mode-3 unfolding of the tensor is the transpose of A_bar, so the SVD rank at
  gamma / sqrt(3) equals the T-HOSVD r_beta at gamma (this pins the threshold
  convention of both: gamma for the SVD, gamma / sqrt(3) per Tucker mode, the
  note under Table II);
* apply: aggregation / disaggregation equal the dense Eqs. 3 / 5 of the
  reconstructed matrix, and the weighted adjointness <A x, W g> = <x, A^H W g>;
* B has orthogonal columns with descending norms (the singular values), V is
  orthonormal.
The paper's Table IV SVD rank is checked with the Tucker ranks in
test_oracle_hosvd.py (same 2-lambda box).
"""
import numpy as np
import pytest

from oracle import apply, hosvd, svd
from paper_2103_05822_gb300.inputs import complex_gaussian


def _low_rank_tensor(shape, r, seed):
    nt, npf, nb = shape
    rng = np.random.default_rng(seed)
    L = rng.normal(size=(nt * npf, r)) + 1j * rng.normal(size=(nt * npf, r))
    R = rng.normal(size=(r, nb)) + 1j * rng.normal(size=(r, nb))
    return (L @ R).reshape(nt, npf, nb, order="F")


def test_exact_low_rank_recovered():
    A = _low_rank_tensor((6, 8, 20), 3, 1)
    S = svd.truncated_svd(A, 1e-10)
    assert S.rank == 3
    M = apply.dense_matrix(A)
    assert np.linalg.norm(svd.reconstruct(S) - M) <= 1e-13 * np.linalg.norm(M)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_error_bound_and_minimal_rank_on_far_fields(sphere2_oracle, tol):
    for g in (0, 7, 20):
        for A in sphere2_oracle.tensors[g]:
            M = apply.dense_matrix(A)
            S = svd.truncated_svd(A, tol)
            err = np.linalg.norm(svd.reconstruct(S) - M)
            assert err <= tol * np.linalg.norm(M)
            if S.rank > 1:  # one singular value fewer breaks the bound
                B1, V1 = S.B[:, :-1], S.V[:, :-1]
                assert np.linalg.norm(B1 @ V1.conj().T - M) > tol * np.linalg.norm(M)
            assert 1 <= S.rank <= min(M.shape)


def test_zero_tolerance_reproduces_matrix(sphere2_oracle):
    A = sphere2_oracle.tensors[3][0]
    M = apply.dense_matrix(A)
    S = svd.truncated_svd(A, 0.0)
    assert np.linalg.norm(svd.reconstruct(S) - M) <= 1e-13 * np.linalg.norm(M)


@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_svd_rank_equals_tucker_beta_rank_at_the_per_mode_tolerance(sphere2_oracle, tol):
    for g in (1, 9, 30):
        for A in sphere2_oracle.tensors[g]:
            rb = hosvd.thosvd(A, tol).ranks[2]
            assert svd.truncated_svd(A, tol / np.sqrt(3.0)).rank == rb
            # at the same gamma the SVD keeps no more than the Tucker beta mode
            assert svd.truncated_svd(A, tol).rank <= rb


def test_factors_orthogonal_with_singular_value_norms(sphere2_oracle):
    A = sphere2_oracle.tensors[5][1]
    S = svd.truncated_svd(A, 1e-6)
    assert np.allclose(S.V.conj().T @ S.V, np.eye(S.rank), atol=1e-13)
    G = S.B.conj().T @ S.B
    d = np.real(np.diag(G))
    assert np.max(np.abs(G - np.diag(d))) <= 1e-13 * d[0]
    assert np.all(np.diff(d) <= 0)
    s = np.linalg.svd(apply.dense_matrix(A), compute_uv=False)
    assert np.allclose(np.sqrt(d), s[:S.rank], rtol=1e-10)


def test_apply_equals_dense_apply_of_reconstruction_and_is_adjoint(sphere2_oracle):
    P = sphere2_oracle
    A = P.tensors[4][0]
    S = svd.truncated_svd(A, 1e-4)
    M = svd.reconstruct(S)
    nb = A.shape[2]
    x = complex_gaussian((nb, 3), 5)
    g = complex_gaussian((M.shape[0], 3), 6)
    w = P.grid.weights
    F = svd.svd_aggregate(S, x)
    assert np.linalg.norm(F - M @ x) <= 1e-13 * np.linalg.norm(M @ x)
    y = svd.svd_disaggregate(S, g, w)
    ref = M.conj().T @ (w[:, None] * g)
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
    lhs = np.vdot(w[:, None] * g, F)
    rhs = np.vdot(y, x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(F) * np.linalg.norm(w[:, None] * g)
    # against the uncompressed matrix: ||(A - A_hat) x|| <= gamma ||A||_F ||x|| per column
    Md = apply.dense_matrix(A)
    for c in range(3):
        assert np.linalg.norm(F[:, c] - Md @ x[:, c]) <= 1e-4 * np.linalg.norm(Md) * np.linalg.norm(x[:, c])


def test_memory_formula():
    # Sec. II.C: (n_theta n_phi + n_beta) r complex numbers per group and component
    assert svd.memory_bytes([(3200, 940, 170), (3200, 100, 60)]) == ((3200 + 940) * 170 + (3200 + 100) * 60) * 16
