"""Pins of the oracle's aggregation / disaggregation (Eqs. 3, 5; Figs. 2b, 3b) and memory model."""
import json
import math
import os

import numpy as np
import pytest

from oracle import apply, hosvd, memory
from paper_2103_05822_gb300.inputs import complex_gaussian, synthetic_tucker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _tucker_from(sg):
    return hosvd.Tucker(sg.U_theta, sg.U_phi, sg.U_beta, sg.core)


@pytest.mark.parametrize("shape", [(5, 9, 13, (2, 3, 4)), (14, 28, 77, (10, 13, 45)), (4, 8, 1, (4, 1, 1))])
def test_tucker_procedures_equal_reconstructed_dense(shape):
    """Figs. 2b / 3b applied to the factors == Eqs. 3 / 5 applied to the reconstructed tensor."""
    nt, npf, nb, ranks = shape
    T = _tucker_from(synthetic_tucker(nt, npf, [nb], [[ranks, ranks]], seed=3)[0][0])
    A = hosvd.reconstruct(T)
    x = complex_gaussian((nb, 3), 5)
    g = complex_gaussian((nt * npf, 3), 6)
    w = np.random.default_rng(1).uniform(0.1, 1.0, nt * npf)
    assert np.allclose(apply.tucker_aggregate(T, x), apply.dense_aggregate(A, x), rtol=0, atol=1e-13)
    for weights in (None, w):
        assert np.allclose(apply.tucker_disaggregate(T, g, weights),
                           apply.dense_disaggregate(A, g, weights), rtol=0, atol=1e-13)


def test_dense_matrix_is_column_major_tensorisation():
    A = complex_gaussian((3, 4, 5), 2)
    P = apply.dense_matrix(A)
    for it in range(3):
        for ip in range(4):
            assert np.array_equal(P[it + 3 * ip], A[it, ip, :])


@pytest.mark.parametrize("tucker", [True, False])
def test_disaggregation_is_weighted_adjoint(sphere2_oracle, tucker):
    """<A x, W g> = <x, disagg(g)>: disaggregation is the quadrature-weighted adjoint."""
    P = sphere2_oracle
    ops = P.tucker if tucker else P.tensors
    x = complex_gaussian(P.n_rwg, 11)
    F = apply.aggregate_all(ops, P.groups.members, x, tucker=tucker)
    g = complex_gaussian(F.shape, 12)
    y = apply.disaggregate_all(ops, P.groups.members, g, P.n_rwg, P.grid.weights, tucker=tucker)
    lhs = np.vdot(P.grid.weights[None, None, :] * g, F)   # sum conj(W g) * (A x)
    rhs = np.vdot(y, x)                                   # sum conj(y) * x
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    y0 = apply.disaggregate_all(ops, P.groups.members, g, P.n_rwg, None, tucker=tucker)
    assert abs(np.vdot(g, F) - np.vdot(y0, x)) <= 1e-12 * abs(np.vdot(g, F))


def test_tucker_apply_error_within_truncation_bound(sphere2_oracle):
    P = sphere2_oracle
    x = complex_gaussian(P.n_rwg, 21)
    for g in (0, 11, 30):
        ids = P.groups.members[g]
        for a in range(2):
            A = P.tensors[g][a]
            T = P.tucker[g][a]
            err = np.linalg.norm(apply.tucker_aggregate(T, x[ids]) - apply.dense_aggregate(A, x[ids]))
            bound = np.linalg.norm(hosvd.reconstruct(T) - A) * np.linalg.norm(x[ids])
            assert err <= bound * (1 + 1e-12)
            assert bound <= P.tol * np.linalg.norm(A) * np.linalg.norm(x[ids])


def test_multi_rhs_columns_are_independent(sphere2_oracle):
    P = sphere2_oracle
    X = complex_gaussian((P.n_rwg, 4), 31)
    F = apply.aggregate_all(P.tucker, P.groups.members, X)
    for r in range(4):
        Fr = apply.aggregate_all(P.tucker, P.groups.members, X[:, r])
        assert np.allclose(F[..., r], Fr, rtol=0, atol=1e-13 * np.abs(Fr).max())
    y0 = complex_gaussian((P.n_rwg, 4), 32)
    y = apply.disaggregate_all(P.tucker, P.groups.members, F, P.n_rwg, P.grid.weights, beta=0.5 - 0.25j, y0=y0)
    yz = apply.disaggregate_all(P.tucker, P.groups.members, F, P.n_rwg, P.grid.weights)
    assert np.allclose(y, yz + (0.5 - 0.25j) * y0, rtol=0, atol=1e-13)


def test_linearity_and_group_locality(sphere2_oracle):
    P = sphere2_oracle
    x = np.zeros(P.n_rwg, complex)
    ids = P.groups.members[4]
    x[ids[3]] = 1.0
    F = apply.aggregate_all(P.tucker, P.groups.members, x)
    assert np.count_nonzero(np.abs(F).sum(axis=(1, 2))) == 1
    assert np.abs(F[4]).sum() > 0


def test_dense_memory_matches_paper_tables():
    gold = json.load(open(GOLDEN))["dense_memory_mb"]
    for row in gold:
        n_phi = 2 * row["L"] + 1
        mb = memory.dense_bytes(row["n_rwg"], row["L"], n_phi) / 2 ** 20
        # the tables print whole MiB (3694.44 -> 3694, 81783.38 -> 81784): agree to the last digit
        assert abs(mb - row["megabytes"]) < 1.0, row["cite"]
        # and FP32 or a single component would be off by 2x
        assert abs(mb / 2 - row["megabytes"]) > 1000


def test_tucker_memory_counts_every_array(sphere2_oracle):
    P = sphere2_oracle
    shapes = []
    nbytes = 0
    for g in range(P.groups.n_groups):
        for T in P.tucker[g]:
            rt, rp, rb = T.ranks
            shapes.append((T.U_theta.shape[0], T.U_phi.shape[0], T.U_beta.shape[0], rt, rp, rb))
            nbytes += sum(a.nbytes for a in (T.U_theta, T.U_phi, T.U_beta, T.core))
    assert memory.tucker_bytes(shapes) == nbytes
    dense = memory.dense_bytes(P.n_rwg, P.grid.L, P.grid.n_phi)
    assert dense == sum(a.nbytes for t in P.tensors for a in t)
    assert dense / nbytes > 1.0
