"""Pins of the oracle's translation stage (Sec. II.A; refs. [7, 8], addition theorem of [25]).

The far part of Z x assembled as aggregation -> translation -> weighted
disaggregation must reproduce the EFIE interaction of RWG pairs in far boxes,
computed directly as the mixed-potential double integral with the Green's
function exp(-jkR)/(4 pi R) by the test's own quadrature:
* column n of the far matvec (x = e_n) against the direct Z_mn for RWGs m in
  boxes far from n's box, within the FMM accuracy 10^-(d0 - 1) (worst) of the
  two-group pin in test_oracle_farfield.py;
* pairs in touching boxes get nothing (their interaction is the near field);
* the same with the Tucker factors (gamma = 1e-8) in place of the dense
  tensors, and the far matvec is linear.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import apply, hosvd, translation
from paper_2103_05822_gb300.inputs import complex_gaussian, icosphere

from test_oracle_farfield import _direct_efie


@pytest.fixture(scope="module")
def small_problem():
    """A 1.5-lambda sphere in 0.5-lambda boxes, 5 digits: far box pairs exist."""
    v, f = icosphere(1.5, 6)
    P = oracle.problem.build(v, f, k=2 * math.pi, box=0.5, digits=5, tol=1e-8, nphi_rule="2L+1")
    return v, f, P


@pytest.mark.parametrize("tucker", [False, True])
def test_far_column_matches_direct_efie(small_problem, tucker):
    v, f, P = small_problem
    k = P.k
    rng = np.random.default_rng(4)
    n = int(rng.integers(P.n_rwg))
    gn = next(g for g, m in enumerate(P.groups.members) if n in m)
    x = np.zeros(P.n_rwg, complex)
    x[n] = 1.0
    y = translation.far_matvec(P.tucker if tucker else P.tensors, P.groups, P.grid, x, k, tucker=tucker)
    far = [g for g in range(P.groups.n_groups) if translation.is_far(P.groups.box_index[g], P.groups.box_index[gn])]
    near = [g for g in range(P.groups.n_groups) if g not in far]
    assert far and near
    for g in near:  # touching boxes (and n's own) get no far interaction
        assert np.all(y[P.groups.members[g]] == 0)
    worst = 0.0
    for g in rng.choice(far, size=min(6, len(far)), replace=False):
        for m in rng.choice(P.groups.members[g], size=2, replace=False):
            z = _direct_efie(P.verts, P.tris, P.rwg, int(m), n, k)
            worst = max(worst, abs(y[m] - z) / abs(z))
    print("far column worst rel err", "tucker" if tucker else "dense", worst)
    assert worst <= 1e-4


def test_far_matvec_is_linear(small_problem):
    v, f, P = small_problem
    x = complex_gaussian(P.n_rwg, 9)
    x2 = complex_gaussian(P.n_rwg, 10)
    y1 = translation.far_matvec(P.tucker, P.groups, P.grid, x, P.k)
    y2 = translation.far_matvec(P.tucker, P.groups, P.grid, x2, P.k)
    y12 = translation.far_matvec(P.tucker, P.groups, P.grid, x + 2j * x2, P.k)
    assert np.linalg.norm(y12 - (y1 + 2j * y2)) <= 1e-12 * np.linalg.norm(y12)
