"""The truncated-SVD comparator of Sec. II.C (ref. [11]) on the GPU, against the oracle.

tfmm_params.compression = 1 makes the library compress every group's N_dir x
n_beta aggregation matrix by a truncated SVD at tolerance gamma (the note under
Table II) instead of the Tucker format, and its hot path applies
F = B (V^H x) and y = V (B^H W g).  On the 2-lambda sphere (0.5 lambda boxes,
3 digits, gamma = 1e-4) and on four groups of the 10-lambda sphere (gamma = 1e-6):
* the factors are orthonormal where the format says so and the ranks equal the
  oracle's SVD ranks (within one, at the truncation boundary);
* ||A_bar - B V^H||_F <= gamma ||A_bar||_F against the oracle's far-fields;
* the GPU apply equals the oracle's SVD apply of the GPU's own factors in FP32
  (l2 and element-wise, 1e-5 per output vector);
* end to end: within the gamma bound of the oracle's dense Eqs. 3 / 5;
* the stored bytes are the SVD format's (n_beta + N_dir) r per group and component.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import apply, svd as osvd
from paper_2103_05822_gb300.inputs import WORKLOADS, complex_gaussian

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = WORKLOADS["sphere2"]
TOL = 1e-5


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _elem(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


@pytest.fixture(scope="module")
def svd_plan(sphere2_mesh):
    from paper_2103_05822_gb300 import tfmm
    v, f = sphere2_mesh
    mesh = tfmm.tfmm_mesh_create(v, f)
    prm = tfmm.tfmm_params_default(k=2 * math.pi, box=W.box, digits=float(W.digits), tol=W.tol, max_rhs=3,
                                   compression=tfmm.SVD)
    return tfmm.tfmm_plan_create(mesh, prm)


def _svd_factors(plan, g, a):
    """(B, V) of group g, component a from the plan's Tucker-format export."""
    from paper_2103_05822_gb300 import tfmm
    Ut, Up, Ub, C = tfmm.tfmm_plan_export_factors(plan, g, a)
    nt, npf = Ut.shape[0], Up.shape[0]
    assert Ut.shape == (nt, nt) and Up.shape == (npf, npf)
    assert np.array_equal(Ut, np.eye(nt)) and np.array_equal(Up, np.eye(npf))
    r = C.shape[2]
    B = C.reshape(nt * npf, r, order="F")  # column c = vec of core slice c, direction i_theta + n_theta i_phi
    return osvd.SVDFactors(B, Ub.conj())


def test_svd_factors_ranks_and_bound(svd_plan, sphere2_oracle):
    P = sphere2_oracle
    for g in range(P.groups.n_groups):
        for a in range(2):
            S = _svd_factors(svd_plan, g, a)
            assert np.allclose(S.V.conj().T @ S.V, np.eye(S.rank), atol=1e-10)
            M = apply.dense_matrix(P.tensors[g][a])
            err = np.linalg.norm(osvd.reconstruct(S) - M)
            assert err <= (W.tol * 1.0001 + 1e-8) * np.linalg.norm(M), (g, a)
            ro = osvd.truncated_svd(P.tensors[g][a], W.tol).rank
            assert abs(S.rank - ro) <= 1, (g, a, S.rank, ro)


def test_svd_apply_matches_oracle_with_gpu_factors(svd_plan, sphere2_oracle):
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    info = svd_plan.info
    G, nd, n, R = info["n_groups"], info["n_dir"], info["n_rwg"], 3
    X = complex_gaussian((R, n), 41)
    gin = complex_gaussian((R, G, 2, nd), 42)
    xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    spec = torch.full((R, G, 2, nd), float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(svd_plan, xd, spec)
    gd = torch.from_numpy(gin.astype(np.complex64)).cuda()
    yd = torch.full((R, n), float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(svd_plan, gd, yd)
    torch.cuda.synchronize()
    S_all = [[_svd_factors(svd_plan, g, a) for a in range(2)] for g in range(G)]
    Sg, Y = spec.cpu().numpy(), yd.cpu().numpy()
    for r in range(R):
        y_ref = np.zeros(n, complex)
        for g, ids in enumerate(P.groups.members):
            for a in range(2):
                ref = osvd.svd_aggregate(S_all[g][a], X[r, ids])
                assert _rel(Sg[r, g, a], ref) <= TOL and _elem(Sg[r, g, a], ref) <= TOL, (r, g, a)
                y_ref[ids] += osvd.svd_disaggregate(S_all[g][a], gin[r, g, a], P.grid.weights)
        for ids in P.groups.members:
            assert _rel(Y[r, ids], y_ref[ids]) <= TOL and _elem(Y[r, ids], y_ref[ids]) <= TOL, r


def test_svd_end_to_end_against_dense_oracle(svd_plan, sphere2_oracle):
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    info = svd_plan.info
    x = complex_gaussian(P.n_rwg, 7)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    spec = torch.empty((1, info["n_groups"], 2, info["n_dir"]), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(svd_plan, xd, spec)
    y = torch.zeros(P.n_rwg, dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(svd_plan, spec, y)
    torch.cuda.synchronize()
    F = apply.aggregate_all(P.tensors, P.groups.members, x, tucker=False)
    got = spec.cpu().numpy()[0]
    for g in range(P.groups.n_groups):
        xn = np.linalg.norm(x[P.groups.members[g]])
        for a in range(2):
            bound = W.tol * np.linalg.norm(P.tensors[g][a]) * xn
            assert np.linalg.norm(got[g, a] - F[g, a]) <= bound + 1e-5 * np.linalg.norm(F[g, a])
    yo = apply.disaggregate_all(P.tensors, P.groups.members, got.astype(np.complex128), P.n_rwg, P.grid.weights,
                                tucker=False)
    assert np.linalg.norm(y.cpu().numpy() - yo) <= W.tol * np.linalg.norm(yo)


def test_svd_memory_is_the_svd_format(svd_plan):
    from paper_2103_05822_gb300 import tfmm
    info = svd_plan.info
    nd = info["n_dir"]
    total = 0
    for g in range(info["n_groups"]):
        for a in range(2):
            nb, (rt, rp, rb) = tfmm.tfmm_plan_group(svd_plan, g, a)
            assert (rt, rp) == (info["n_theta"], info["n_phi"])
            total += (nb + nd) * rb
    assert info["tucker_bytes_alg"] == 8 * total


def test_svd_ranks_on_paper_shaped_groups():
    """10-lambda sphere, 1-lambda boxes, 6 digits, gamma = 1e-6: the SVD ranks of four groups
    equal the oracle's and the bound holds; the SVD keeps no more than the Tucker beta rank
    of the same group (gamma vs gamma / sqrt(3) on the same singular values)."""
    from paper_2103_05822_gb300 import tfmm
    from paper_2103_05822_gb300.inputs import icosphere
    w = WORKLOADS["sphere10"]
    v, f = icosphere(w.diameter, w.nu)
    mesh = tfmm.tfmm_mesh_create(v, f)
    prm = dict(k=2 * math.pi, box=w.box, digits=float(w.digits), tol=w.tol)
    plan_s = tfmm.tfmm_plan_create(mesh, tfmm.tfmm_params_default(**prm, compression=tfmm.SVD))
    plan_t = tfmm.tfmm_plan_create(mesh, tfmm.tfmm_params_default(**prm))
    members = tfmm.tfmm_plan_members(plan_s)
    sizes = np.array([len(m) for m in members])
    order = np.argsort(sizes, kind="stable")
    pick = sorted({int(order[i]) for i in np.linspace(0, len(order) - 1, 4).round().astype(int)})
    P = oracle.problem.build(v, f, k=2 * math.pi, box=w.box, digits=w.digits, tol=w.tol, compress=False,
                             keep_tensors=True, groups_subset=pick)
    for g in pick:
        for a in range(2):
            S = _svd_factors(plan_s, g, a)
            M = apply.dense_matrix(P.tensors[g][a])
            assert np.linalg.norm(osvd.reconstruct(S) - M) <= (w.tol * 1.0001 + 1e-9) * np.linalg.norm(M), (g, a)
            ro = osvd.truncated_svd(P.tensors[g][a], w.tol).rank
            assert abs(S.rank - ro) <= 1, (g, a, S.rank, ro)
            assert S.rank <= tfmm.tfmm_plan_group(plan_t, g, a)[1][2] + 2
