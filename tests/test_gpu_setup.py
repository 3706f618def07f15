"""GPU setup parity on the 2-lambda sphere (0.5 lambda boxes, 3 digits, gamma = 1e-4).

The library builds its own groups, grid, far-fields (Eq. 4, FP64 on the GPU)
and sequentially truncated HOSVD (Eq. 6, FP64 on the GPU) from the mesh; the
oracle builds its own from the same mesh.  Checks:
* groups and RWG membership: bit-exact;
* quadrature nodes: to rounding;
* far-field tensors: element-wise, relative 1e-9 (two quadrature rules of
  different order, both converged far below that);
* compression: factors orthonormal, ||A_oracle - A_hat_gpu||_F <= gamma ||A||_F
  (plus the 1e-9 far-field difference), ranks within the rank bounds;
* end to end: GPU Tucker aggregation / disaggregation against the oracle's dense
  Eqs. 3 / 5 within the Tucker bound and FP32 rounding;
* plane-wave excitation against the oracle's, FP32 rounding.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import apply, hosvd, planewave
from paper_2103_05822_gb300.inputs import WORKLOADS, complex_gaussian

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = WORKLOADS["sphere2"]


@pytest.fixture(scope="module")
def gpu_plan(sphere2_mesh):
    from paper_2103_05822_gb300 import tfmm
    v, f = sphere2_mesh
    mesh = tfmm.tfmm_mesh_create(v, f)
    prm = tfmm.tfmm_params_default(k=2 * math.pi, box=W.box, digits=float(W.digits), tol=W.tol,
                                   keep_dense=1, max_rhs=2)
    plan = tfmm.tfmm_plan_create(mesh, prm)
    return plan


def test_groups_and_grid_match_oracle(gpu_plan, sphere2_oracle):
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    info = gpu_plan.info
    assert info["L"] == P.grid.L == 13
    assert (info["n_theta"], info["n_phi"]) == (14, 28)
    assert info["n_groups"] == P.groups.n_groups
    assert tuple(info["K"]) == P.groups.K
    members = tfmm.tfmm_plan_members(gpu_plan)
    for a, b in zip(members, P.groups.members):
        assert np.array_equal(a, b)
    assert np.array_equal(tfmm.tfmm_plan_centres(gpu_plan), P.groups.centre)
    th, wt, ph, wp = tfmm.tfmm_plan_quadrature(gpu_plan)
    assert np.allclose(th, P.grid.theta, rtol=0, atol=1e-13)
    assert np.allclose(wt, P.grid.w_theta, rtol=0, atol=1e-14)
    assert np.allclose(ph, P.grid.phi, rtol=0, atol=1e-14) and abs(wp - P.grid.w_phi) < 1e-15


def test_far_field_tensors_match_oracle(gpu_plan, sphere2_oracle):
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    for g in (0, 9, P.groups.n_groups - 1):
        At, Ap = tfmm.tfmm_plan_farfield(gpu_plan, g)
        for got, ref in ((At, P.tensors[g][0]), (Ap, P.tensors[g][1])):
            err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err < 1e-9, (g, err)


def test_compression_meets_tucker_bound(gpu_plan, sphere2_oracle):
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    for g in range(P.groups.n_groups):
        for a in range(2):
            Ut, Up, Ub, C = tfmm.tfmm_plan_export_factors(gpu_plan, g, a)
            for U in (Ut, Up, Ub):
                assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-10)
            A = P.tensors[g][a]
            Ah = hosvd.reconstruct(hosvd.Tucker(Ut, Up, Ub, C))
            assert np.linalg.norm(Ah - A) <= (W.tol * 1.0001 + 1e-8) * np.linalg.norm(A)
            nt, npf, nb = A.shape
            rt, rp, rb = C.shape
            assert rt <= nt and rp <= npf and rb <= min(nb, rt * rp)
            # the oracle's plain T-HOSVD ranks are an upper bound of the sequential ones, near them
            ro = P.tucker[g][a].ranks
            assert rt == ro[0] and rp <= ro[1] and rb <= ro[2] + 2


def test_end_to_end_against_dense_oracle(gpu_plan, sphere2_oracle):
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    info = gpu_plan.info
    x = complex_gaussian(P.n_rwg, W.seed)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    spec = torch.empty((1, info["n_groups"], 2, info["n_dir"]), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(gpu_plan, xd, spec)
    dspec = torch.empty_like(spec)
    tfmm.tfmm_aggregate_dense(gpu_plan, xd, dspec)
    y = torch.zeros(P.n_rwg, dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(gpu_plan, spec, y)
    yd = torch.zeros_like(y)
    tfmm.tfmm_disaggregate_dense(gpu_plan, spec, yd)
    torch.cuda.synchronize()
    F = apply.aggregate_all(P.tensors, P.groups.members, x, tucker=False)
    got = spec.cpu().numpy()[0]
    # per group: ||(A - A_hat) x|| <= gamma ||A||_F ||x|| (+ FP32 rounding)
    for g in range(P.groups.n_groups):
        xn = np.linalg.norm(x[P.groups.members[g]])
        for a in range(2):
            bound = W.tol * np.linalg.norm(P.tensors[g][a]) * xn
            assert np.linalg.norm(got[g, a] - F[g, a]) <= bound + 1e-5 * np.linalg.norm(F[g, a])
    rel = np.linalg.norm(got - F) / np.linalg.norm(F)
    assert rel < W.tol
    # dense GPU path: FP32 rounding only
    assert np.linalg.norm(dspec.cpu().numpy()[0] - F) <= 1e-5 * np.linalg.norm(F)
    Sd = got.astype(np.complex128)
    yo = apply.disaggregate_all(P.tensors, P.groups.members, Sd, P.n_rwg, P.grid.weights, tucker=False)
    assert np.linalg.norm(yd.cpu().numpy() - yo) <= 1e-5 * np.linalg.norm(yo)
    assert np.linalg.norm(y.cpu().numpy() - yo) <= W.tol * np.linalg.norm(yo)


def test_oracle_factors_through_gpu_kernels(sphere2_oracle):
    """The oracle's own T-HOSVD factors run through the GPU kernels: FP32 rounding only."""
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    factors = [[(t.U_theta, t.U_phi, t.U_beta, t.core) for t in per] for per in P.tucker]
    plan = tfmm.tfmm_plan_from_tucker(P.n_rwg, P.grid.n_theta, P.grid.n_phi, P.groups.members, factors,
                                      weights=P.grid.weights)
    x = complex_gaussian(P.n_rwg, 77)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    spec = torch.empty((1, P.groups.n_groups, 2, P.grid.n_dir), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, xd, spec)
    y = torch.zeros(P.n_rwg, dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(plan, spec, y)
    torch.cuda.synchronize()
    F = apply.aggregate_all(P.tucker, P.groups.members, x)
    assert np.linalg.norm(spec.cpu().numpy()[0] - F) <= 1e-5 * np.linalg.norm(F)
    yo = apply.disaggregate_all(P.tucker, P.groups.members, spec.cpu().numpy()[0].astype(np.complex128),
                                P.n_rwg, P.grid.weights)
    assert np.linalg.norm(y.cpu().numpy() - yo) <= 1e-5 * np.linalg.norm(yo)


def test_planewave_excitation_matches_oracle(gpu_plan, sphere2_oracle):
    from paper_2103_05822_gb300 import tfmm
    P = sphere2_oracle
    angles = [(0.0, 0.0), (0.7, 1.3), (math.pi, 0.0)]
    kh, pol = [], []
    for t, p in angles:
        k_inc, th, ph = planewave.incidence(t, p)
        kh.append(k_inc)
        pol.append(th)
    V = torch.empty((len(angles), P.n_rwg), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_planewave(gpu_plan, np.array(kh), np.array(pol), V)
    torch.cuda.synchronize()
    got = V.cpu().numpy()
    for r in range(len(angles)):
        ref = planewave.planewave_rhs(P.verts, P.rwg, P.k, kh[r], pol[r])
        assert np.linalg.norm(got[r] - ref) <= 1e-6 * np.linalg.norm(ref)
