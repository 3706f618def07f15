"""The GPU compressor meets the Tucker bound of Eq. 6 at tight tolerances.

Sec. III.A truncates every mode at gamma / sqrt(3) of ||A||_F, which bounds the
whole reconstruction error by gamma ||A||_F (the HOSVD bound of ref. [26]).  The
library compresses in FP64 on the GPU; here, for sampled groups of full-size
plans, the exported FP64 factors are multiplied out on the host in FP64 and
compared with the group's FP64 far-field tensors (Eq. 4, recomputed on the GPU by
tfmm_plan_farfield with the same quadrature the compression used):

    ||A - C x1 U_theta x2 U_phi x3 U_beta||_F <= gamma ||A||_F

at gamma = 1e-6 (10-lambda sphere, 1-lambda boxes) and gamma = 1e-8 (20-lambda
sphere, 1- and 2-lambda boxes, the tightest point of the parameter sweep).  The
check itself is exact to ~1e-15 ||A||_F, far below both bounds.  The factors
must also be orthonormal (U^H U = I to 1e-10) and the ranks within the tensor
sizes.
"""
import math

import numpy as np
import pytest

from oracle import hosvd
from paper_2103_05822_gb300.inputs import WORKLOADS, icosphere

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    # name: (diameter, nu, box, digits, gamma)
    "sphere10_g1e-6": (10.0, 60, 1.0, 6, 1e-6),
    "sphere20_box1_g1e-8": (20.0, 120, 1.0, 6, 1e-8),
    "sphere20_box2_g1e-8": (20.0, 120, 2.0, 6, 1e-8),
}


def _sample(sizes, count=6):
    """Group ids at evenly spaced size quantiles, the largest and the smallest included."""
    order = np.argsort(sizes, kind="stable")
    q = np.linspace(0, len(order) - 1, count).round().astype(int)
    return sorted({int(order[i]) for i in q})


@pytest.fixture(scope="module", params=sorted(CASES))
def plan_case(request):
    from paper_2103_05822_gb300 import tfmm
    d, nu, box, digits, gamma = CASES[request.param]
    v, f = icosphere(d, nu)
    mesh = tfmm.tfmm_mesh_create(v, f)
    prm = tfmm.tfmm_params_default(k=2 * math.pi, box=box, digits=float(digits), tol=gamma, max_rhs=1)
    plan = tfmm.tfmm_plan_create(mesh, prm)
    return request.param, gamma, plan


def test_reconstruction_within_tucker_bound(plan_case):
    from paper_2103_05822_gb300 import tfmm
    name, gamma, plan = plan_case
    members = tfmm.tfmm_plan_members(plan)
    sizes = np.array([len(m) for m in members])
    worst = 0.0
    for g in _sample(sizes):
        A_pair = tfmm.tfmm_plan_farfield(plan, g)
        for a in range(2):
            Ut, Up, Ub, C = tfmm.tfmm_plan_export_factors(plan, g, a)
            for U in (Ut, Up, Ub):
                assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), rtol=0, atol=1e-10), (name, g, a)
            A = A_pair[a]
            nt, npf, nb = A.shape
            rt, rp, rb = C.shape
            assert 1 <= rt <= nt and 1 <= rp <= npf and 1 <= rb <= min(nb, rt * rp)
            Ah = hosvd.reconstruct(hosvd.Tucker(Ut, Up, Ub, C))
            rel = np.linalg.norm(Ah - A) / np.linalg.norm(A)
            worst = max(worst, rel)
            assert rel <= gamma, (name, g, a, rel, (rt, rp, rb))
    print(f"{name}: worst ||A - A_hat|| / ||A|| = {worst:.3e} (gamma {gamma:g})")
