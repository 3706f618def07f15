"""The translation stage on the GPU (tfmm_translate, FMM-FFT) against the oracle's direct sums.

1.5-lambda sphere, 0.5-lambda boxes, 5 digits (N_phi = 2L + 1), gamma = 1e-8:
* the incoming spectra of every group and component from seeded outgoing
  spectra against oracle.translation.translate (a double loop over far box
  pairs with T_L of ref. [25]);
* the whole far matvec, aggregation -> translation -> weighted disaggregation
  on the GPU, against the direct EFIE double integral of RWG pairs in far boxes
  (the FMM accuracy of 5 digits, as the oracle's own pin, plus the FP32 rounding
  of the spectra through the quadrature sum, whose cancellation is measured);
* R = 2 equals two single calls; touching boxes receive nothing from each
  other (beyond the FFT's FP32 rounding); a plan without box geometry is refused.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import apply, translation
from paper_2103_05822_gb300.inputs import complex_gaussian, icosphere

from test_oracle_farfield import _direct_efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2103_05822_gb300 import tfmm
    v, f = icosphere(1.5, 6)
    P = oracle.problem.build(v, f, k=2 * math.pi, box=0.5, digits=5, tol=1e-8, nphi_rule="2L+1", compress=False)
    mesh = tfmm.tfmm_mesh_create(v, f)
    prm = tfmm.tfmm_params_default(k=2 * math.pi, box=0.5, digits=5.0, tol=1e-8, nphi_rule=0, max_rhs=2)
    plan = tfmm.tfmm_plan_create(mesh, prm)
    assert plan.info["n_groups"] == P.groups.n_groups and plan.info["L"] == P.grid.L
    return v, f, P, plan


def test_translation_matches_direct_sums(setup):
    from paper_2103_05822_gb300 import tfmm
    v, f, P, plan = setup
    G, nd = P.groups.n_groups, P.grid.n_dir
    F = complex_gaussian((G, 2, nd), 3)
    ref = translation.translate(F, P.groups, P.grid, P.k)
    fo = torch.from_numpy(F.astype(np.complex64)).cuda().reshape(1, G, 2, nd)
    gi = torch.full_like(fo, float("nan"))
    tfmm.tfmm_translate(plan, fo, gi)
    torch.cuda.synchronize()
    got = gi.cpu().numpy()[0]
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    worst = max(np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g]) for g in range(G))
    elem = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"translation: whole {rel:.2e}, worst group {worst:.2e}, element-wise {elem:.2e}")
    assert rel <= 1e-5 and worst <= 1e-4 and elem <= 1e-5


def test_far_matvec_column_matches_direct_efie(setup):
    from paper_2103_05822_gb300 import tfmm
    v, f, P, plan = setup
    G, nd, N = P.groups.n_groups, P.grid.n_dir, P.n_rwg
    rng = np.random.default_rng(8)
    n = int(rng.integers(N))
    gn = next(g for g, m in enumerate(P.groups.members) if n in m)
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    x[n] = 1.0
    so = torch.empty((1, G, 2, nd), dtype=torch.complex64, device="cuda")
    si = torch.empty_like(so)
    y = torch.empty(N, dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, x, so)
    tfmm.tfmm_translate(plan, so, si)
    tfmm.tfmm_disaggregate(plan, si, y)
    torch.cuda.synchronize()
    yh = y.cpu().numpy()
    far = [g for g in range(G) if translation.is_far(P.groups.box_index[g], P.groups.box_index[gn])]
    near = [g for g in range(G) if g not in far]
    # touching boxes get no far interaction: only the FFT's FP32 rounding (relative to the
    # largest spectrum value over the grid) reaches them
    scale = np.max(np.abs(yh))
    for g in near:
        assert np.max(np.abs(yh[P.groups.members[g]])) <= 1e-3 * scale
    # sampled far entries against the direct EFIE: the FMM accuracy of 5 digits (as the
    # oracle's own pin) plus the FP32 rounding of the incoming spectra carried through the
    # quadrature sum of Fig. 3b.  That sum cancels strongly with 0.5-lambda boxes (T_L at
    # two box widths grows fast with l): sum |w A| max|g| exceeds |y_m| by up to ~1e5 here,
    # and the translation is accurate to 1e-5 of max|g| per element (the test above), so
    # an entry may be off by 1e-5 sum_dir |w A_m| max_alpha-group |g|.
    gmax = np.abs(si.cpu().numpy()[0]).max(axis=2, keepdims=True) * np.ones((1, 1, nd))
    absA = [[np.abs(A) for A in per] for per in P.tensors]
    cond = np.abs(apply.disaggregate_all(absA, P.groups.members, gmax, N, P.grid.weights, tucker=False))
    worst = 0.0
    for g in rng.choice(far, size=min(6, len(far)), replace=False):
        for m in rng.choice(P.groups.members[g], size=2, replace=False):
            z = _direct_efie(P.verts, P.tris, P.rwg, int(m), n, P.k)
            worst = max(worst, abs(yh[m] - z) / (1e-4 * abs(z) + 1e-5 * cond[m]))
    print("GPU far column worst error / (FMM + FP32 bound)", worst)
    assert worst <= 1.0


def test_two_columns_equal_single_calls(setup):
    from paper_2103_05822_gb300 import tfmm
    v, f, P, plan = setup
    G, nd = P.groups.n_groups, P.grid.n_dir
    F = torch.from_numpy(complex_gaussian((2, G, 2, nd), 4).astype(np.complex64)).cuda()
    g2 = torch.empty_like(F)
    tfmm.tfmm_translate(plan, F, g2)
    g0 = torch.empty_like(F[:1])
    g1 = torch.empty_like(F[:1])
    tfmm.tfmm_translate(plan, F[:1].contiguous(), g0)
    tfmm.tfmm_translate(plan, F[1:].contiguous(), g1)
    torch.cuda.synchronize()
    assert torch.equal(g2[:1], g0) and torch.equal(g2[1:], g1)


def test_plan_without_geometry_is_refused():
    from paper_2103_05822_gb300 import tfmm
    from paper_2103_05822_gb300.inputs import synthetic_tucker
    syn = synthetic_tucker(4, 8, [5, 3], [[(2, 2, 2), (2, 2, 2)]] * 2, 1)
    factors = [[(s.U_theta, s.U_phi, s.U_beta, s.core) for s in per] for per in syn]
    plan = tfmm.tfmm_plan_from_tucker(8, 4, 8, [np.arange(5), np.arange(5, 8)], factors)
    so = torch.zeros((1, 2, 2, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_translate(plan, so, torch.empty_like(so))
    assert e.value.status == tfmm.INVALID_ARG
