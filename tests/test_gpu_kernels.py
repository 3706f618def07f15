"""GPU parity of the hot-path kernels against the FP64 oracle (Figs. 2b, 3b; Eqs. 3, 5).

The factors are seeded synthetic inputs with ragged shapes, given to both sides:
the oracle applies the Tucker procedures in complex128, the library runs its
FP32 kernels through the C ABI.  Tolerance: per output vector (one RHS, group
and component), relative l2 error <= 1e-5 and every element within 1e-5 of the
vector's largest magnitude (FP32 storage of the factors, ~6e-8 each, and FP32
accumulation over at most a few thousand terms).  The element-wise check keeps
a wrong low-magnitude band (a direction row, the last phi column of an odd
grid) from hiding under the norm of a long vector.

The split-BF16 tensor-core chain with three terms holds every FP32 operand
exactly and accumulates in chunks of at most four K steps per TMEM accumulator;
it is held to the Tucker tolerance gamma = 1e-6 of the many-RHS workload.  Two
terms keep 16 significant bits per operand and are held to 5e-5.
"""
import math

import numpy as np
import pytest

from oracle import apply, hosvd
from paper_2103_05822_gb300.inputs import complex_gaussian, synthetic_tucker

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _tfmm():
    from paper_2103_05822_gb300 import tfmm
    return tfmm


def _case(seed, n_theta, n_phi, nbetas, rank_fn):
    rng = np.random.default_rng(seed)
    ranks = [rank_fn(rng, nb) for nb in nbetas]
    syn = synthetic_tucker(n_theta, n_phi, nbetas, ranks, seed)
    n_rwg = sum(nbetas)
    perm = rng.permutation(n_rwg)
    members, pos = [], 0
    for nb in nbetas:
        members.append(np.sort(perm[pos:pos + nb]))
        pos += nb
    T = [[hosvd.Tucker(s.U_theta, s.U_phi, s.U_beta, s.core) for s in per] for per in syn]
    factors = [[(t.U_theta, t.U_phi, t.U_beta, t.core) for t in per] for per in T]
    return n_rwg, members, T, factors


CASES = {
    # name: (n_theta, n_phi, n_beta per group, rank function)
    "tiny": (3, 6, [1, 2, 5], lambda rng, nb: [(1, 1, 1), (min(2, 3), 2, min(nb, 2))]),
    "ragged": (14, 28, [77, 12, 98, 3, 64], lambda rng, nb: [
        (int(rng.integers(1, 14)), int(rng.integers(1, 28)), int(rng.integers(1, nb + 1))) for _ in range(2)]),
    "paper_like": (40, 80, [940, 1786, 411], lambda rng, nb: [
        (int(rng.integers(24, 31)), int(rng.integers(28, 36)), int(rng.integers(170, 201))) for _ in range(2)]),
    "odd_grid": (13, 25, [33, 50], lambda rng, nb: [(5, 7, 9), (13, 25, 33 if nb == 33 else 50)]),
    # more phi samples than TMEM lanes: the tensor-core chain runs AG3 and AG4 apart
    "wide": (9, 136, [60, 33], lambda rng, nb: [(int(rng.integers(1, 10)), int(rng.integers(20, 60)),
                                                 int(rng.integers(1, nb + 1))) for _ in range(2)]),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    tfmm = _tfmm()
    nt, npf, nbetas, rank_fn = CASES[request.param]
    n_rwg, members, T, factors = _case(100 + sorted(CASES).index(request.param), nt, npf, nbetas, rank_fn)
    w = np.random.default_rng(5).uniform(0.05, 1.0, nt * npf)
    plan = tfmm.tfmm_plan_from_tucker(n_rwg, nt, npf, members, factors, weights=w, max_rhs=4)
    return dict(plan=plan, n_rwg=n_rwg, members=members, T=T, w=w, nt=nt, npf=npf, G=len(members))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _elem(a, b):
    """Largest element-wise error relative to the largest reference magnitude."""
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def _close(a, b, tol):
    """Both the relative l2 error and the element-wise error within tol."""
    return _rel(a, b) <= tol and _elem(a, b) <= tol


def test_aggregate_matches_oracle(case):
    tfmm = _tfmm()
    x = complex_gaussian(case["n_rwg"], 11)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    spec = torch.full((1, case["G"], 2, case["nt"] * case["npf"]), float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(case["plan"], xd, spec)
    torch.cuda.synchronize()
    got = spec.cpu().numpy()[0]
    ref = apply.aggregate_all(case["T"], case["members"], x)
    assert np.isfinite(got).all()
    for g in range(case["G"]):
        for a in range(2):
            assert _close(got[g, a], ref[g, a], TOL), (g, a, _rel(got[g, a], ref[g, a]), _elem(got[g, a], ref[g, a]))


@pytest.mark.parametrize("weights,beta", [(True, 0.0), (False, 0.0), (True, 0.5 - 0.25j)])
def test_disaggregate_matches_oracle(case, weights, beta):
    tfmm = _tfmm()
    G, nd = case["G"], case["nt"] * case["npf"]
    g_in = complex_gaussian((G, 2, nd), 12)
    y0 = complex_gaussian(case["n_rwg"], 13)
    gd = torch.from_numpy(g_in.astype(np.complex64)).cuda().reshape(1, G, 2, nd)
    yd = torch.from_numpy(y0.astype(np.complex64)).cuda()
    tfmm.tfmm_disaggregate(case["plan"], gd, yd, apply_weights=weights, beta=beta)
    torch.cuda.synchronize()
    got = yd.cpu().numpy()
    ref = apply.disaggregate_all(case["T"], case["members"], g_in, case["n_rwg"],
                                 case["w"] if weights else None, beta=beta, y0=y0)
    for g, ids in enumerate(case["members"]):
        assert _close(got[ids], ref[ids], TOL), (g, _rel(got[ids], ref[ids]), _elem(got[ids], ref[ids]))


def test_multi_rhs_and_leading_dimension(case):
    tfmm = _tfmm()
    R, n = 3, case["n_rwg"]
    ld = n + 5
    X = complex_gaussian((R, ld), 21)
    xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    spec = torch.empty((R, case["G"], 2, case["nt"] * case["npf"]), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(case["plan"], xd, spec, R=R, ldx=ld)
    yd = torch.zeros((R, ld), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(case["plan"], spec, yd, R=R, ldy=ld)
    torch.cuda.synchronize()
    S = spec.cpu().numpy()
    Y = yd.cpu().numpy()
    for r in range(R):
        ref = apply.aggregate_all(case["T"], case["members"], X[r, :n])
        for g in range(case["G"]):
            for a in range(2):
                assert _close(S[r, g, a], ref[g, a], TOL), (r, g, a)
        refy = apply.disaggregate_all(case["T"], case["members"], S[r].astype(np.complex128), n, case["w"])
        for ids in case["members"]:
            assert _close(Y[r, ids], refy[ids], TOL), r
        assert np.all(Y[r, n:] == 0)  # padding rows untouched


def test_repeated_launches_reuse_the_work_queue(case):
    """The self-resetting queue: identical results over many back-to-back launches."""
    tfmm = _tfmm()
    x = complex_gaussian(case["n_rwg"], 31)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    spec = torch.empty((1, case["G"], 2, case["nt"] * case["npf"]), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(case["plan"], xd, spec)
    first = spec.clone()
    for _ in range(20):
        tfmm.tfmm_aggregate(case["plan"], xd, spec)
    torch.cuda.synchronize()
    assert torch.equal(first, spec)


def test_adjointness_on_gpu_outputs(case):
    tfmm = _tfmm()
    G, nd, n = case["G"], case["nt"] * case["npf"], case["n_rwg"]
    x = complex_gaussian(n, 41)
    g_in = complex_gaussian((G, 2, nd), 42)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    spec = torch.empty((1, G, 2, nd), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(case["plan"], xd, spec)
    yd = torch.zeros(n, dtype=torch.complex64, device="cuda")
    gd = torch.from_numpy(g_in.astype(np.complex64)).cuda().reshape(1, G, 2, nd)
    tfmm.tfmm_disaggregate(case["plan"], gd, yd)
    torch.cuda.synchronize()
    F = spec.cpu().numpy()[0].astype(np.complex128)
    y = yd.cpu().numpy().astype(np.complex128)
    lhs = np.vdot(case["w"][None, None, :] * g_in, F)
    rhs = np.vdot(y, x)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(F) * np.linalg.norm(case["w"][None, None, :] * g_in)


def test_dense_kernels_match_oracle(case):
    tfmm = _tfmm()
    tensors = [[hosvd.reconstruct(t) for t in per] for per in case["T"]]
    tfmm.tfmm_plan_set_dense(case["plan"], tensors)
    G, nd, n = case["G"], case["nt"] * case["npf"], case["n_rwg"]
    x = complex_gaussian(n, 51)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    spec = torch.empty((1, G, 2, nd), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate_dense(case["plan"], xd, spec)
    yd = torch.zeros(n, dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate_dense(case["plan"], spec, yd)
    torch.cuda.synchronize()
    F = spec.cpu().numpy()[0]
    ref = apply.aggregate_all(tensors, case["members"], x, tucker=False)
    for g in range(G):
        for a in range(2):
            assert _close(F[g, a], ref[g, a], TOL), (g, a)
    refy = apply.disaggregate_all(tensors, case["members"], F.astype(np.complex128), n, case["w"], tucker=False)
    yg = yd.cpu().numpy()
    for ids in case["members"]:
        assert _close(yg[ids], refy[ids], TOL)


def test_host_matvec_equals_device_path(case):
    tfmm = _tfmm()
    n = case["n_rwg"]
    x = complex_gaussian(n, 61).astype(np.complex64)
    y = np.zeros(n, np.complex64)
    tfmm.tfmm_matvec_host(case["plan"], x, y)
    xd = torch.from_numpy(x).cuda()
    spec = torch.empty((1, case["G"], 2, case["nt"] * case["npf"]), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(case["plan"], xd, spec)
    yd = torch.zeros(n, dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(case["plan"], spec, yd)
    torch.cuda.synchronize()
    assert np.array_equal(y, yd.cpu().numpy())


def test_hot_path_argument_errors(case):
    tfmm = _tfmm()
    n = case["n_rwg"]
    xd = torch.zeros(n, dtype=torch.complex64, device="cuda")
    spec = torch.empty((8, case["G"], 2, case["nt"] * case["npf"]), dtype=torch.complex64, device="cuda")
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_aggregate(case["plan"], xd, spec, R=5)  # > max_rhs
    assert e.value.status == tfmm.INVALID_ARG
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_aggregate(case["plan"], xd, spec, R=1, ldx=n - 1)
    assert e.value.status == tfmm.INVALID_ARG


def test_from_tucker_rejects_bad_ranks():
    tfmm = _tfmm()
    n_rwg, members, T, factors = _case(3, 4, 8, [5], lambda rng, nb: [(2, 2, 2), (2, 2, 2)])
    Ut, Up, Ub, C = factors[0][0]
    bad = [[(Ut, Up, Ub, np.zeros((2, 2, 9), complex)), factors[0][1]]]  # r_beta 9 > n_beta 5
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_plan_from_tucker(n_rwg, 4, 8, members, bad)
    assert e.value.status == tfmm.INVALID_ARG
    with pytest.raises(tfmm.TfmmError):
        tfmm.tfmm_plan_from_tucker(n_rwg, 4, 8, [np.array([0, 0, 1, 2, 3])], factors)  # repeated id


@pytest.mark.parametrize("name,R", [("paper_like", 16), ("ragged", 7), ("odd_grid", 2)])
def test_multi_rhs_chain_matches_oracle(name, R):
    """R > 1 runs the grouped-GEMM chains (AG1-AG4, DG1-DG3); every column against the oracle."""
    tfmm = _tfmm()
    nt, npf, nbetas, rank_fn = CASES[name]
    n_rwg, members, T, factors = _case(300 + R, nt, npf, nbetas, rank_fn)
    w = np.random.default_rng(9).uniform(0.05, 1.0, nt * npf)
    plan = tfmm.tfmm_plan_from_tucker(n_rwg, nt, npf, members, factors, weights=w, max_rhs=R)
    G, nd = len(members), nt * npf
    X = complex_gaussian((R, n_rwg), 400 + R)
    xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, xd, spec)
    g_in = complex_gaussian((R, G, 2, nd), 500 + R)
    y0 = complex_gaussian((R, n_rwg), 600 + R)
    gd = torch.from_numpy(g_in.astype(np.complex64)).cuda()
    yd = torch.from_numpy(y0.astype(np.complex64)).cuda()
    beta = 0.25 + 0.5j
    tfmm.tfmm_disaggregate(plan, gd, yd, beta=beta)
    torch.cuda.synchronize()
    S = spec.cpu().numpy()
    Y = yd.cpu().numpy()
    for r in range(R):
        ref = apply.aggregate_all(T, members, X[r])
        for g in range(G):
            for a in range(2):
                assert _close(S[r, g, a], ref[g, a], TOL), (r, g, a)
        refy = apply.disaggregate_all(T, members, g_in[r], n_rwg, w, beta=beta, y0=y0[r])
        for ids in members:
            assert _close(Y[r, ids], refy[ids], TOL), r


@pytest.mark.parametrize("terms,tol", [(3, 1e-6), (2, 5e-5)])
@pytest.mark.parametrize("name,R", [("paper_like", 16), ("ragged", 7), ("odd_grid", 3), ("wide", 5),
                                    ("paper_like", 128)])
def test_tensor_core_chain_matches_oracle(name, R, terms, tol):
    """tcgen05 chains with FP32 operands split into `terms` BF16 terms, FP32 accumulation."""
    tfmm = _tfmm()
    nt, npf, nbetas, rank_fn = CASES[name]
    n_rwg, members, T, factors = _case(700 + R, nt, npf, nbetas, rank_fn)
    w = np.random.default_rng(19).uniform(0.05, 1.0, nt * npf)
    plan = tfmm.tfmm_plan_from_tucker(n_rwg, nt, npf, members, factors, weights=w, max_rhs=R, mrhs_precision=terms)
    G, nd = len(members), nt * npf
    X = complex_gaussian((R, n_rwg), 800 + R)
    xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    spec = torch.full((R, G, 2, nd), float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, xd, spec)
    g_in = complex_gaussian((R, G, 2, nd), 900 + R)
    y0 = complex_gaussian((R, n_rwg), 1000 + R)
    gd = torch.from_numpy(g_in.astype(np.complex64)).cuda()
    yd = torch.from_numpy(y0.astype(np.complex64)).cuda()
    beta = -0.5 + 0.125j
    tfmm.tfmm_disaggregate(plan, gd, yd, beta=beta)
    torch.cuda.synchronize()
    assert plan.info["kernel_errors"] == 0
    S = spec.cpu().numpy()
    Y = yd.cpu().numpy()
    assert np.isfinite(S).all() and np.isfinite(Y).all()
    worst = [0.0, 0.0]
    for r in range(R):
        ref = apply.aggregate_all(T, members, X[r])
        for g in range(G):
            for a in range(2):
                e = (_rel(S[r, g, a], ref[g, a]), _elem(S[r, g, a], ref[g, a]))
                worst[0] = max(worst[0], *e)
                assert max(e) <= tol, (r, g, a, e)
        refy = apply.disaggregate_all(T, members, g_in[r], n_rwg, w, beta=beta, y0=y0[r])
        for ids in members:
            e = (_rel(Y[r, ids], refy[ids]), _elem(Y[r, ids], refy[ids]))
            worst[1] = max(worst[1], *e)
            assert max(e) <= tol, (r, e)
    print(f"{name} R={R} terms={terms}: worst aggregation {worst[0]:.2e}, disaggregation {worst[1]:.2e}")


@pytest.mark.parametrize("terms", [3, 2])
def test_stacked_dg1_forms_match_the_generic_stage_kernel(terms, monkeypatch):
    """DG1a / DG1b with the BF16 terms of U_theta / U_phi stacked along N (the default when
    they fit) against the generic stage kernels (TFMM_TC_CAT=0 while the chain is planned)
    and the oracle: both within the chain's tolerance, and within twice it of each other."""
    tfmm = _tfmm()
    nt, npf, nbetas, rank_fn = CASES["paper_like"]
    R = 16
    n_rwg, members, T, factors = _case(700 + R, nt, npf, nbetas, rank_fn)
    w = np.random.default_rng(19).uniform(0.05, 1.0, nt * npf)
    G, nd = len(members), nt * npf
    g_in = complex_gaussian((R, G, 2, nd), 900 + R)
    gd = torch.from_numpy(g_in.astype(np.complex64)).cuda()
    tol = 1e-6 if terms == 3 else 5e-5
    out = {}
    for cat in ("1", "0"):
        monkeypatch.setenv("TFMM_TC_CAT", cat)
        plan = tfmm.tfmm_plan_from_tucker(n_rwg, nt, npf, members, factors, weights=w, max_rhs=R,
                                          mrhs_precision=terms)
        yd = torch.zeros((R, n_rwg), dtype=torch.complex64, device="cuda")
        tfmm.tfmm_disaggregate(plan, gd, yd)
        torch.cuda.synchronize()
        assert plan.info["kernel_errors"] == 0
        out[cat] = yd.cpu().numpy()
    monkeypatch.delenv("TFMM_TC_CAT")
    for r in range(R):
        refy = apply.disaggregate_all(T, members, g_in[r], n_rwg, w)
        for ids in members:
            for cat in ("1", "0"):
                assert _close(out[cat][r, ids], refy[ids], tol), (cat, r)
            assert _close(out["1"][r, ids], out["0"][r, ids], 2 * tol), r


@pytest.mark.parametrize("terms", [3, 2])
@pytest.mark.parametrize("name,R", [("paper_like", 16), ("ragged", 7)])
def test_tma_fed_stages_equal_the_cp_async_kernel(name, R, terms, monkeypatch):
    """AG1, AG2, DG2 and DG3 fed by the tensor-memory accelerator (the default) against
    the same stages with operands staged by cp.async (TFMM_TC_TMA=0 while the chain is
    planned): the same MMAs in the same order, so the same bits."""
    tfmm = _tfmm()
    nt, npf, nbetas, rank_fn = CASES[name]
    n_rwg, members, T, factors = _case(700 + R, nt, npf, nbetas, rank_fn)
    w = np.random.default_rng(19).uniform(0.05, 1.0, nt * npf)
    G, nd = len(members), nt * npf
    X = torch.from_numpy(complex_gaussian((R, n_rwg), 800 + R).astype(np.complex64)).cuda()
    g_in = torch.from_numpy(complex_gaussian((R, G, 2, nd), 900 + R).astype(np.complex64)).cuda()
    out = {}
    for tma in ("1", "0"):
        monkeypatch.setenv("TFMM_TC_TMA", tma)
        plan = tfmm.tfmm_plan_from_tucker(n_rwg, nt, npf, members, factors, weights=w, max_rhs=R,
                                          mrhs_precision=terms)
        spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
        tfmm.tfmm_aggregate(plan, X, spec)
        y = torch.zeros((R, n_rwg), dtype=torch.complex64, device="cuda")
        tfmm.tfmm_disaggregate(plan, g_in, y)
        torch.cuda.synchronize()
        assert plan.info["kernel_errors"] == 0
        out[tma] = (spec, y)
    monkeypatch.delenv("TFMM_TC_TMA")
    assert torch.equal(out["1"][0], out["0"][0]) and torch.equal(out["1"][1], out["0"][1])


def test_tensor_core_chain_on_far_field_factors():
    """The 3-term tensor-core chain on the oracle's own T-HOSVD factors of real far-field
    tensors (orthonormal factors, paper-shaped ranks): 10-lambda sphere, 1-lambda boxes,
    6 digits (26 x 52 directions), gamma = 1e-6, four groups at size quantiles, 128 RHS.
    Every (RHS, group, component) spectrum and every group's currents within gamma of the
    oracle's Tucker procedures with the same factors, in l2 and element-wise."""
    import oracle
    from paper_2103_05822_gb300.inputs import WORKLOADS, icosphere
    tfmm = _tfmm()
    w = WORKLOADS["sphere10"]
    v, f = icosphere(w.diameter, w.nu)
    P0 = oracle.problem.build(v, f, k=2 * math.pi, box=w.box, digits=w.digits, tol=w.tol,
                              compress=False, keep_tensors=False)
    sizes = np.array([len(m) for m in P0.groups.members])
    order = np.argsort(sizes, kind="stable")
    pick = sorted({int(order[i]) for i in np.linspace(0, len(order) - 1, 4).round().astype(int)})
    P = oracle.problem.build(v, f, k=2 * math.pi, box=w.box, digits=w.digits, tol=w.tol,
                             compress=True, keep_tensors=False, groups_subset=pick)
    # the picked groups' RWGs renumbered 0..n-1
    members, pos = [], 0
    for g in pick:
        members.append(np.arange(pos, pos + len(P.groups.members[g])))
        pos += len(P.groups.members[g])
    T = [P.tucker[g] for g in pick]
    factors = [[(t.U_theta, t.U_phi, t.U_beta, t.core) for t in per] for per in T]
    nt, npf = P.grid.n_theta, P.grid.n_phi
    R, G, nd = 128, len(pick), nt * npf
    plan = tfmm.tfmm_plan_from_tucker(pos, nt, npf, members, factors, weights=P.grid.weights, max_rhs=R,
                                      mrhs_precision=3)
    X = complex_gaussian((R, pos), 31)
    gin = complex_gaussian((R, G, 2, nd), 32)
    xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    spec = torch.full((R, G, 2, nd), float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, xd, spec)
    gd = torch.from_numpy(gin.astype(np.complex64)).cuda()
    yd = torch.full((R, pos), float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(plan, gd, yd)
    torch.cuda.synchronize()
    assert plan.info["kernel_errors"] == 0
    S, Y = spec.cpu().numpy(), yd.cpu().numpy()
    gamma = w.tol
    worst = [0.0, 0.0]
    for r in range(R):
        ref = apply.aggregate_all(T, members, X[r])
        refy = apply.disaggregate_all(T, members, gin[r], pos, P.grid.weights)
        for k in range(G):
            for a in range(2):
                e = max(_rel(S[r, k, a], ref[k, a]), _elem(S[r, k, a], ref[k, a]))
                worst[0] = max(worst[0], e)
                assert e <= gamma, (r, pick[k], a, e)
            ids = members[k]
            e = max(_rel(Y[r, ids], refy[ids]), _elem(Y[r, ids], refy[ids]))
            worst[1] = max(worst[1], e)
            assert e <= gamma, (r, pick[k], e)
    print(f"far-field factors, groups {pick}: worst aggregation {worst[0]:.2e}, disaggregation {worst[1]:.2e}")
