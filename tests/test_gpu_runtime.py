"""Runtime services around the hot path, through the C ABI on the GPU.

* RWG -> (group, slot) table against the member lists;
* checkpoints: a saved and reloaded plan reproduces the original bit for bit
  (same FP64 factors, same FP32 packing, same kernels), and damaged files are
  refused with TFMM_IO;
* CUDA graphs: replays equal the eager calls and follow new input contents;
* tuning: every launch shape and queue order gives the oracle's result; the
  autotuner's choice does too;
* tfmm_sync reports a healthy plan.
"""
import math

import numpy as np
import pytest

from oracle import apply, hosvd
from paper_2103_05822_gb300.inputs import WORKLOADS, complex_gaussian, synthetic_tucker

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W2 = WORKLOADS["sphere2"]


def _tfmm():
    from paper_2103_05822_gb300 import tfmm
    return tfmm


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def synth():
    """A ragged synthetic plan (paper-like grid, uneven ranks) and its oracle factors."""
    tfmm = _tfmm()
    nt, npf, nbetas = 40, 80, [940, 37, 411, 1786, 5]
    rng = np.random.default_rng(21)
    ranks = [[(int(rng.integers(1, 31)), int(rng.integers(1, 36)), int(rng.integers(1, nb + 1))) for _ in range(2)]
             for nb in nbetas]
    syn = synthetic_tucker(nt, npf, nbetas, ranks, 21)
    n_rwg = sum(nbetas)
    perm = rng.permutation(n_rwg)
    members, pos = [], 0
    for nb in nbetas:
        members.append(np.sort(perm[pos:pos + nb]))
        pos += nb
    T = [[hosvd.Tucker(s.U_theta, s.U_phi, s.U_beta, s.core) for s in per] for per in syn]
    factors = [[(t.U_theta, t.U_phi, t.U_beta, t.core) for t in per] for per in T]
    w = np.random.default_rng(22).uniform(0.05, 1.0, nt * npf)
    plan = tfmm.tfmm_plan_from_tucker(n_rwg, nt, npf, members, factors, weights=w, max_rhs=4)
    return dict(plan=plan, T=T, members=members, n_rwg=n_rwg, nt=nt, npf=npf, w=w, factors=factors)


@pytest.fixture(scope="module")
def sphere2_plan(sphere2_mesh):
    tfmm = _tfmm()
    v, f = sphere2_mesh
    mesh = tfmm.tfmm_mesh_create(v, f)
    prm = tfmm.tfmm_params_default(k=2 * math.pi, box=W2.box, digits=float(W2.digits), tol=W2.tol, max_rhs=2)
    return tfmm.tfmm_plan_create(mesh, prm)


def _agg_dis(plan, x, g, R=1):
    tfmm = _tfmm()
    info = plan.info
    shape = (R, info["n_groups"], 2, info["n_dir"])
    spec = torch.full(shape, float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, x, spec)
    y = torch.zeros_like(x)
    tfmm.tfmm_disaggregate(plan, g, y)
    torch.cuda.synchronize()
    return spec.cpu().numpy(), y.cpu().numpy()


def test_rwg_perm_matches_members(sphere2_plan):
    tfmm = _tfmm()
    grp, slot = tfmm.tfmm_plan_rwg_perm(sphere2_plan)
    members = tfmm.tfmm_plan_members(sphere2_plan)
    n = sphere2_plan.info["n_rwg"]
    assert grp.shape == (n,) and slot.shape == (n,)
    for g, m in enumerate(members):
        assert np.all(grp[m] == g)
        assert np.array_equal(slot[m], np.arange(len(m)))


def test_checkpoint_roundtrip_is_bit_exact(sphere2_plan, tmp_path):
    tfmm = _tfmm()
    path = str(tmp_path / "sphere2.tfmm")
    tfmm.tfmm_plan_save(sphere2_plan, path)
    loaded = tfmm.tfmm_plan_load(path)
    a, b = sphere2_plan.info, loaded.info
    for k in ("L", "n_theta", "n_phi", "n_groups", "K", "n_rwg", "max_rank", "tucker_bytes", "setup_ms"):
        assert a[k] == b[k], k
    for q1, q2 in zip(tfmm.tfmm_plan_quadrature(sphere2_plan), tfmm.tfmm_plan_quadrature(loaded)):
        assert np.array_equal(np.asarray(q1), np.asarray(q2))
    assert np.array_equal(tfmm.tfmm_plan_centres(sphere2_plan), tfmm.tfmm_plan_centres(loaded))
    for g in (0, a["n_groups"] - 1):
        for al in range(2):
            for u, v in zip(tfmm.tfmm_plan_export_factors(sphere2_plan, g, al),
                            tfmm.tfmm_plan_export_factors(loaded, g, al)):
                assert np.array_equal(u, v)
    n, G, nd = a["n_rwg"], a["n_groups"], a["n_dir"]
    x = torch.from_numpy(complex_gaussian(n, 31).astype(np.complex64)).cuda()
    g = torch.from_numpy(complex_gaussian((1, G, 2, nd), 32).astype(np.complex64)).cuda()
    s1, y1 = _agg_dis(sphere2_plan, x, g)
    s2, y2 = _agg_dis(loaded, x, g)
    assert np.array_equal(s1, s2) and np.array_equal(y1, y2)
    # the geometry came along: plane-wave excitation and far-fields agree too
    kh, pol = np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])
    V1 = torch.empty((1, n), dtype=torch.complex64, device="cuda")
    V2 = torch.empty_like(V1)
    tfmm.tfmm_planewave(sphere2_plan, kh, pol, V1)
    tfmm.tfmm_planewave(loaded, kh, pol, V2)
    torch.cuda.synchronize()
    assert torch.equal(V1, V2)
    At1, _ = tfmm.tfmm_plan_farfield(sphere2_plan, 3)
    At2, _ = tfmm.tfmm_plan_farfield(loaded, 3)
    assert np.array_equal(At1, At2)


def test_checkpoint_of_a_factor_plan(synth, tmp_path):
    tfmm = _tfmm()
    path = str(tmp_path / "synth.tfmm")
    tfmm.tfmm_plan_save(synth["plan"], path)
    loaded = tfmm.tfmm_plan_load(path)
    with pytest.raises(tfmm.TfmmError):
        tfmm.tfmm_plan_quadrature(loaded)  # a plan made from factors has no grid, before and after
    x = torch.from_numpy(complex_gaussian(synth["n_rwg"], 41).astype(np.complex64)).cuda()
    g = torch.from_numpy(complex_gaussian((1, len(synth["members"]), 2, synth["nt"] * synth["npf"]), 42)
                         .astype(np.complex64)).cuda()
    s1, y1 = _agg_dis(synth["plan"], x, g)
    s2, y2 = _agg_dis(loaded, x, g)
    assert np.array_equal(s1, s2) and np.array_equal(y1, y2)


def test_damaged_checkpoints_are_refused(synth, tmp_path):
    tfmm = _tfmm()
    path = tmp_path / "ok.tfmm"
    tfmm.tfmm_plan_save(synth["plan"], str(path))
    data = bytearray(path.read_bytes())
    cases = {
        "truncated": bytes(data[:len(data) // 2]),
        "trailing": bytes(data) + b"x",
        "bad_trailer": bytes(data[:-1]) + b"?",
        "bad_version": bytes(data[:8]) + (7).to_bytes(4, "little") + bytes(data[12:]),
    }
    for name, blob in cases.items():
        p = tmp_path / f"{name}.tfmm"
        p.write_bytes(blob)
        with pytest.raises(tfmm.TfmmError) as e:
            tfmm.tfmm_plan_load(str(p))
        assert e.value.status == tfmm.IO, name


def test_graph_replays_equal_eager_calls(synth):
    tfmm = _tfmm()
    plan = synth["plan"]
    G, nd, n = len(synth["members"]), synth["nt"] * synth["npf"], synth["n_rwg"]
    for R in (1, 3):
        xs = [complex_gaussian((R, n), 50 + R), complex_gaussian((R, n), 60 + R)]
        x = torch.from_numpy(xs[0].astype(np.complex64)).cuda()
        spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
        y = torch.zeros((R, n), dtype=torch.complex64, device="cuda")
        graph = tfmm.tfmm_graph_capture(plan, 3, spec, x=x, y=y, R=R, beta=0.0)
        for xv in xs:
            x.copy_(torch.from_numpy(xv.astype(np.complex64)))
            y.fill_(float("nan"))
            graph.launch()
            torch.cuda.synchronize()
            ref_s = torch.empty_like(spec)
            tfmm.tfmm_aggregate(plan, x, ref_s)
            ref_y = torch.zeros_like(y)
            tfmm.tfmm_disaggregate(plan, spec, ref_y)
            torch.cuda.synchronize()
            assert torch.equal(spec, ref_s) and torch.equal(y, ref_y)
            ref = [apply.aggregate_all(synth["T"], synth["members"], xv[r]) for r in range(R)]
            assert max(_rel(spec.cpu().numpy()[r], ref[r]) for r in range(R)) <= 1e-5
        with pytest.raises(tfmm.TfmmError):
            tfmm._check(tfmm.load().tfmm_plan_destroy(plan.handle))  # refused while a graph exists
        tfmm.tfmm_graph_destroy(graph)
    tfmm.tfmm_sync(plan)


@pytest.mark.parametrize("threads,ctas,order", [(512, 0, 0), (256, 1, 1), (384, 2, 0), (64, 0, 1)])
def test_every_launch_shape_matches_oracle(synth, threads, ctas, order):
    tfmm = _tfmm()
    plan = synth["plan"]
    # the persistent kernels (this few-group plan takes the split path by default)
    tfmm.tfmm_plan_tuning_set(plan, agg_threads=threads, agg_ctas_per_sm=ctas, agg_order=order,
                              dis_threads=threads, dis_ctas_per_sm=ctas, dis_order=order, single_rhs_split=2)
    t = tfmm.tfmm_plan_tuning_get(plan)
    assert (t["agg_threads"], t["agg_order"], t["dis_threads"], t["dis_order"]) == (threads, order, threads, order)
    assert t["agg_blocks"] >= 1 and t["dis_blocks"] >= 1
    G, nd, n = len(synth["members"]), synth["nt"] * synth["npf"], synth["n_rwg"]
    xv = complex_gaussian(n, 70)
    gv = complex_gaussian((1, G, 2, nd), 71)
    s, y = _agg_dis(plan, torch.from_numpy(xv.astype(np.complex64)).cuda(),
                    torch.from_numpy(gv.astype(np.complex64)).cuda())
    ref = apply.aggregate_all(synth["T"], synth["members"], xv)
    for g in range(G):
        for a in range(2):
            assert _rel(s[0, g, a], ref[g, a]) <= 1e-5
    refy = apply.disaggregate_all(synth["T"], synth["members"], gv[0], n, synth["w"])
    assert _rel(y, refy) <= 1e-5


def test_split_path_matches_persistent_kernels_and_oracle(synth):
    """Few groups: each stage as three launches spreading every item over many CTAs
    (row blocks of U_beta / C_(3), column blocks, one CTA per item for the theta / phi
    steps).  Same results as the persistent kernels (FP32 rounding) and the oracle."""
    tfmm = _tfmm()
    plan = synth["plan"]
    G, nd, n = len(synth["members"]), synth["nt"] * synth["npf"], synth["n_rwg"]
    xv = torch.from_numpy(complex_gaussian(n, 72).astype(np.complex64)).cuda()
    gv = torch.from_numpy(complex_gaussian((1, G, 2, nd), 73).astype(np.complex64)).cuda()
    out = {}
    for split in (1, 2):
        tfmm.tfmm_plan_tuning_set(plan, single_rhs_split=split)
        assert tfmm.tfmm_plan_tuning_get(plan)["single_rhs_split"] == split
        out[split] = _agg_dis(plan, xv, gv)
    tfmm.tfmm_plan_tuning_set(plan, single_rhs_split=0)
    ref = apply.aggregate_all(synth["T"], synth["members"], xv.cpu().numpy().astype(np.complex128))
    refy = apply.disaggregate_all(synth["T"], synth["members"], gv.cpu().numpy()[0].astype(np.complex128), n, synth["w"])
    for split in (1, 2):
        s_, y_ = out[split]
        for g in range(G):
            for a in range(2):
                assert _rel(s_[0, g, a], ref[g, a]) <= 1e-5, (split, g, a)
        assert _rel(y_, refy) <= 1e-5, split
    assert _rel(out[1][0], out[2][0]) <= 1e-5 and _rel(out[1][1], out[2][1]) <= 1e-5
    with pytest.raises(tfmm.TfmmError):
        tfmm.tfmm_plan_tuning_set(plan, single_rhs_split=3)


def test_tuning_rejects_bad_shapes(synth):
    tfmm = _tfmm()
    for bad in ({"agg_threads": 1024}, {"dis_threads": 100}, {"agg_order": 2}, {"dis_ctas_per_sm": -1},
                {"mrhs_precision": 4}, {"mrhs_precision": -1}):
        with pytest.raises(tfmm.TfmmError) as e:
            tfmm.tfmm_plan_tuning_set(synth["plan"], **bad)
        assert e.value.status == tfmm.INVALID_ARG


@pytest.mark.parametrize("R", [1, 4])
def test_autotuner_choice_matches_oracle(synth, R):
    tfmm = _tfmm()
    plan = synth["plan"]
    t = tfmm.tfmm_autotune(plan, R=R, budget_ms=3000.0)
    assert t["agg_ms"] > 0 and t["dis_ms"] > 0
    if R > 1:
        assert t["mrhs_precision"] in (0, 1, 3)
    G, nd, n = len(synth["members"]), synth["nt"] * synth["npf"], synth["n_rwg"]
    X = complex_gaussian((R, n), 80)
    x = torch.from_numpy(X.astype(np.complex64)).cuda()
    spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, x if R > 1 else x[0], spec)
    tfmm.tfmm_sync(plan)
    for r in range(R):
        ref = apply.aggregate_all(synth["T"], synth["members"], X[r])
        assert _rel(spec.cpu().numpy()[r], ref) <= 1e-5


def test_column_engine_matches_oracle(synth):
    """mrhs_precision 1: the single-RHS kernels, one column after another."""
    tfmm = _tfmm()
    plan = synth["plan"]
    tfmm.tfmm_plan_set_mrhs_precision(plan, 1)
    R, G, nd, n = 3, len(synth["members"]), synth["nt"] * synth["npf"], synth["n_rwg"]
    X = complex_gaussian((R, n), 90)
    gv = complex_gaussian((R, G, 2, nd), 91)
    spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, torch.from_numpy(X.astype(np.complex64)).cuda(), spec)
    y = torch.zeros((R, n), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(plan, torch.from_numpy(gv.astype(np.complex64)).cuda(), y)
    tfmm.tfmm_sync(plan)
    for r in range(R):
        assert _rel(spec.cpu().numpy()[r], apply.aggregate_all(synth["T"], synth["members"], X[r])) <= 1e-5
        refy = apply.disaggregate_all(synth["T"], synth["members"], gv[r], n, synth["w"])
        assert _rel(y.cpu().numpy()[r], refy) <= 1e-5
    tfmm.tfmm_plan_set_mrhs_precision(plan, 0)


def test_items_too_large_for_one_cta_fall_back_to_the_chain():
    """A group with 30,000 RWGs does not fit the single-RHS kernels' shared memory:
    every call (R = 1 included) then runs the grouped-GEMM chain, same results."""
    tfmm = _tfmm()
    nt, npf, nbetas = 6, 12, [30000, 40]
    ranks = [[(3, 4, 5), (2, 3, 4)], [(4, 5, 6), (3, 3, 7)]]
    syn = synthetic_tucker(nt, npf, nbetas, ranks, 33)
    n_rwg = sum(nbetas)
    perm = np.random.default_rng(34).permutation(n_rwg)
    members = [np.sort(perm[:nbetas[0]]), np.sort(perm[nbetas[0]:])]
    T = [[hosvd.Tucker(s.U_theta, s.U_phi, s.U_beta, s.core) for s in per] for per in syn]
    factors = [[(t.U_theta, t.U_phi, t.U_beta, t.core) for t in per] for per in T]
    w = np.random.default_rng(35).uniform(0.05, 1.0, nt * npf)
    plan = tfmm.tfmm_plan_from_tucker(n_rwg, nt, npf, members, factors, weights=w, max_rhs=2)
    t = tfmm.tfmm_plan_tuning_get(plan)
    assert t["agg_blocks"] == 0 or t["dis_blocks"] == 0
    for R in (1, 2):
        X = complex_gaussian((R, n_rwg), 36 + R)
        gv = complex_gaussian((R, 2, 2, nt * npf), 38 + R)
        spec = torch.empty((R, 2, 2, nt * npf), dtype=torch.complex64, device="cuda")
        xd = torch.from_numpy(X.astype(np.complex64)).cuda()
        tfmm.tfmm_aggregate(plan, xd if R > 1 else xd[0], spec)
        y = torch.zeros((R, n_rwg), dtype=torch.complex64, device="cuda")
        tfmm.tfmm_disaggregate(plan, torch.from_numpy(gv.astype(np.complex64)).cuda(), y if R > 1 else y[0])
        tfmm.tfmm_sync(plan)
        for r in range(R):
            assert _rel(spec.cpu().numpy()[r], apply.aggregate_all(T, members, X[r])) <= 1e-5
            assert _rel(y.cpu().numpy()[r], apply.disaggregate_all(T, members, gv[r], n_rwg, w)) <= 1e-5


@pytest.mark.parametrize("n1,pairs", [(32, 64), (0, 128), (128, 0), (16, 0)])
def test_tensor_core_tile_shapes_match_oracle(synth, n1, pairs):
    """The fused AG3+AG4 block size and the DG1a pair count only change the tiling."""
    tfmm = _tfmm()
    plan = synth["plan"]
    tfmm.tfmm_plan_tuning_set(plan, mrhs_precision=3, tc_f34_n1=n1, tc_dg1a_pairs=pairs)
    t = tfmm.tfmm_plan_tuning_get(plan)
    assert (t["tc_f34_n1"], t["tc_dg1a_pairs"], t["mrhs_precision"]) == (n1, pairs, 3)
    R, G, nd, n = 4, len(synth["members"]), synth["nt"] * synth["npf"], synth["n_rwg"]
    X = complex_gaussian((R, n), 100 + n1 + pairs)
    gv = complex_gaussian((R, G, 2, nd), 101 + n1 + pairs)
    spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, torch.from_numpy(X.astype(np.complex64)).cuda(), spec)
    y = torch.zeros((R, n), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_disaggregate(plan, torch.from_numpy(gv.astype(np.complex64)).cuda(), y)
    tfmm.tfmm_sync(plan)
    for r in range(R):
        assert _rel(spec.cpu().numpy()[r], apply.aggregate_all(synth["T"], synth["members"], X[r])) <= 1e-5
        refy = apply.disaggregate_all(synth["T"], synth["members"], gv[r], n, synth["w"])
        assert _rel(y.cpu().numpy()[r], refy) <= 1e-5
    tfmm.tfmm_plan_tuning_set(plan, mrhs_precision=0, tc_f34_n1=0, tc_dg1a_pairs=0)


def test_tensor_core_tile_shapes_are_validated(synth):
    tfmm = _tfmm()
    for bad in ({"tc_f34_n1": 20}, {"tc_f34_n1": 272}, {"tc_dg1a_pairs": 100}):
        with pytest.raises(tfmm.TfmmError) as e:
            tfmm.tfmm_plan_tuning_set(synth["plan"], **bad)
        assert e.value.status == tfmm.INVALID_ARG
