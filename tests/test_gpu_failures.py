"""Error paths on the GPU without a GPU fault: injected allocation failures.

tfmm_test_fail_allocation(n) makes the library's n-th device allocation fail as if
the device were out of memory.  For a range of n the setup of a plan (with the
uncompressed tensors kept) and the first calls of the hot path (single RHS, the
tensor-core chain with its plan-owned scratch, the host-buffer matvec, the
translation stage) must return TFMM_OOM or succeed, never crash; after each
attempt the device's free memory must be back at its level before the attempt
(nothing leaked), and a plan made afterwards must give the same result as before.
"""
import math

import numpy as np
import pytest

from paper_2103_05822_gb300.inputs import complex_gaussian, icosphere

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(tfmm, mesh, x, R=2):
    prm = tfmm.tfmm_params_default(k=2 * math.pi, box=0.5, digits=3.0, tol=1e-4, keep_dense=1, max_rhs=R,
                                   mrhs_precision=3)
    plan = tfmm.tfmm_plan_create(mesh, prm)
    info = plan.info
    G, nd, n = info["n_groups"], info["n_dir"], info["n_rwg"]
    spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
    y = torch.empty((R, n), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_aggregate(plan, x[:1].reshape(-1), spec[:1])
    tfmm.tfmm_aggregate(plan, x, spec)
    tfmm.tfmm_disaggregate(plan, spec, y)
    gin = torch.empty_like(spec)
    tfmm.tfmm_translate(plan, spec, gin)
    yh = np.zeros(n, np.complex64)
    tfmm.tfmm_matvec_host(plan, x[0].cpu().numpy(), yh)
    torch.cuda.synchronize()
    out = (spec.cpu().numpy(), y.cpu().numpy(), gin.cpu().numpy(), yh)
    del plan, spec, y, gin
    return out


def test_injected_allocation_failures_return_oom_and_leak_nothing():
    from paper_2103_05822_gb300 import tfmm
    v, f = icosphere(1.0, 6)
    mesh = tfmm.tfmm_mesh_create(v, f)
    n = tfmm.tfmm_mesh_num_rwg(mesh)
    x = torch.from_numpy(complex_gaussian((2, n), 3).astype(np.complex64)).cuda()
    ref = _run(tfmm, mesh, x)  # loads every kernel once; its allocations are freed with the plan
    torch.cuda.synchronize()
    failures = 0
    for nth in (1, 2, 3, 4, 6, 9, 13, 19, 28, 41, 60, 90, 130):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # torch's own cached blocks are not the library's
        free0 = torch.cuda.mem_get_info()[0]
        tfmm.tfmm_test_fail_allocation(nth)
        try:
            _run(tfmm, mesh, x)
        except tfmm.TfmmError as e:
            assert e.status == tfmm.OOM, (nth, e)
            failures += 1
        finally:
            tfmm.tfmm_test_fail_allocation(0)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        assert torch.cuda.mem_get_info()[0] == free0, nth
    assert failures >= 8
    got = _run(tfmm, mesh, x)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
