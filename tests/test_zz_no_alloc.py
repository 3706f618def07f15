"""tfmm_planewave_noalloc against tfmm_planewave, through the C ABI.

Some callers cannot allocate device memory while they call the library: their
device memory is all handed out by their own pool allocator, or they cannot
afford the device-wide synchronisation of a cudaFree.  The allocation-free
entry point stages the incidence table in a fixed array inside the library
instead.  This file is collected last so that a run stopping at the first
failure has run every other test; it also passes alone in a fresh process.

Two calls in a row with different incidences (and different counts) must
match the allocating entry point, so a table left over from the first call
would show in the second.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6  # FP32 output, same kernel on both paths


def _incidences(rng, R):
    theta = rng.uniform(0.0, math.pi, R)
    phi = rng.uniform(0.0, 2 * math.pi, R)
    k = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
    pol = np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], axis=1)
    return k, pol


def test_noalloc_planewave_matches_allocating_entry_point():
    from paper_2103_05822_gb300 import tfmm
    from paper_2103_05822_gb300.inputs import icosphere

    v, f = icosphere(1.0, 4)
    mesh = tfmm.tfmm_mesh_create(v, f)
    plan = tfmm.tfmm_plan_create(mesh, tfmm.tfmm_params_default(box=0.5, digits=3.0, tol=1e-4))
    n = plan.info["n_rwg"]
    rng = np.random.default_rng(2024)
    for R in (5, 3):
        k, pol = _incidences(rng, R)
        ref = torch.empty((R, n), dtype=torch.complex64, device="cuda")
        got = torch.full((R, n), float("nan"), dtype=torch.complex64, device="cuda")
        tfmm.tfmm_planewave(plan, k, pol, ref)
        tfmm.tfmm_planewave_noalloc(plan, k, pol, got)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref))
        assert err <= TOL, (R, err)


def test_noalloc_planewave_allocates_nothing_and_frees_caller_arrays_at_once():
    """Pinned caller arrays may be overwritten as soon as the call returns, and a
    call after the first (which looks up the table's device address) leaves the
    device's free memory unchanged."""
    from paper_2103_05822_gb300 import tfmm
    from paper_2103_05822_gb300.inputs import icosphere

    v, f = icosphere(1.0, 4)
    mesh = tfmm.tfmm_mesh_create(v, f)
    plan = tfmm.tfmm_plan_create(mesh, tfmm.tfmm_params_default(box=0.5, digits=3.0, tol=1e-4))
    n = plan.info["n_rwg"]
    rng = np.random.default_rng(7)
    R = 64
    k, pol = _incidences(rng, R)
    ref = torch.empty((R, n), dtype=torch.complex64, device="cuda")
    got = torch.full((R, n), float("nan"), dtype=torch.complex64, device="cuda")
    tfmm.tfmm_planewave(plan, k, pol, ref)
    tfmm.tfmm_planewave_noalloc(plan, k, pol, got)  # first call on this device: set-up
    torch.cuda.synchronize()
    kp = torch.empty((R, 3), dtype=torch.float64).pin_memory()
    pp = torch.empty((R, 3), dtype=torch.float64).pin_memory()
    kp.numpy()[:] = k
    pp.numpy()[:] = pol
    got.fill_(float("nan"))
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    tfmm.tfmm_planewave_noalloc(plan, kp.numpy(), pp.numpy(), got)
    kp.fill_(float("nan"))  # the caller reuses its pinned arrays at once
    pp.fill_(float("nan"))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    err = float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref))
    assert err <= TOL, err


def test_noalloc_planewave_rejects_more_incidences_than_the_table_holds():
    from paper_2103_05822_gb300 import tfmm
    from paper_2103_05822_gb300.inputs import icosphere

    v, f = icosphere(1.0, 2)
    mesh = tfmm.tfmm_mesh_create(v, f)
    plan = tfmm.tfmm_plan_create(mesh, tfmm.tfmm_params_default(box=0.5, digits=3.0, tol=1e-4))
    n = plan.info["n_rwg"]
    R = 1025
    k = np.tile([0.0, 0.0, 1.0], (R, 1))
    pol = np.tile([1.0, 0.0, 0.0], (R, 1))
    V = torch.empty((R, n), dtype=torch.complex64, device="cuda")
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_planewave_noalloc(plan, k, pol, V)
    assert e.value.status == tfmm.INVALID_ARG
    assert "1024" in str(e.value)
