"""C-ABI library: loads, exports what include/tfmm.h declares, host-side logic (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2103_05822_gb300 import tfmm
from paper_2103_05822_gb300.inputs import icosphere

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tfmm.library_path()):
        from paper_2103_05822_gb300 import build
        build.build()
    return tfmm.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tfmm_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert declared == set(tfmm.EXPORTED)


def test_params_default(lib):
    p = tfmm.tfmm_params_default()
    assert abs(p.k - 2 * np.pi) < 1e-15 and p.quad_order == 5 and p.max_rhs == 1 and p.nphi_rule == 1


@pytest.mark.parametrize("nu", [1, 4, 12])
def test_rwg_table_matches_oracle_bit_exact(lib, nu):
    v, f = icosphere(2.0, nu)
    mesh = tfmm.tfmm_mesh_create(v, f)
    edge, tri, free = tfmm.tfmm_mesh_rwg(mesh)
    r = oracle.rwg.build_rwg(v, f)
    assert np.array_equal(edge, r.edge)
    assert np.array_equal(tri, r.tri)
    assert np.array_equal(free, r.free)


def test_open_and_nonmanifold_meshes(lib):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0.5, 0.5, 1.0]], float)
    # edge (1, 2) shared by three triangles: not an RWG; (0,1,2)-(1,3,2) pair would be
    f = np.array([[0, 1, 2], [1, 3, 2], [1, 2, 4]])
    mesh = tfmm.tfmm_mesh_create(v, f)
    assert tfmm.tfmm_mesh_num_rwg(mesh) == len(oracle.rwg.build_rwg(v, f).length) == 0
    mesh2 = tfmm.tfmm_mesh_create(v, f[:2])
    assert tfmm.tfmm_mesh_num_rwg(mesh2) == 1


@pytest.mark.parametrize("case", ["oob", "repeat", "degenerate", "nan"])
def test_mesh_create_rejects_bad_input(lib, case):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [2, 0, 0]], float)
    f = np.array([[0, 1, 2]])
    if case == "oob":
        f = np.array([[0, 1, 7]])
    elif case == "repeat":
        f = np.array([[0, 1, 1]])
    elif case == "degenerate":
        f = np.array([[0, 1, 3]])  # collinear
    elif case == "nan":
        v[2, 1] = np.nan
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_mesh_create(v, f)
    assert e.value.status == tfmm.INVALID_ARG
    assert len(lib.tfmm_last_error()) > 0


def test_null_pointers_are_rejected(lib):
    out = ctypes.c_void_p()
    assert lib.tfmm_mesh_create(None, 3, None, 1, ctypes.byref(out)) == tfmm.INVALID_ARG
    assert lib.tfmm_mesh_num_rwg(None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_plan_info_get(None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_aggregate(None, None, 1, 1, None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_params_default(None) == tfmm.INVALID_ARG
    assert lib.tfmm_mesh_destroy(None) == tfmm.OK
    assert lib.tfmm_plan_destroy(None) == tfmm.OK


def test_plan_params_validated_before_any_gpu_work(lib):
    v, f = icosphere(1.0, 2)
    mesh = tfmm.tfmm_mesh_create(v, f)
    for bad in ({"k": -1.0}, {"box": 0.0}, {"digits": 0.0}, {"tol": -1e-3}, {"quad_order": 11},
                {"nphi_rule": 3}, {"max_rhs": 0}):
        p = tfmm.tfmm_params_default(**bad)
        with pytest.raises(tfmm.TfmmError) as e:
            tfmm.tfmm_plan_create(mesh, p, stream=0)
        assert e.value.status == tfmm.INVALID_ARG


def test_runtime_calls_reject_null_arguments(lib):
    out = ctypes.c_void_p()
    z = tfmm.cfloat(0.0, 0.0)
    assert lib.tfmm_sync(None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_plan_rwg_perm(None, None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_plan_save(None, b"/nonexistent/x") == tfmm.INVALID_ARG
    assert lib.tfmm_plan_load(None, None, ctypes.byref(out)) == tfmm.INVALID_ARG
    assert lib.tfmm_graph_capture(None, 1, None, 1, 1, None, 1, z, None, 1, ctypes.byref(out)) == tfmm.INVALID_ARG
    assert lib.tfmm_graph_launch(None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_graph_destroy(None) == tfmm.OK
    assert lib.tfmm_plan_tuning_get(None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_plan_tuning_set(None, None, None) == tfmm.INVALID_ARG
    assert lib.tfmm_autotune(None, 1, 10.0, 0, None, None) == tfmm.INVALID_ARG


def test_checkpoint_load_rejects_missing_and_foreign_files(lib, tmp_path):
    """Header checks run before any device work, so they are testable here."""
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_plan_load(str(tmp_path / "missing.tfmm"), stream=0)
    assert e.value.status == tfmm.IO
    junk = tmp_path / "junk.tfmm"
    junk.write_bytes(b"NOTAPLAN" + bytes(64))
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_plan_load(str(junk), stream=0)
    assert e.value.status == tfmm.IO
    short = tmp_path / "short.tfmm"
    short.write_bytes(b"TFMMPLAN\x01\x00")
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_plan_load(str(short), stream=0)
    assert e.value.status == tfmm.IO and "truncated" in str(e.value)


def test_binding_structs_match_the_header(tmp_path):
    """ctypes mirrors of tfmm_params / tfmm_plan_info / tfmm_tuning have the C layout."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tfmm.h"\n'
        'int main(void) {\n'
        '  printf("%zu %zu %zu\\n", sizeof(tfmm_params), sizeof(tfmm_plan_info), sizeof(tfmm_tuning));\n'
        '  printf("%zu %zu %zu %zu\\n", offsetof(tfmm_params, mrhs_precision), offsetof(tfmm_params, compression),\n'
        '         offsetof(tfmm_plan_info, kernel_errors), offsetof(tfmm_tuning, agg_ms));\n'
        '  return 0;\n}\n')
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = [int(v) for v in out]
    want = [ctypes.sizeof(tfmm.Params), ctypes.sizeof(tfmm.PlanInfo), ctypes.sizeof(tfmm.Tuning),
            tfmm.Params.mrhs_precision.offset, tfmm.Params.compression.offset, tfmm.PlanInfo.kernel_errors.offset,
            tfmm.Tuning.agg_ms.offset]
    assert got == want


def test_checkpoint_header_announcing_huge_arrays_is_refused(lib, tmp_path):
    """A corrupt header cannot make the loader allocate: sizes are checked against the file."""
    import struct
    p = tfmm.tfmm_params_default()
    head = b"TFMMPLAN" + struct.pack("<III", 1, 0, ctypes.sizeof(tfmm.Params)) + bytes(p)
    dims = struct.pack("<7i", 10, 11, 22, 1 << 20, 1, 1, 1) + struct.pack("<q", (1 << 31) - 1)
    f = tmp_path / "huge.tfmm"
    f.write_bytes(head + dims + bytes(64))
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_plan_load(str(f), stream=0)
    assert e.value.status == tfmm.IO and "shorter" in str(e.value)


def test_well_formed_checkpoint_passes_the_header_checks(lib, tmp_path):
    """A complete file of the documented layout gets past every file check; on a machine
    without a GPU the load then stops at the first device call (status CUDA, not IO)."""
    import struct
    import numpy as np
    nt, npf, G, N = 2, 3, 1, 2
    p = tfmm.tfmm_params_default()
    blob = b"TFMMPLAN" + struct.pack("<III", 1, 2, ctypes.sizeof(tfmm.Params)) + bytes(p)
    blob += struct.pack("<7i", nt - 1, nt, npf, G, 1, 1, 1) + struct.pack("<q", N)
    blob += struct.pack("<6d", 2 * np.pi, 2 * np.pi / npf, 0, 0, 0, 0)
    blob += np.linspace(0.5, 2.5, nt).tobytes() + np.full(nt, 1.0).tobytes() + np.arange(npf, dtype=np.float64).tobytes()
    blob += np.full(nt * npf, 0.5, np.float32).tobytes()
    blob += np.array([0, N], np.int64).tobytes() + np.array([1, 0], np.int64).tobytes()
    blob += np.zeros(3 * G).tobytes() + np.ones(6 * G, np.int32).tobytes()
    per_alpha = nt + npf + N + 1
    blob += np.ones(2 * per_alpha, np.complex128).tobytes() + b"TFMMEND."
    f = tmp_path / "tiny.tfmm"
    f.write_bytes(blob)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if has_gpu:
        plan = tfmm.tfmm_plan_load(str(f), stream=0)
        assert plan.info["n_rwg"] == N
    else:
        with pytest.raises(tfmm.TfmmError) as e:
            tfmm.tfmm_plan_load(str(f), stream=0)
        assert e.value.status == tfmm.CUDA, str(e.value)


def test_allocation_failure_hook_arguments(lib):
    """The error-path test hook accepts nth >= 0 (0 disarms) and refuses negative counts."""
    tfmm.tfmm_test_fail_allocation(0)
    with pytest.raises(tfmm.TfmmError) as e:
        tfmm.tfmm_test_fail_allocation(-1)
    assert e.value.status == tfmm.INVALID_ARG
