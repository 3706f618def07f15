"""Thin Python binding of ``libtfmm.so`` (the C ABI declared in ``include/tfmm.h``).

Argument marshalling only: every function here forwards to the C entry point of
the same name; all computation runs in the library's CUDA kernels.  Device
buffers are torch CUDA tensors (complex64 on the hot path); the CUDA stream
defaults to torch's current stream.  There is no CPU fallback: importing
works anywhere, but every call raises if the library was not built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtfmm.so")
_lib = None

OK, INVALID_ARG, OOM, CUDA, NUMERIC, NOT_BUILT, IO = range(7)
TUCKER, SVD = 0, 1  # tfmm_params.compression

EXPORTED = [
    "tfmm_params_default", "tfmm_last_error",
    "tfmm_mesh_create", "tfmm_mesh_num_rwg", "tfmm_mesh_rwg", "tfmm_mesh_destroy",
    "tfmm_plan_create", "tfmm_plan_from_tucker", "tfmm_plan_set_dense", "tfmm_plan_info_get",
    "tfmm_plan_group", "tfmm_plan_members", "tfmm_plan_centres", "tfmm_plan_quadrature",
    "tfmm_plan_export_factors", "tfmm_plan_farfield", "tfmm_plan_destroy",
    "tfmm_aggregate", "tfmm_disaggregate", "tfmm_aggregate_dense", "tfmm_disaggregate_dense",
    "tfmm_matvec_host", "tfmm_planewave", "tfmm_planewave_noalloc", "tfmm_plan_set_mrhs_precision", "tfmm_translate",
    "tfmm_sync", "tfmm_plan_rwg_perm", "tfmm_plan_save", "tfmm_plan_load",
    "tfmm_graph_capture", "tfmm_graph_launch", "tfmm_graph_destroy",
    "tfmm_plan_tuning_get", "tfmm_plan_tuning_set", "tfmm_autotune", "tfmm_test_fail_allocation",
]


class TfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tfmm status {status}: {msg}")
        self.status = status


class cfloat(ctypes.Structure):
    _fields_ = [("re", ctypes.c_float), ("im", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_double), ("box", ctypes.c_double), ("digits", ctypes.c_double),
        ("nphi_rule", ctypes.c_int32), ("L_override", ctypes.c_int32), ("tol", ctypes.c_double),
        ("quad_order", ctypes.c_int32), ("keep_dense", ctypes.c_int32), ("max_rhs", ctypes.c_int32),
        ("batch_groups", ctypes.c_int32), ("mrhs_precision", ctypes.c_int32), ("compression", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 4),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("n_phi", ctypes.c_int32), ("n_dir", ctypes.c_int32),
        ("n_groups", ctypes.c_int32), ("K", ctypes.c_int32 * 3), ("n_rwg", ctypes.c_int64),
        ("max_n_beta", ctypes.c_int32), ("max_rank", ctypes.c_int32 * 3),
        ("tucker_bytes", ctypes.c_int64), ("tucker_bytes_alg", ctypes.c_int64), ("dense_bytes", ctypes.c_int64),
        ("setup_ms", ctypes.c_double * 4), ("kernel_errors", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]

    def as_dict(self):
        return {
            "L": self.L, "n_theta": self.n_theta, "n_phi": self.n_phi, "n_dir": self.n_dir,
            "n_groups": self.n_groups, "K": list(self.K), "n_rwg": self.n_rwg, "max_n_beta": self.max_n_beta,
            "max_rank": list(self.max_rank), "tucker_bytes": self.tucker_bytes,
            "tucker_bytes_alg": self.tucker_bytes_alg, "dense_bytes": self.dense_bytes,
            "setup_ms": list(self.setup_ms), "kernel_errors": self.kernel_errors,
        }


class Tuning(ctypes.Structure):
    _fields_ = [
        ("agg_threads", ctypes.c_int32), ("agg_ctas_per_sm", ctypes.c_int32), ("agg_order", ctypes.c_int32),
        ("dis_threads", ctypes.c_int32), ("dis_ctas_per_sm", ctypes.c_int32), ("dis_order", ctypes.c_int32),
        ("agg_blocks", ctypes.c_int32), ("dis_blocks", ctypes.c_int32), ("mrhs_precision", ctypes.c_int32),
        ("tc_f34_n1", ctypes.c_int32), ("tc_dg1a_pairs", ctypes.c_int32), ("single_rhs_split", ctypes.c_int32),
        ("agg_ms", ctypes.c_double), ("dis_ms", ctypes.c_double),
    ]
    _names = ("agg_threads", "agg_ctas_per_sm", "agg_order", "dis_threads", "dis_ctas_per_sm", "dis_order",
              "agg_blocks", "dis_blocks", "mrhs_precision", "tc_f34_n1", "tc_dg1a_pairs", "single_rhs_split",
              "agg_ms", "dis_ms")

    def as_dict(self):
        return {k: getattr(self, k) for k in self._names}


def library_path():
    return _LIB_PATH


def load():
    """Loads the library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(_LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "tfmm_params_default": [P],
        "tfmm_mesh_create": [P, I64, P, I64, P],
        "tfmm_mesh_num_rwg": [P, P],
        "tfmm_mesh_rwg": [P, P, P, P],
        "tfmm_mesh_destroy": [P],
        "tfmm_plan_create": [P, P, P, P],
        "tfmm_plan_from_tucker": [I64, I32, I32, I32, P, P, P, P, P, I32, P, P],
        "tfmm_plan_set_dense": [P, P, P],
        "tfmm_plan_info_get": [P, P],
        "tfmm_plan_group": [P, I32, I32, P, P],
        "tfmm_plan_members": [P, P, P],
        "tfmm_plan_centres": [P, P],
        "tfmm_plan_quadrature": [P, P, P, P, P],
        "tfmm_plan_export_factors": [P, I32, I32, P, P, P, P],
        "tfmm_plan_farfield": [P, I32, P, P, P],
        "tfmm_plan_destroy": [P],
        "tfmm_aggregate": [P, P, I32, I64, P, P],
        "tfmm_disaggregate": [P, P, I32, I32, cfloat, P, I64, P],
        "tfmm_aggregate_dense": [P, P, I32, I64, P, P],
        "tfmm_disaggregate_dense": [P, P, I32, I32, cfloat, P, I64, P],
        "tfmm_matvec_host": [P, P, P, I32, I32, P],
        "tfmm_planewave": [P, P, P, I32, P, P],
        "tfmm_planewave_noalloc": [P, P, P, I32, P, P],
        "tfmm_translate": [P, P, I32, P, P],
        "tfmm_plan_set_mrhs_precision": [P, I32],
        "tfmm_sync": [P, P],
        "tfmm_plan_rwg_perm": [P, P, P],
        "tfmm_plan_save": [P, ctypes.c_char_p],
        "tfmm_plan_load": [ctypes.c_char_p, P, P],
        "tfmm_graph_capture": [P, I32, P, I32, I64, P, I32, cfloat, P, I64, P],
        "tfmm_graph_launch": [P, P],
        "tfmm_graph_destroy": [P],
        "tfmm_plan_tuning_get": [P, P],
        "tfmm_plan_tuning_set": [P, P, P],
        "tfmm_autotune": [P, I32, D, I32, P, P],
        "tfmm_test_fail_allocation": [I64],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.tfmm_last_error.argtypes = []
    L.tfmm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status):
    if status != OK:
        msg = load().tfmm_last_error().decode(errors="replace")
        raise TfmmError(status, msg)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev_ptr(t, dtype_name="complex64"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype).split(".")[-1] != dtype_name:
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------- mesh
def tfmm_params_default(**overrides):
    p = Params()
    _check(load().tfmm_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Mesh:
    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tfmm_mesh_destroy(self.handle)
            self.handle = None


def tfmm_mesh_create(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    if v.ndim != 2 or v.shape[1] != 3 or t.ndim != 2 or t.shape[1] != 3:
        raise ValueError("verts must be (nv, 3) and tris (nt, 3)")
    h = ctypes.c_void_p()
    _check(load().tfmm_mesh_create(_np_ptr(v), v.shape[0], _np_ptr(t), t.shape[0], ctypes.byref(h)))
    return Mesh(h)


def tfmm_mesh_num_rwg(mesh):
    n = ctypes.c_int64()
    _check(load().tfmm_mesh_num_rwg(mesh.handle, ctypes.byref(n)))
    return n.value


def tfmm_mesh_rwg(mesh):
    n = tfmm_mesh_num_rwg(mesh)
    edge = np.empty((n, 2), np.int64)
    tri = np.empty((n, 2), np.int64)
    free = np.empty((n, 2), np.int64)
    _check(load().tfmm_mesh_rwg(mesh.handle, _np_ptr(edge), _np_ptr(tri), _np_ptr(free)))
    return edge, tri, free


# ---------------------------------------------------------------------- plan
class Plan:
    def __init__(self, handle):
        self.handle = handle
        self._info = None

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tfmm_plan_destroy(self.handle)
            self.handle = None

    @property
    def info(self):
        if self._info is None:
            self._info = tfmm_plan_info_get(self)
        return self._info


def tfmm_plan_create(mesh, params, stream=None):
    h = ctypes.c_void_p()
    _check(load().tfmm_plan_create(mesh.handle, ctypes.byref(params), _stream(stream), ctypes.byref(h)))
    return Plan(h)


def tfmm_plan_from_tucker(n_rwg, n_theta, n_phi, members, factors, weights=None, max_rhs=1, stream=None,
                          mrhs_precision=0):
    """``members[g]``: global RWG ids of group g; ``factors[g][alpha] = (U_theta, U_phi, U_beta, core)``."""
    G = len(members)
    offsets = np.zeros(G + 1, np.int64)
    offsets[1:] = np.cumsum([len(m) for m in members])
    ids = np.ascontiguousarray(np.concatenate([np.asarray(m, np.int64) for m in members]))
    ranks = np.zeros((G, 2, 3), np.int32)
    chunks = []
    for g in range(G):
        for a in range(2):
            Ut, Up, Ub, C = factors[g][a]
            ranks[g, a] = C.shape
            for arr in (Ut, Up, Ub, C):
                chunks.append(np.asarray(arr, np.complex128).reshape(-1, order="F"))
    flat = np.ascontiguousarray(np.concatenate(chunks))
    w = None if weights is None else np.ascontiguousarray(weights, np.float64)
    h = ctypes.c_void_p()
    _check(load().tfmm_plan_from_tucker(n_rwg, G, n_theta, n_phi, _np_ptr(offsets), _np_ptr(ids), _np_ptr(ranks),
                                        _np_ptr(flat), None if w is None else _np_ptr(w), max_rhs, _stream(stream),
                                        ctypes.byref(h)))
    plan = Plan(h)
    if mrhs_precision:
        tfmm_plan_set_mrhs_precision(plan, mrhs_precision)
    return plan


def tfmm_plan_set_mrhs_precision(plan, precision):
    """0: FP32 CUDA-core chain for R > 1; 2 or 3: tensor cores with 2- or 3-term split BF16."""
    _check(load().tfmm_plan_set_mrhs_precision(plan.handle, int(precision)))


def tfmm_plan_set_dense(plan, tensors, stream=None):
    """``tensors[g][alpha]``: n_theta x n_phi x n_beta complex arrays."""
    flat = np.ascontiguousarray(np.concatenate(
        [np.asarray(A, np.complex128).reshape(-1, order="F") for per in tensors for A in per]))
    _check(load().tfmm_plan_set_dense(plan.handle, _np_ptr(flat), _stream(stream)))
    plan._info = None


def tfmm_plan_info_get(plan):
    info = PlanInfo()
    _check(load().tfmm_plan_info_get(plan.handle, ctypes.byref(info)))
    return info.as_dict()


def tfmm_plan_group(plan, g, alpha):
    nb = ctypes.c_int64()
    r = (ctypes.c_int32 * 3)()
    _check(load().tfmm_plan_group(plan.handle, g, alpha, ctypes.byref(nb), r))
    return nb.value, tuple(r)


def tfmm_plan_members(plan):
    info = plan.info
    off = np.empty(info["n_groups"] + 1, np.int64)
    ids = np.empty(info["n_rwg"], np.int64)
    _check(load().tfmm_plan_members(plan.handle, _np_ptr(off), _np_ptr(ids)))
    return [ids[off[g]:off[g + 1]] for g in range(info["n_groups"])]


def tfmm_plan_centres(plan):
    c = np.empty((plan.info["n_groups"], 3), np.float64)
    _check(load().tfmm_plan_centres(plan.handle, _np_ptr(c)))
    return c


def tfmm_plan_quadrature(plan):
    info = plan.info
    th = np.empty(info["n_theta"])
    wt = np.empty(info["n_theta"])
    ph = np.empty(info["n_phi"])
    wp = ctypes.c_double()
    _check(load().tfmm_plan_quadrature(plan.handle, _np_ptr(th), _np_ptr(wt), _np_ptr(ph), ctypes.byref(wp)))
    return th, wt, ph, wp.value


def tfmm_plan_export_factors(plan, g, alpha):
    nb, (rt, rp, rb) = tfmm_plan_group(plan, g, alpha)
    info = plan.info
    Ut = np.empty(info["n_theta"] * rt, np.complex128)
    Up = np.empty(info["n_phi"] * rp, np.complex128)
    Ub = np.empty(nb * rb, np.complex128)
    C = np.empty(rt * rp * rb, np.complex128)
    _check(load().tfmm_plan_export_factors(plan.handle, g, alpha, _np_ptr(Ut), _np_ptr(Up), _np_ptr(Ub), _np_ptr(C)))
    return (Ut.reshape(info["n_theta"], rt, order="F"), Up.reshape(info["n_phi"], rp, order="F"),
            Ub.reshape(nb, rb, order="F"), C.reshape(rt, rp, rb, order="F"))


def tfmm_plan_farfield(plan, g, stream=None):
    nb, _ = tfmm_plan_group(plan, g, 0)
    info = plan.info
    At = np.empty(info["n_dir"] * nb, np.complex128)
    Ap = np.empty(info["n_dir"] * nb, np.complex128)
    _check(load().tfmm_plan_farfield(plan.handle, g, _np_ptr(At), _np_ptr(Ap), _stream(stream)))
    shape = (info["n_theta"], info["n_phi"], nb)
    return At.reshape(shape, order="F"), Ap.reshape(shape, order="F")


# ------------------------------------------------------------------ hot path
def _ld(t, n_rwg):
    if t.dim() == 1:
        return t.shape[0], 1
    # column-major n_rwg x R block: a (R, ld) row-major tensor
    return t.stride(0), t.shape[0]


def tfmm_aggregate(plan, x, spectra, R=None, ldx=None, stream=None, dense=False):
    """x: complex64 CUDA tensor (n_rwg,) or (R, ldx); spectra: (R, G, 2, N_dir) complex64."""
    if R is None:
        R = 1 if x.dim() == 1 else x.shape[0]
    if ldx is None:
        ldx = x.shape[0] if x.dim() == 1 else x.stride(0)
    fn = load().tfmm_aggregate_dense if dense else load().tfmm_aggregate
    _check(fn(plan.handle, _dev_ptr(x), R, ldx, _dev_ptr(spectra), _stream(stream)))


def tfmm_disaggregate(plan, spectra, y, R=None, apply_weights=True, beta=0.0, ldy=None, stream=None, dense=False):
    if R is None:
        R = 1 if y.dim() == 1 else y.shape[0]
    if ldy is None:
        ldy = y.shape[0] if y.dim() == 1 else y.stride(0)
    b = cfloat(float(np.real(beta)), float(np.imag(beta)))
    fn = load().tfmm_disaggregate_dense if dense else load().tfmm_disaggregate
    _check(fn(plan.handle, _dev_ptr(spectra), R, int(bool(apply_weights)), b, _dev_ptr(y), ldy, _stream(stream)))


def tfmm_aggregate_dense(plan, x, spectra, **kw):
    tfmm_aggregate(plan, x, spectra, dense=True, **kw)


def tfmm_disaggregate_dense(plan, spectra, y, **kw):
    tfmm_disaggregate(plan, spectra, y, dense=True, **kw)


def tfmm_matvec_host(plan, x_host, y_host, R=1, dense=False, stream=None):
    """x_host / y_host: host complex64 buffers (numpy arrays or pinned torch tensors), n_rwg x R column-major."""
    def ptr(a):
        if hasattr(a, "data_ptr"):
            return ctypes.c_void_p(a.data_ptr())
        return _np_ptr(a)
    _check(load().tfmm_matvec_host(plan.handle, ptr(x_host), ptr(y_host), R, int(bool(dense)), _stream(stream)))


def tfmm_translate(plan, spectra_out, spectra_in, R=None, stream=None):
    """Incoming spectra of every group from the outgoing ones (far box pairs), (R, G, 2, N_dir) complex64."""
    if R is None:
        R = spectra_out.shape[0]
    _check(load().tfmm_translate(plan.handle, _dev_ptr(spectra_out), int(R), _dev_ptr(spectra_in), _stream(stream)))


def tfmm_planewave(plan, khat, pol, V, stream=None):
    k = np.ascontiguousarray(khat, np.float64).reshape(-1, 3)
    p = np.ascontiguousarray(pol, np.float64).reshape(-1, 3)
    _check(load().tfmm_planewave(plan.handle, _np_ptr(k), _np_ptr(p), k.shape[0], _dev_ptr(V), _stream(stream)))


def tfmm_planewave_noalloc(plan, khat, pol, V, stream=None):
    """Same as tfmm_planewave, staged through the library's fixed incidence table (no allocation)."""
    k = np.ascontiguousarray(khat, np.float64).reshape(-1, 3)
    p = np.ascontiguousarray(pol, np.float64).reshape(-1, 3)
    _check(load().tfmm_planewave_noalloc(plan.handle, _np_ptr(k), _np_ptr(p), k.shape[0], _dev_ptr(V),
                                         _stream(stream)))


# ------------------------------------------------------------------- runtime
def tfmm_sync(plan, stream=None):
    """Waits for `stream`; raises if a tensor-core tile gave up waiting."""
    _check(load().tfmm_sync(plan.handle, _stream(stream)))


def tfmm_plan_rwg_perm(plan):
    """(group, slot) int32 arrays over the RWGs in mesh order."""
    n = plan.info["n_rwg"]
    grp = np.empty(n, np.int32)
    slot = np.empty(n, np.int32)
    _check(load().tfmm_plan_rwg_perm(plan.handle, _np_ptr(grp), _np_ptr(slot)))
    return grp, slot


def tfmm_plan_save(plan, path):
    _check(load().tfmm_plan_save(plan.handle, os.fsencode(path)))


def tfmm_plan_load(path, stream=None):
    h = ctypes.c_void_p()
    _check(load().tfmm_plan_load(os.fsencode(path), _stream(stream), ctypes.byref(h)))
    return Plan(h)


class Graph:
    """A captured aggregate / disaggregate (tfmm_graph); keeps its plan and buffers alive."""

    def __init__(self, handle, plan, buffers):
        self.handle = handle
        self.plan = plan
        self.buffers = buffers

    def launch(self, stream=None):
        _check(load().tfmm_graph_launch(self.handle, _stream(stream)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tfmm_graph_destroy(self.handle)
            self.handle = None


def tfmm_graph_capture(plan, stages, spectra, x=None, y=None, R=None, apply_weights=True, beta=0.0):
    """stages: 1 aggregate x -> spectra, 2 disaggregate spectra -> y, 3 both (runs them once eagerly)."""
    if R is None:
        R = spectra.shape[0]
    ldx = 0 if x is None else (x.shape[0] if x.dim() == 1 else x.stride(0))
    ldy = 0 if y is None else (y.shape[0] if y.dim() == 1 else y.stride(0))
    b = cfloat(float(np.real(beta)), float(np.imag(beta)))
    h = ctypes.c_void_p()
    _check(load().tfmm_graph_capture(plan.handle, int(stages), None if x is None else _dev_ptr(x), R, ldx,
                                     _dev_ptr(spectra), int(bool(apply_weights)), b,
                                     None if y is None else _dev_ptr(y), ldy, ctypes.byref(h)))
    return Graph(h, plan, (x, spectra, y))


def tfmm_graph_launch(graph, stream=None):
    graph.launch(stream)


def tfmm_graph_destroy(graph):
    if graph.handle:
        _check(load().tfmm_graph_destroy(graph.handle))
        graph.handle = None


def tfmm_plan_tuning_get(plan):
    t = Tuning()
    _check(load().tfmm_plan_tuning_get(plan.handle, ctypes.byref(t)))
    return t.as_dict()


def tfmm_plan_tuning_set(plan, stream=None, **fields):
    t = Tuning()
    _check(load().tfmm_plan_tuning_get(plan.handle, ctypes.byref(t)))
    for k, v in fields.items():
        setattr(t, k, v)
    _check(load().tfmm_plan_tuning_set(plan.handle, ctypes.byref(t), _stream(stream)))


def tfmm_autotune(plan, R=1, budget_ms=2000.0, allow_two_term=False, stream=None):
    t = Tuning()
    _check(load().tfmm_autotune(plan.handle, int(R), float(budget_ms), int(bool(allow_two_term)), _stream(stream),
                                ctypes.byref(t)))
    return t.as_dict()


def tfmm_test_fail_allocation(nth):
    """Test hook: the nth device allocation the library makes from now on fails (0 disarms)."""
    _check(load().tfmm_test_fail_allocation(int(nth)))
