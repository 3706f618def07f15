"""Seeded synthetic inputs shared by the CUDA path, its tests, the benchmark and the oracle.

This module holds geometry and random numbers only: none of the method's
arithmetic (no basis functions, far-fields, grids or compression) lives here.

* ``icosphere(diameter, nu)`` - class-I geodesic sphere: every face of an
  icosahedron is cut into ``nu**2`` triangles and the vertices are pushed onto
  the sphere.  ``20 nu^2`` triangles, ``10 nu^2 + 2`` vertices, and (the mesh
  being closed) ``30 nu^2`` interior edges, i.e. RWG basis functions.
  nu = 6 D / lambda gives edges of about lambda / 10, the mesh density of the
  30-lambda sphere of Sec. III.B (940,308 RWGs there, 972,000 here).
* ``trihedral(edge, n)`` - square trihedral corner reflector: three mutually
  perpendicular square plates of side ``edge`` meeting at the origin (in the
  planes x = 0, y = 0, z = 0, each in the positive quadrant), every plate an
  n x n grid of squares cut into two right triangles.  ``6 n^2`` triangles and
  ``9 n^2 - 3 n`` interior edges (the three fold edges included), i.e. RWGs;
  n = 69 at edge = 6 lambda gives 42,642 RWGs, the density of the 42,477-RWG
  reflector of Sec. III.A.
* ``complex_gaussian(n, seed)`` - CN(0, 1) vectors: re, im ~ N(0, 1/2).
* ``synthetic_tucker(...)`` - random cores and factors with prescribed, ragged
  shapes, used to exercise the contraction kernels on their own.
* ``WORKLOADS`` - the sphere workloads (diameter, mesh frequency, box size,
  FMM digits, Tucker tolerance, right-hand sides) the tests and the benchmark
  run on.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "icosphere",
    "trihedral",
    "workload_mesh",
    "complex_gaussian",
    "synthetic_tucker",
    "Workload",
    "WORKLOADS",
]


def _icosahedron():
    """12 unit vertices and 20 outward-wound faces of a regular icosahedron."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    # make every face wind counter-clockwise seen from outside
    c = v[f].mean(axis=1)
    nrm = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, c) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def icosphere(diameter: float, nu: int, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere mesh.

    Returns ``(verts, tris)``: ``verts`` float64 (nv, 3), ``tris`` int32 (nt, 3)
    wound counter-clockwise seen from outside.  Vertices are identified
    combinatorially (icosahedron vertex / edge point / face point), so points on
    shared icosahedron edges are never duplicated.
    """
    if nu < 1:
        raise ValueError("nu must be >= 1")
    V, F = _icosahedron()
    # canonical edge ids of the icosahedron
    edges = {}
    for fa in F:
        for a, b in ((fa[0], fa[1]), (fa[1], fa[2]), (fa[2], fa[0])):
            key = (min(a, b), max(a, b))
            if key not in edges:
                edges[key] = len(edges)
    n_edge_pts = nu - 1
    n_face_pts = (nu - 1) * (nu - 2) // 2
    base_edge = 12
    base_face = 12 + len(edges) * n_edge_pts
    nv = base_face + len(F) * n_face_pts
    pos = np.zeros((nv, 3))
    pos[:12] = V
    for (a, b), e in edges.items():
        s = np.arange(1, nu) / nu
        pos[base_edge + e * n_edge_pts: base_edge + (e + 1) * n_edge_pts] = (
            (1 - s)[:, None] * V[a] + s[:, None] * V[b]
        )

    tris = []
    for fi, (A, B, C) in enumerate(F):
        # lattice point (i, j): weight i on B, j on C, nu-i-j on A
        idx = np.full((nu + 1, nu + 1), -1, dtype=np.int64)
        face_counter = 0
        for i in range(nu + 1):
            for j in range(nu + 1 - i):
                k = nu - i - j
                if i == 0 and j == 0:
                    idx[i, j] = A
                elif i == nu:
                    idx[i, j] = B
                elif j == nu:
                    idx[i, j] = C
                elif j == 0:  # on edge A-B, i steps from A
                    idx[i, j] = _edge_point(edges, A, B, i, nu, base_edge)
                elif i == 0:  # on edge A-C
                    idx[i, j] = _edge_point(edges, A, C, j, nu, base_edge)
                elif k == 0:  # on edge B-C, j steps from B
                    idx[i, j] = _edge_point(edges, B, C, j, nu, base_edge)
                else:
                    gid = base_face + fi * n_face_pts + face_counter
                    face_counter += 1
                    pos[gid] = (k * V[A] + i * V[B] + j * V[C]) / nu
                    idx[i, j] = gid
        for i in range(nu):
            for j in range(nu - i):
                tris.append((idx[i, j], idx[i + 1, j], idx[i, j + 1]))
                if i + j < nu - 1:
                    tris.append((idx[i + 1, j], idx[i + 1, j + 1], idx[i, j + 1]))
    pos /= np.linalg.norm(pos, axis=1, keepdims=True)
    pos = pos * (0.5 * diameter) + np.asarray(center, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int32)
    return pos, tris


def trihedral(edge: float, n: int):
    """Square trihedral corner reflector (three plates of side ``edge``, n x n squares each).

    Returns ``(verts, tris)`` like ``icosphere``.  Vertices are the lattice points
    (i, j, k) h, h = edge / n, with at least one index zero; a point with two zero
    indices lies on a fold line and belongs to two plates, so the plates are
    joined along the three axes.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = edge / n
    ids = {}
    pos = []

    def vid(i, j, k):
        key = (i, j, k)
        v = ids.get(key)
        if v is None:
            v = len(pos)
            ids[key] = v
            pos.append((i * h, j * h, k * h))
        return v

    tris = []
    # plate z = 0 (x, y), plate y = 0 (x, z), plate x = 0 (y, z)
    planes = (lambda a, b: (a, b, 0), lambda a, b: (a, 0, b), lambda a, b: (0, a, b))
    for P in planes:
        for a in range(n):
            for b in range(n):
                p00, p10 = vid(*P(a, b)), vid(*P(a + 1, b))
                p01, p11 = vid(*P(a, b + 1)), vid(*P(a + 1, b + 1))
                tris.append((p00, p10, p11))
                tris.append((p00, p11, p01))
    return np.asarray(pos, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def _edge_point(edges, a, b, step, nu, base_edge):
    """Global id of the point ``step`` lattice steps from ``a`` towards ``b``."""
    key = (min(a, b), max(a, b))
    e = edges[key]
    s = step if a < b else nu - step
    return base_edge + e * (nu - 1) + (s - 1)


def complex_gaussian(shape, seed: int, dtype=np.complex128):
    """Seeded CN(0, 1) samples: real and imaginary parts ~ N(0, 1/2)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return ((re + 1j * im) * math.sqrt(0.5)).astype(dtype)


@dataclasses.dataclass
class SyntheticGroup:
    """Factors of one (group, component) pair, in the shapes of Eq. 6."""

    U_theta: np.ndarray  # n_theta x r_theta
    U_phi: np.ndarray    # n_phi x r_phi
    U_beta: np.ndarray   # n_beta x r_beta
    core: np.ndarray     # r_theta x r_phi x r_beta


def synthetic_tucker(n_theta, n_phi, n_beta_list, ranks_list, seed):
    """Random factors with given shapes; ``ranks_list[g] = ((rt, rp, rb), (rt, rp, rb))``.

    Entries are CN(0, 1) scaled by 1/sqrt(n) so that the contractions stay O(1).
    Returns ``[[SyntheticGroup(theta), SyntheticGroup(phi)] for each group]``.
    """
    rng = np.random.default_rng(seed)

    def cn(*shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * math.sqrt(0.5)

    out = []
    for nb, ranks in zip(n_beta_list, ranks_list):
        per_alpha = []
        for (rt, rp, rb) in ranks:
            per_alpha.append(
                SyntheticGroup(
                    U_theta=cn(n_theta, rt) / math.sqrt(n_theta),
                    U_phi=cn(n_phi, rp) / math.sqrt(n_phi),
                    U_beta=cn(nb, rb) / math.sqrt(max(nb, 1)),
                    core=cn(rt, rp, rb) / math.sqrt(rb),
                )
            )
        out.append(per_alpha)
    return out


@dataclasses.dataclass(frozen=True)
class Workload:
    """A PEC workload: mesh, box grid, FMM accuracy, Tucker tolerance, RHS."""

    name: str
    diameter: float      # sphere diameter, or trihedral plate edge, in wavelengths (lambda = 1, k = 2 pi)
    nu: int              # icosphere frequency (20 nu^2 triangles, 30 nu^2 RWGs) or squares per plate edge
    box: float           # leaf box edge a, in wavelengths
    digits: int          # FMM accuracy d0
    tol: float           # Tucker tolerance gamma
    nrhs: int            # right-hand sides
    rhs: str             # "gaussian" | "planewave+gaussian" | "planewave_sweep" | "planewave_corner"
    seed: int
    shape: str = "sphere"  # "sphere" | "trihedral"
    nphi_rule: int = 1     # 1: N_phi = 2(L+1) (the sphere workloads), 0: 2L+1 (the paper's grid)

    @property
    def n_tri(self):
        if self.shape == "trihedral":
            return 6 * self.nu * self.nu
        return 20 * self.nu * self.nu

    @property
    def n_rwg(self):
        if self.shape == "trihedral":
            return 9 * self.nu * self.nu - 3 * self.nu
        return 30 * self.nu * self.nu


def workload_mesh(w: Workload):
    """``(verts, tris)`` of a workload's geometry."""
    if w.shape == "trihedral":
        return trihedral(w.diameter, w.nu)
    return icosphere(w.diameter, w.nu)


WORKLOADS = {
    "sphere2": Workload("sphere2", 2.0, 12, 0.5, 3, 1e-4, 1, "gaussian", 1),
    "sphere10": Workload("sphere10", 10.0, 60, 1.0, 6, 1e-6, 1, "planewave+gaussian", 2),
    "sphere30": Workload("sphere30", 30.0, 180, 2.0, 6, 1e-6, 1, "gaussian", 3),
    "sphere30_rcs128": Workload("sphere30_rcs128", 30.0, 180, 2.0, 6, 1e-6, 128, "planewave_sweep", 4),
    "sphere20_sweep": Workload("sphere20_sweep", 20.0, 120, 2.0, 6, 1e-6, 16, "gaussian", 5),
    # the 10-lambda sphere with 128 CN(0,1) RHS: a small case of the many-RHS path (profiling)
    "sphere10_rhs128": Workload("sphere10_rhs128", 10.0, 60, 1.0, 6, 1e-6, 128, "gaussian", 6),
    # the trihedral corner reflector of Sec. III.A: 6-lambda plates, 2-lambda boxes, 5 digits
    # (L = 37), N_phi = 2L + 1 as in Tables I-II, gamma = 1e-6, the paper's plane wave
    # (theta_inc = 135 deg, phi_inc = 225 deg, theta-polarised)
    "corner6": Workload("corner6", 6.0, 69, 2.0, 5, 1e-6, 1, "planewave_corner", 7, shape="trihedral", nphi_rule=0),
}
