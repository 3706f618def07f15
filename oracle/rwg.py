"""RWG basis functions (Sec. II.A; Rao-Wilton-Glisson, ref. [20]).

An RWG function lives on the two triangles T+ and T- sharing an interior edge
of length l.  With p+ / p- the vertices of T+ / T- opposite that edge and A+ /
A- their areas:

    b(r) = l / (2 A+) (r - p+)   on T+
    b(r) = l / (2 A-) (p- - r)   on T-

Reading of what the paper leaves open (it cites [20] only):
* only edges shared by exactly two triangles carry an RWG;
* RWGs are numbered by their edge (min vertex id, max vertex id), ascending;
* T+ is the adjacent triangle with the lower triangle index.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class RWG:
    edge: np.ndarray     # (N, 2) vertex ids of the common edge, ascending
    tri: np.ndarray      # (N, 2) triangle ids (T+, T-)
    free: np.ndarray     # (N, 2) vertex ids of p+ and p-
    length: np.ndarray   # (N,)   common edge length l
    area: np.ndarray     # (N, 2) areas A+ and A-

    @property
    def n(self):
        return len(self.length)


def build_rwg(verts: np.ndarray, tris: np.ndarray) -> RWG:
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    owners = {}
    for t, (a, b, c) in enumerate(tris):
        for u, v, w in ((a, b, c), (b, c, a), (c, a, b)):
            key = (min(u, v), max(u, v))
            owners.setdefault(key, []).append((t, w))
    keys = sorted(k for k, o in owners.items() if len(o) == 2)
    edge = np.array(keys, dtype=np.int64).reshape(-1, 2)
    tri = np.empty((len(keys), 2), dtype=np.int64)
    free = np.empty((len(keys), 2), dtype=np.int64)
    for i, k in enumerate(keys):
        (t0, f0), (t1, f1) = sorted(owners[k])
        tri[i] = (t0, t1)
        free[i] = (f0, f1)
    length = np.linalg.norm(verts[edge[:, 1]] - verts[edge[:, 0]], axis=1)
    area = np.empty((len(keys), 2))
    for s in range(2):
        p = verts[tris[tri[:, s]]]
        area[:, s] = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)
    return RWG(edge=edge, tri=tri, free=free, length=length, area=area)


def midpoints(verts, rwg: RWG):
    """Midpoint of each RWG's common edge (the point used to assign it to a box)."""
    verts = np.asarray(verts, dtype=np.float64)
    return 0.5 * (verts[rwg.edge[:, 0]] + verts[rwg.edge[:, 1]])


def evaluate(verts, rwg: RWG, n: int, side: int, r: np.ndarray):
    """b_n(r) at points r (..., 3) that lie on triangle ``side`` (0: T+, 1: T-)."""
    verts = np.asarray(verts, dtype=np.float64)
    p = verts[rwg.free[n, side]]
    scale = rwg.length[n] / (2.0 * rwg.area[n, side])
    return scale * (r - p) if side == 0 else scale * (p - r)


def divergence(rwg: RWG, n: int, side: int):
    """Surface divergence of b_n: +l/A+ on T+, -l/A- on T-."""
    v = rwg.length[n] / rwg.area[n, side]
    return v if side == 0 else -v
