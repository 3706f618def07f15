"""FMM-FFT box grid and groups (Sec. II.A, the K_x x K_y x K_z grid of Eq. 3).

Readings of what the paper leaves open:
* the grid of cubes of edge a is anchored at the minimum corner of the mesh's
  bounding box; K_p = max(1, ceil(extent_p / a));
* an RWG belongs to the box holding the midpoint of its common edge,
  floor((x - x0) / a) clamped to [0, K_p - 1];
* the box centre r_v is x0 + (index + 1/2) a;
* only non-empty boxes ("groups") are kept, ordered by the linear box index
  ix + K_x (iy + K_y iz) (z slowest); inside a group RWGs keep ascending
  global order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Groups:
    box: float
    origin: np.ndarray     # (3,)
    K: tuple               # (Kx, Ky, Kz)
    box_index: np.ndarray  # (G, 3) integer box coordinates
    centre: np.ndarray     # (G, 3)
    members: list          # G arrays of global RWG ids, ascending

    @property
    def n_groups(self):
        return len(self.members)


def make_groups(points: np.ndarray, box: float) -> Groups:
    """Group the RWG reference points ``points`` (N, 3) into boxes of edge ``box``."""
    points = np.asarray(points, dtype=np.float64)
    lo = points.min(axis=0)
    hi = points.max(axis=0)
    K = tuple(max(1, int(math.ceil((hi[p] - lo[p]) / box))) for p in range(3))
    idx = np.floor((points - lo) / box).astype(np.int64)
    for p in range(3):
        idx[:, p] = np.clip(idx[:, p], 0, K[p] - 1)
    lin = idx[:, 0] + K[0] * (idx[:, 1] + K[1] * idx[:, 2])
    boxes = np.unique(lin)
    members = []
    bidx = np.empty((len(boxes), 3), dtype=np.int64)
    for g, b in enumerate(boxes):
        members.append(np.nonzero(lin == b)[0])
        bidx[g] = (b % K[0], (b // K[0]) % K[1], b // (K[0] * K[1]))
    centre = lo + (bidx + 0.5) * box
    return Groups(box, lo, K, bidx, centre, members)
