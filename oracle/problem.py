"""Whole-problem setup of the oracle: mesh -> RWGs -> groups -> grid -> tensors -> Tucker.

The setup stage of Sec. II (far-fields of every group by Eq. 4, stored as
n_theta x n_phi x n_beta tensors, Fig. 1a, then compressed by Eq. 6).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import farfield, grid as grid_mod, groups as groups_mod, hosvd, rwg as rwg_mod


@dataclasses.dataclass
class Problem:
    verts: np.ndarray
    tris: np.ndarray
    k: float
    rwg: rwg_mod.RWG
    groups: groups_mod.Groups
    grid: grid_mod.SphereGrid
    tol: float
    order: int
    tensors: list = None   # tensors[g] = (A_theta, A_phi) or None when streaming
    tucker: list = None    # tucker[g] = (Tucker_theta, Tucker_phi)

    @property
    def n_rwg(self):
        return self.rwg.n

    def group_tensors(self, g):
        if self.tensors is not None:
            return self.tensors[g]
        return farfield.group_tensors(self.verts, self.rwg, self.groups.members[g],
                                      self.groups.centre[g], self.k, self.grid, self.order)


def build(verts, tris, k=2.0 * math.pi, box=0.5, digits=3, tol=1e-4, nphi_rule="2L+2",
          L_override=None, order=6, compress=True, keep_tensors=True, groups_subset=None):
    """Build the oracle problem.  ``groups_subset`` restricts tensors/Tucker to some groups."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    r = rwg_mod.build_rwg(verts, tris)
    grp = groups_mod.make_groups(rwg_mod.midpoints(verts, r), box)
    L = L_override if L_override is not None else grid_mod.bandwidth(k, box, digits)
    sg = grid_mod.make_grid(L, nphi_rule)
    P = Problem(verts, tris, k, r, grp, sg, tol, order)
    todo = range(grp.n_groups) if groups_subset is None else groups_subset
    if keep_tensors or compress:
        tens = {}
        tuck = {}
        for g in todo:
            At, Ap = farfield.group_tensors(verts, r, grp.members[g], grp.centre[g], k, sg, order)
            if keep_tensors:
                tens[g] = (At, Ap)
            if compress:
                tuck[g] = (hosvd.thosvd(At, tol), hosvd.thosvd(Ap, tol))
        if groups_subset is None:
            P.tensors = [tens[g] for g in range(grp.n_groups)] if keep_tensors else None
            P.tucker = [tuck[g] for g in range(grp.n_groups)] if compress else None
        else:
            P.tensors = tens if keep_tensors else None
            P.tucker = tuck if compress else None
    return P
