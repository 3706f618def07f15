"""FP64 CPU oracle for Tucker-compressed FMM aggregation / disaggregation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the C-ABI library and its Python binding) never calls it and shares no code
with it; the only thing both sides consume is the seeded input module
``paper_2103_05822_gb300.inputs`` (meshes and random numbers).

Everything is plain NumPy in complex128 / float64, written from the paper:

* ``rwg``      - RWG basis functions on a triangle mesh (Sec. II.A, ref. [20]).
* ``grid``     - FMM bandwidth L and the (L+1) x N_phi spherical grid (Sec. II.A).
* ``groups``   - the FMM-FFT box grid and its non-empty boxes (Sec. II.A, Eq. 3).
* ``farfield`` - the far-field of each RWG, Eq. 4, by triangle quadrature.
* ``hosvd``    - truncated higher-order SVD, Eq. 6 (Sec. II.B, ref. [26]).
* ``apply``    - dense aggregation / disaggregation (Eqs. 3, 5, Figs. 2a, 3a)
                 and the Tucker procedures of Figs. 2b and 3b.
* ``planewave``- the RWG-tested plane-wave excitation V_m of Eq. 2.
* ``memory``   - far-field storage of the dense and the Tucker format.
* ``svd``      - the truncated-SVD comparator of Sec. II.C (ref. [11]).
* ``translation`` - the FMM translation stage between aggregation and
                 disaggregation (addition theorem, ref. [25]), by direct sums.

Every function is pinned by ``tests/test_oracle_*.py`` to something other than
itself (closed forms, brute force, invariants, the paper's printed numbers).
"""
from . import rwg, grid, groups, farfield, hosvd, apply, planewave, memory, problem, svd, translation  # noqa: F401
