"""End-to-end oracle: coupled-channel problem -> X, R, U (complex128).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

Follows the paper's Type-1 algorithm (Sec. 3.1): build M (here C, in MeV) and
the surface right-hand sides, solve M X = B for all nch columns by partial
pivoting LU, contract to R, then match to the asymptotic functions for U.
The solve is refined with a double-double residual (oracle.refine) unless
``refine_steps=0``.
"""
from __future__ import annotations

import numpy as np

from cc_problems import potential_at

from .collision import collision_matrix, r_matrix
from .lu import lu_factor, lu_solve
from .mesh import kinetic_bloch, lagrange_mesh
from .refine import truth_solve
from .system import assemble_dense


def oracle_solve(p, refine_steps: int = 3, V=None, mesh=None):
    m = mesh if mesh is not None else lagrange_mesh(p.nlag, p.a)
    T0 = kinetic_bloch(p.nlag, p.a, m)
    if V is None:
        V = potential_at(p, m["r"])
    C, Phi = assemble_dense(p, V, m, T0)
    if refine_steps > 0:
        X, hist = truth_solve(C, Phi, steps=refine_steps)
    else:
        LU, piv, info = lu_factor(C)
        if info:
            raise np.linalg.LinAlgError(f"exactly singular pivot at column {info}")
        X = lu_solve(LU, piv, Phi)
        hist = []
    R = r_matrix(p, X, m["f_a"])
    U, nopen = collision_matrix(p, R)
    return {"mesh": m, "T0": T0, "V": V, "C": C, "Phi": Phi, "X": X, "R": R, "U": U,
            "nopen": nopen, "refine_history": hist}
