"""Oracle jobs that GPU tests run in spawned worker processes (test infrastructure only).

Each job rebuilds its seeded inputs from a small spec, so only the spec and the
result cross the process boundary.  Workers are started with the ``spawn``
method: they never inherit a CUDA context.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2106_02858_gb300 import inputs as I

# Shapes of the uneven-batch recipe checked against the oracle: (n, q, omega).
BLOCK_SHAPES = [(8, 1, 2 * math.pi), (7, 1, 4 * math.pi), (6, 2, 4 * math.pi), (6, 3, 8 * math.pi)]
BLOCK_SEED = 1


def problem(spec):
    kind = spec[0]
    if kind == "block":
        return I.block_eps_subset(BLOCK_SHAPES, seed=BLOCK_SEED)[spec[1]]
    if kind == "rhs":  # source k of the batched-source workload (32 sources, 384-tet cube, P3)
        b = I.batched_rhs(nrhs=32)
        return I.Problem(f"rhs{spec[1]}", b.mesh, b.eps, b.mu, b.omega, b.order, b.j_re[spec[1]], b.j_im[spec[1]],
                         b.tol)
    raise ValueError(spec)


def cmcg_solve(spec, tol: float, max_iter: int):
    """Filtered CMCG result of the oracle, (nt, 6, Np) complex, and its iteration count."""
    from oracle import cmcg as ocmcg
    from oracle.geometry import build_geometry
    from oracle.timestep import Stepper
    p = problem(spec)
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)
    r = ocmcg.solve(Stepper(g, p.omega), p.j_re, p.j_im, tol=tol, max_iter=max_iter)
    return np.asarray(r.filtered), int(r.iters)
