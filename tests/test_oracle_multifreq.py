"""Pins of the oracle's multi-frequency CMCG (the Conclusion's "one shot" solve), no GPU.

* One harmonic: the same arithmetic as the single-frequency solve (oracle.cmcg), so the
  results agree to rounding.
* Linearity: a sweep with the summed source equals the source-free sweep plus the sweeps from
  rest driven by each harmonic alone (same dt and M), to rounding.
* End to end: each harmonic's filtered result converges to the dense frequency-domain DG solve
  (Section 6's FS, here (i k w0 - B) U = J_k) at that frequency, at second order for P1 / RK2
  with the trapezoid filter as the period is refined.
"""
import math

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I
from oracle import cmcg, dense
from oracle import multifreq as MF
from oracle.dg import inner
from oracle.geometry import build_geometry
from oracle.timestep import Stepper


def _setup(K=2, seed=0):
    p = I.cube_problem(2, 1, 2 * math.pi, (0.5, 0.5, 0.5), (0.3, 1.0, -0.2), 0.3, tol=1e-12,
                       eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.0, 1.0))
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 1)
    rng = np.random.default_rng(seed)
    nodes = I.physical_nodes(p.mesh.verts, p.mesh.tets, 1)
    J = np.stack([I.gaussian_current(nodes, rng.uniform(0.3, 0.7, 3), I.unit_vector(rng), 0.3) for _ in range(K)])
    Ji = 0.5 * np.roll(J, 1, axis=0)
    return p, g, J, Ji


def _rel(a, b, g):
    d = a - b
    return math.sqrt(abs(inner(d, d, g)) / abs(inner(b, b, g)))


def test_one_harmonic_is_the_single_frequency_solve():
    p, g, J, Ji = _setup(K=1)
    a = MF.solve(MF.MultiStepper(g, p.omega, [1]), J, Ji, tol=1e-10, max_iter=200)[0]
    b = cmcg.solve(Stepper(g, p.omega), J[0], Ji[0], tol=1e-10, max_iter=200)
    assert a.iters == b.iters
    assert _rel(a.filtered, b.filtered, g) < 1e-13


def test_summed_source_sweep_is_linear_in_the_harmonics():
    p, g, J, Ji = _setup(K=3)
    harm = [1, 2, 4]
    st = MF.MultiStepper(g, p.omega, harm)
    U = I.random_field(np.random.default_rng(1), p.nt, 1)
    zero = np.zeros_like(U)
    total = st.P(U)
    for k, jr, ji in zip(harm, J, Ji):
        total = total + MF.MultiStepper(g, p.omega, [k]).P_psi(zero, jr[None], ji[None])
    assert _rel(st.P_psi(U, J, Ji), total, g) < 1e-13


def test_every_harmonic_converges_to_its_frequency_domain_solve():
    p, g, J, Ji = _setup(K=2)
    harm = [1, 3]
    errs = {k: [] for k in harm}
    for M in (30, 60):
        res = MF.solve(MF.MultiStepper(g, p.omega, harm, M=M), J, Ji, tol=1e-11, max_iter=400)
        for k, r, jr, ji in zip(harm, res, J, Ji):
            errs[k].append(_rel(r.filtered, dense.frequency_solve(g, k * p.omega, jr, ji), g))
    for k in harm:
        assert errs[k][1] < 5e-2
        assert errs[k][0] / errs[k][1] > 3.0  # second order: the error drops by ~4 as dt halves


def test_harmonics_must_be_positive():
    p, g, J, Ji = _setup(K=1)
    with pytest.raises(ValueError):
        MF.MultiStepper(g, p.omega, [0])
