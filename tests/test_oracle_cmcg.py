"""Pins of the oracle's controllability solver (no GPU).

* Brute force: on a 2^3-cube P1 mesh (1,152 dofs) the dense period map P is
  assembled from the dense B, (I - P) x = G is solved in the (eps,mu)-weighted
  minimum-norm least-squares sense, and both x and F_psi(x) agree with the
  oracle's CG (Section 2.2, Algorithm cmcg) to 1e-10 relative.
* J(U0^l) decreases monotonically along the CG iterates (CG on a quadratic).
* Section 6: CMCG and the frequency-domain DG solve (i w M + K) U = M J differ
  only by the time discretisation, so F_psi(x) -> U_FS at the integrator's
  order (2 for RK2 + trapezoid, 4 for RK4 + Hermite).  This pins the 2/T of the
  filter, the source timing and the sign choices.
* The discrete operator has a kernel (static gradient modes) and the filter
  removes it: F_w(v) = 0 for v in ker B.
"""
import math

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I
from oracle import cmcg, dense
from oracle.dg import inner
from oracle.filtering import filtered_sweep
from oracle.geometry import build_geometry
from oracle.timestep import Stepper


def _problem(n, q, omega, centre=(0.5, 0.5, 0.5)):
    p = I.cube_problem(n, q, omega, centre, (0.3, 1.0, -0.2), 0.3, tol=1e-12)
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, q)
    return p, g


def _min_norm_solution(g, P, G):
    Mfull = dense.dense_M(g)
    C = np.linalg.cholesky(Mfull)  # M = C C^T, ||v||_M = ||C^T v||
    Ct = C.T
    n = P.shape[0]
    A = Ct @ (np.eye(n) - P) @ np.linalg.inv(Ct)
    y = np.linalg.lstsq(A, Ct @ G.reshape(-1), rcond=1e-10)[0]
    return np.linalg.solve(Ct, y).reshape(G.shape)


def _rel(a, b, g):
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


def test_cg_matches_dense_minimum_norm_solution():
    p, g = _problem(2, 1, 2 * math.pi)
    st = Stepper(g, p.omega)
    res = cmcg.solve(st, p.j_re, p.j_im, tol=1e-12, max_iter=400, track_functional=True)
    assert res.converged
    P = dense.period_map(dense.dense_B(g), st.dt, st.M, st.integrator)
    G = st.P_psi(np.zeros((p.nt, 6, p.np_)), p.j_re, p.j_im)
    x = _min_norm_solution(g, P, G)
    # (I - P) really is singular here, so the minimum-norm choice matters
    sv = np.linalg.svd(np.eye(P.shape[0]) - P, compute_uv=False)
    assert sv[-1] < 1e-10 * sv[0]
    assert _rel(res.U0, x, g) < 1e-9
    assert _rel(res.filtered, filtered_sweep(st, x, p.j_re, p.j_im), g) < 1e-10
    J = np.array(res.functionals)
    assert np.all(np.diff(J) <= 1e-14 * J[0])


@pytest.mark.parametrize("q,order", [(1, 2), (2, 4)])
def test_filtered_periodic_solution_converges_to_frequency_domain_solution(q, order):
    p, g = _problem(1, q, 2 * math.pi)
    U_fs = dense.frequency_solve(g, p.omega, p.j_re, p.j_im)
    B = dense.dense_B(g)
    st0 = Stepper(g, p.omega)
    errs = []
    for M in (st0.M, 2 * st0.M, 4 * st0.M):
        st = Stepper(g, p.omega, M=M)
        P = dense.period_map(B, st.dt, st.M, st.integrator)
        G = st.P_psi(np.zeros((p.nt, 6, p.np_)), p.j_re, p.j_im)
        x = _min_norm_solution(g, P, G)
        errs.append(_rel(filtered_sweep(st, x, p.j_re, p.j_im), U_fs, g))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - order) < 0.35, (errs, rates)


def test_filter_removes_static_kernel_modes():
    p, g = _problem(2, 1, 2 * math.pi)
    st = Stepper(g, p.omega)
    B = dense.dense_B(g)
    w, V = np.linalg.eigh(B.T @ B)
    ker = V[:, w < 1e-20 * w.max()]
    assert ker.shape[1] >= 1
    v = ker[:, 0].reshape(p.nt, 6, p.np_)
    assert np.allclose(st.P(v), v, atol=1e-12)
    F = filtered_sweep(st, v)  # no source
    assert np.abs(F).max() < 1e-12
