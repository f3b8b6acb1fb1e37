"""Pins of the oracle's time stepping, propagators and filters (no GPU).

* CFL: M from Eq. cfl with the printed c_1 = 0.24 and the closed-form inradius
  h / (1 + sqrt 2) of a Kuhn tetrahedron (41 steps on the 4^3 cube at w = 2 pi).
* The sweep equals the dense amplification polynomial: P v = R(dt lambda)^M v
  for eigenvectors v of the dense B, with R the RK2 / RK4 stability polynomial.
* RK2 / RK4 converge to exp(T B) at orders 2 / 4 (scipy.linalg.expm).
* Adjoint: (P U, W)_M = (U, P* W)_M, and P* = Sigma P Sigma (Section 4.1.2).
* Affine decomposition P_psi U = P U + P_psi 0 (Eq. decomposition_propagator).
* Filters: the trapezoid rule returns a exactly for sampled Re(a e^{i w t});
  the Hermite rule integrates cubic x e^{-i w t} exactly (Gauss-Legendre check);
  a constant filters to 0; the moments match quadrature.
* Stability of the printed c_q on Kuhn meshes: spectral radius of R(dt B) <= 1.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from paper_2106_02858_gb300 import inputs as I
from oracle import dense, filtering
from oracle.dg import inner
from oracle.geometry import build_geometry
from oracle.timestep import Stepper, steps_per_period

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cfl_constants.json")


def _geo(n, q, eps=None, seed=0):
    m = I.kuhn_cube_mesh(n)
    rng = np.random.default_rng(seed)
    e = np.ones(m.nt) if eps is None else rng.uniform(1, 4, m.nt)
    return build_geometry(m.verts, m.tets, m.tags, e, np.ones(m.nt), q), m


def test_cfl_step_count_matches_printed_constants():
    gold = json.load(open(GOLDEN))
    g, _ = _geo(4, 1)
    h = 0.25
    expected = math.ceil(1.0 / (gold["c1"] * h / (1 + math.sqrt(2))))
    assert expected == 41
    assert steps_per_period(g, 2 * math.pi, c_q=gold["c1"]) == 41
    # the 3D default for P1 is half the printed constant (see the next test)
    assert steps_per_period(g, 2 * math.pi) == math.ceil(1.0 / (0.5 * gold["c1"] * h / (1 + math.sqrt(2)))) == 81
    g3, _ = _geo(4, 3)
    assert steps_per_period(g3, 4 * math.pi) == math.ceil(0.5 / (gold["c3"] * h / (1 + math.sqrt(2))))
    p = I.scatterer_sphere()
    g2 = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 2)
    assert steps_per_period(g2, p.omega) == math.ceil(0.5 / (0.12 * (1 / 24) / (1 + math.sqrt(2)))) == 242


def test_printed_rk2_constant_grows_on_an_8_cube_with_permittivity_blocks():
    """The printed c_1 = 0.24 is a 2D constant (Section 5.3).  On the 8^3 Kuhn cube with eps on a
    2x2x2 block partition (P1, RK2, omega = 4 pi) power iteration on the oracle's period map
    finds a mode that one period multiplies by about 11 at c_1 = 0.24, while at half the
    constant, the 3D default, the period map does not grow (its largest factor tends to 1, the
    static modes).  Smaller meshes (n <= 4) are stable at both constants."""
    gold = json.load(open(GOLDEN))
    p = I.block_eps_problem(8, 1, 4 * math.pi, np.random.default_rng(8))
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 1)
    from oracle.dg import norm

    def growth(c):
        st = Stepper(g, p.omega, c_q=c)
        u = I.random_field(np.random.default_rng(0), p.nt, 1)
        u /= norm(u, g)
        out = []
        for _ in range(4):
            v = st.P(u)
            out.append(norm(v, g))
            u = v / out[-1]
        return st.M, out

    M_printed, g_printed = growth(gold["c1"])
    M_half, g_half = growth(0.5 * gold["c1"])
    assert M_printed == 29 and M_half == 58
    assert g_printed[-1] > 5.0
    assert max(g_half) < 1.0 + 1e-9


@pytest.mark.parametrize("q", [1, 2])
def test_sweep_equals_amplification_polynomial_on_eigenvectors(q):
    g, m = _geo(1, q, eps=True)
    st = Stepper(g, 2 * math.pi)
    B = dense.dense_B(g)
    lam, V = np.linalg.eig(B)
    s = 2 if st.integrator == "rk2" else 4
    for idx in np.argsort(-np.abs(lam))[:6]:
        v = V[:, idx]
        z = st.dt * lam[idx]
        Rz = sum(z**k / math.factorial(k) for k in range(s + 1))
        shape = (m.nt, 6, -1)
        out = st.P(v.real.reshape(shape)) + 1j * st.P(v.imag.reshape(shape))
        assert np.allclose(out.reshape(-1), Rz**st.M * v, atol=1e-12 * max(1.0, abs(Rz) ** st.M))


@pytest.mark.parametrize("q,order", [(1, 2), (2, 4)])
def test_rk_order_against_matrix_exponential(q, order):
    g, m = _geo(1, q)
    B = dense.dense_B(g)
    T = 0.25
    exact = scipy.linalg.expm(T * B)
    U0 = I.random_field(np.random.default_rng(0), m.nt, q)
    ref = (exact @ U0.reshape(-1)).reshape(U0.shape)
    errs = []
    st0 = Stepper(g, 2 * math.pi / T)
    for M in (st0.M * 2, st0.M * 4):
        st = Stepper(g, 2 * math.pi / T, M=M)
        errs.append(np.abs(st.P(U0) - ref).max())
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.3


@pytest.mark.parametrize("q", [1, 2, 3])
def test_discrete_adjoint_identity(q):
    g, m = _geo(1, q, eps=True)
    st = Stepper(g, 4 * math.pi)
    rng = np.random.default_rng(1)
    U, W = I.random_field(rng, m.nt, q), I.random_field(rng, m.nt, q)
    a = inner(st.P(U), W, g)
    b = inner(U, st.P_star(W), g)
    assert abs(a - b) < 1e-13 * max(abs(a), 1.0)
    assert np.allclose(st.P_star(W), st.P_star_via_sigma(W), atol=1e-14)


def test_affine_decomposition():
    p = I.plain_fp64_cube(1, 2)
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 2)
    st = Stepper(g, p.omega)
    U = I.random_field(np.random.default_rng(2), p.nt, 2)
    lhs = st.P_psi(U, p.j_re, p.j_im)
    rhs = st.P(U) + st.P_psi(np.zeros_like(U), p.j_re, p.j_im)
    assert np.allclose(lhs, rhs, atol=1e-13)


def test_trapezoid_filter_recovers_harmonic_amplitude():
    omega, M = 3.0, 17
    T = 2 * math.pi / omega
    dt = T / M
    a = np.array([0.3 - 1.2j, 2.0 + 0.5j])
    states = [np.real(a * np.exp(1j * omega * m * dt)) for m in range(M + 1)]
    F = filtering.filter_trapezoid(states, omega, dt, T)
    assert np.allclose(F, a, atol=1e-14)
    const = [np.ones(2) for _ in range(M + 1)]
    assert np.allclose(filtering.filter_trapezoid(const, omega, dt, T), 0, atol=1e-14)


def test_hermite_filter_exact_for_cubics():
    omega, M = 2.5, 9
    T = 2 * math.pi / omega
    dt = T / M
    c = np.array([0.7, -1.1, 0.4, 0.9])
    p = lambda t: c[0] + c[1] * t + c[2] * t**2 + c[3] * t**3
    dp = lambda t: c[1] + 2 * c[2] * t + 3 * c[3] * t**2
    states = [np.array([p(m * dt)]) for m in range(M + 1)]
    derivs = [np.array([dp(m * dt)]) for m in range(M + 1)]
    F = filtering.filter_hermite(states, derivs, omega, dt, T)[0]
    x, w = np.polynomial.legendre.leggauss(40)
    t = 0.5 * T * (x + 1)
    exact = (2 / T) * 0.5 * T * np.sum(w * p(t) * np.exp(-1j * omega * t))
    assert abs(F - exact) < 1e-13
    const = [np.ones(1) for _ in range(M + 1)]
    zero = [np.zeros(1) for _ in range(M + 1)]
    assert abs(filtering.filter_hermite(const, zero, omega, dt, T)[0]) < 1e-14


@pytest.mark.parametrize("theta", [1e-6, 0.2, 1.0, 3.0, 9.0])
def test_moments_against_quadrature(theta):
    x, w = np.polynomial.legendre.leggauss(60)
    s = 0.5 * (x + 1)
    I_ = filtering.moments(theta)
    for k in range(4):
        assert abs(I_[k] - 0.5 * np.sum(w * s**k * np.exp(-1j * theta * s))) < 1e-14


@pytest.mark.parametrize("q", [1, 2, 3])
def test_printed_cfl_constants_are_stable_on_kuhn_tets(q):
    g, m = _geo(1 if q == 3 else 2, q)
    st = Stepper(g, 2 * math.pi)
    lam = np.linalg.eigvals(dense.dense_B(g))
    s = 2 if st.integrator == "rk2" else 4
    z = st.dt * lam
    R = sum(z**k / math.factorial(k) for k in range(s + 1))
    assert np.max(np.abs(R)) <= 1 + 1e-12
