"""Pins of the oracle's conductivity term (Eq. maxwell_time_strong, Section 1: eps dE/dt + sigma E + curl H = J; coefficients Section 3.1, discrete term Section 5.2.2), no GPU.

* Energy: with the centred flux and PEC walls the only loss is Ohmic, so
  (U, B U)_{eps,mu} = -sum_K sigma_K |J_K| E_K^T M E_K exactly (random sigma and U).
* Adjoint: Sigma leaves E unchanged and the sigma block is symmetric, so P* = Sigma P Sigma
  stays the (eps,mu)-adjoint of P: (P U, W) = (U, P* W).
* Static modes: the kernel of B (sigma = 0) splits into pure-E and pure-H fields; with a uniform
  sigma/eps = s a pure-E kernel field is an eigenvector of B_sigma for -s, so one period
  multiplies it by the RK stability polynomial R(-s dt)^M exactly.
* End to end: CMCG with sigma reaches the frequency-domain DG solve ((i w + sigma/eps) in the
  E rows) up to the time discretisation.
"""
import math

import numpy as np

from paper_2106_02858_gb300 import inputs as I
from oracle import cmcg, dense
from oracle.dg import apply_B, inner
from oracle.geometry import build_geometry
from oracle.refelem import ref_element
from oracle.timestep import Stepper


def _pec_cube(n, q, sigma, eps=None):
    m = I.kuhn_cube_mesh(n)
    tags = np.where(m.tags == I.IMPEDANCE, I.PEC, m.tags).astype(np.uint8)
    eps = np.ones(m.nt) if eps is None else eps
    return m, build_geometry(m.verts, m.tets, tags, eps, np.ones(m.nt), q, sigma=sigma)


def test_ohmic_loss_is_the_only_energy_change_with_the_centred_flux():
    rng = np.random.default_rng(0)
    m = I.kuhn_cube_mesh(2)
    tags = np.where(m.tags == I.IMPEDANCE, I.PEC, m.tags).astype(np.uint8)
    eps, mu, sig = rng.uniform(1, 3, m.nt), rng.uniform(1, 2, m.nt), rng.uniform(0, 2, m.nt)
    g = build_geometry(m.verts, m.tets, tags, eps, mu, 2, sigma=sig)
    U = I.random_field(rng, m.nt, 2)
    lhs = inner(U, apply_B(U, g, flux="centred"), g)
    M = ref_element(2).M
    E = U[:, :3, :]
    rhs = -np.einsum("k,kcn,nm,kcm->", sig * g.J, E, M, E)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_adjoint_identity_with_conductivity():
    rng = np.random.default_rng(1)
    sig = rng.uniform(0, 1.5, 48)
    m, g = _pec_cube(2, 1, sig)
    st = Stepper(g, 2 * math.pi)
    U, W = I.random_field(rng, m.nt, 1), I.random_field(rng, m.nt, 1)
    a, b = inner(st.P(U), W, g), inner(U, st.P_star(W), g)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_static_electric_modes_decay_by_the_stability_polynomial():
    s = 0.7
    m, g0 = _pec_cube(1, 1, None)
    B = dense.dense_B(g0)
    _u, sv, vt = np.linalg.svd(B)
    null = vt[sv < 1e-10 * sv[0]].reshape(-1, m.nt, 6, 4)
    E = null.copy()
    E[:, :, 3:, :] = 0.0
    k = int(np.argmax([np.linalg.norm(x) for x in E]))
    v = E[k] / np.linalg.norm(E[k])
    assert np.abs(apply_B(v, g0)).max() < 1e-10  # the pure-E part is itself static
    _m, gs = _pec_cube(1, 1, np.full(m.nt, s))
    st = Stepper(gs, 2 * math.pi)
    z = -s * st.dt
    R = sum(z ** j / math.factorial(j) for j in range(3 if st.integrator == "rk2" else 5))
    assert np.allclose(st.P(v), R ** st.M * v, rtol=0, atol=1e-12)


def test_cmcg_with_conductivity_reaches_the_frequency_domain_solve():
    rng = np.random.default_rng(2)
    p = I.cube_problem(2, 1, 2 * math.pi, (0.5, 0.5, 0.5), (0.3, 1.0, -0.2), 0.3, tol=1e-12)
    sig = rng.uniform(0.5, 2.0, p.nt)
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 1, sigma=sig)
    fs = dense.frequency_solve(g, p.omega, p.j_re, p.j_im)
    errs = []
    for M in (24, 48):
        st = Stepper(g, p.omega, M=M)
        res = cmcg.solve(st, p.j_re, p.j_im, tol=1e-11, max_iter=400)
        d = res.filtered - fs
        errs.append(math.sqrt(abs(inner(d, d, g)) / abs(inner(fs, fs, g))))
    assert errs[1] < 1e-2
    assert errs[0] / errs[1] > 3.0  # second order (RK2 + trapezoid): ratio 4 as dt halves
