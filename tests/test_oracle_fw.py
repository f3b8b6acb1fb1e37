"""Pins of the oracle's limiting-amplitude (FW) baseline (no GPU).

* Brute force: P_psi is affine, P_psi U = P U + G with G = P_psi 0, so the FW
  state after l periods is (I + P + ... + P^(l-1)) G.  On a 2^3-cube P1 mesh the
  dense period map P (from the dense B and the RK amplification matrix) gives
  that sum independently of the oracle's sweeps; they agree to 1e-11.
* Limit (Section 1, limiting amplitude; Section 6, FW and CMCG share the
  discrete limit): on the open cube the transients decay, and F_psi of the FW
  state approaches the CMCG result at least as fast as the largest |eigenvalue|
  of P below 1 (computed from the dense P) predicts.
* Zero periods: FW returns F_psi 0, the filter of the first period from rest.
"""
import math

import numpy as np

from paper_2106_02858_gb300 import inputs as I
from oracle import cmcg, dense, fw
from oracle.dg import inner
from oracle.filtering import filtered_sweep
from oracle.geometry import build_geometry
from oracle.timestep import Stepper


def _setup(n=2, q=1, omega=2 * math.pi):
    p = I.cube_problem(n, q, omega, (0.5, 0.4, 0.6), (0.3, 1.0, -0.2), 0.3, tol=1e-12)
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, q)
    return p, g, Stepper(g, p.omega)


def _rel(a, b, g):
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


def test_fw_state_is_the_partial_sum_of_the_dense_period_map():
    p, g, st = _setup()
    P = dense.period_map(dense.dense_B(g), st.dt, st.M, st.integrator)
    G = st.P_psi(np.zeros((p.nt, 6, p.np_)), p.j_re, p.j_im).reshape(-1)
    acc, term = np.zeros_like(G), G.copy()
    for l in range(1, 7):
        acc = acc + term
        term = P @ term
        got = fw.fw_state(st, p.j_re, p.j_im, l).reshape(-1)
        assert np.linalg.norm(got - acc) <= 1e-11 * np.linalg.norm(acc)


def test_fw_converges_to_the_cmcg_result_at_the_rate_of_p():
    p, g, st = _setup()
    ref = cmcg.solve(st, p.j_re, p.j_im, tol=1e-12, max_iter=400).filtered
    P = dense.period_map(dense.dense_B(g), st.dt, st.M, st.integrator)
    lam = np.abs(np.linalg.eigvals(P))
    rate = lam[lam < 1 - 1e-8].max()  # |lambda| = 1: static modes, removed by the filter
    assert rate < 0.2  # open cube: transients decay fast
    errs = [_rel(fw.fw_solve(st, p.j_re, p.j_im, l), ref, g) for l in (2, 4, 6)]
    assert errs[-1] < 1e-8
    # no slower than the spectral rate: error(l + 2) <= 2 rate^2 error(l)
    assert all(b <= 2 * rate ** 2 * a for a, b in zip(errs, errs[1:]))


def test_fw_with_zero_periods_filters_the_first_period_from_rest():
    p, g, st = _setup()
    zero = np.zeros((p.nt, 6, p.np_))
    assert np.array_equal(fw.fw_solve(st, p.j_re, p.j_im, 0), filtered_sweep(st, zero, p.j_re, p.j_im))
