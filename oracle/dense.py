"""Brute-force dense linear algebra on tiny meshes (oracle).

* B assembled column by column from the operator (Eq. ode_system).
* The block-diagonal mass matrix M.
* The RK amplification matrices R(dt B) (Algorithms rk2 / rk4 applied to
  dU/dt = B U) and the dense period map P = R^M.
* The frequency-domain DG solve of Section 6, (i w M + K) U = M J, written with
  B = -M^{-1} K as (i w I - B) U = J.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .dg import apply_B, source_term
from .refelem import ref_element


def dense_B(geo, adjoint: bool = False, flux: str = "upwind") -> np.ndarray:
    Np = ref_element(geo.q).Np
    n = geo.nt * 6 * Np
    I = np.eye(n).reshape(n, geo.nt, 6, Np)
    cols = apply_B(I, geo, adjoint=adjoint, flux=flux).reshape(n, n)
    return cols.T  # column c is B e_c


def dense_M(geo) -> np.ndarray:
    R = ref_element(geo.q)
    blocks = []
    for k in range(geo.nt):
        for c in range(6):
            w = geo.eps[k] if c < 3 else geo.mu[k]
            blocks.append(geo.J[k] * w * R.M)
    n = len(blocks) * R.Np
    out = np.zeros((n, n))
    for b, blk in enumerate(blocks):
        s = slice(b * R.Np, (b + 1) * R.Np)
        out[s, s] = blk
    return out


def amplification(B: np.ndarray, dt: float, integrator: str) -> np.ndarray:
    """R(dt B) = sum_{k <= s} (dt B)^k / k!  (s = 2 for RK2, 4 for RK4)."""
    s = 2 if integrator == "rk2" else 4
    n = B.shape[0]
    out = np.eye(n)
    term = np.eye(n)
    for k in range(1, s + 1):
        term = term @ (dt * B) / k
        out = out + term
    return out


def period_map(B: np.ndarray, dt: float, M: int, integrator: str) -> np.ndarray:
    return np.linalg.matrix_power(amplification(B, dt, integrator), M)


def frequency_solve(geo, omega: float, j_re, j_im=None, g_re=None, g_im=None) -> np.ndarray:
    """FS: (i w I - B) U = J + b with J = (j_re + i j_im)/eps on the E rows and b the
    (complex) boundary-data term of g = g_re + i g_im on impedance faces."""
    B = dense_B(geo)
    Jr = source_term(0.0, omega, j_re, j_im, geo)  # Re part of J at t = 0 is j_re / eps
    Ji = -source_term(np.pi / (2 * omega), omega, j_re, j_im, geo) if j_im is not None else np.zeros_like(Jr)
    # at t = pi/(2w): Re(J e^{i pi/2}) = -Im J  ->  Im J = -source_term(...)
    if g_re is not None:  # b(g) = B_g(0, g) is linear in g: real and imaginary parts separately
        zero = np.zeros_like(Jr)
        Jr = Jr + apply_B(zero, geo, G=np.asarray(g_re))
        if g_im is not None:
            Ji = Ji + apply_B(zero, geo, G=np.asarray(g_im))
    J = (Jr + 1j * Ji).reshape(-1)
    n = B.shape[0]
    U = np.linalg.solve(1j * omega * np.eye(n) - B, J)
    return U.reshape(Jr.shape)
