"""Discrete filters F_w (oracle).

Eq. filter defines F_w U = (2/T) int_0^T U(t) e^{-i w t} dt.  Section 5.4 gives
two quadratures; both omit the 2/T factor, which the oracle restores (the
continuous definition fixes it):

* Eq. filtering_RK2 (trapezoid, used with RK2):
    F ~ (2/T) (dt/2) sum_{m=1}^{M} (U_{m-1} e^{-i w t_{m-1}} + U_m e^{-i w t_m})
* Eq. filtering_RK4 (cubic Hermite interpolation, used with RK4): on
  [t_{m-1}, t_m] with s = (t - t_{m-1}) / dt, the Hermite cubics are
    p00 = 1 - 3 s^2 + 2 s^3,   p01 = 3 s^2 - 2 s^3,
    p10 = dt (s - 2 s^2 + s^3), p11 = dt (s^3 - s^2)
  (first index: derivative order, second: node t_{m-1} / t_m) and
    xi_ij = int_{t_{m-1}}^{t_m} p_ij(t) e^{-i w t} dt
          = dt e^{-i w t_{m-1}} int_0^1 p_ij(s) e^{-i theta s} ds,  theta = w dt,
  with Phi_m = Phi(t_m, U_m) as the derivative data.

The moments I_k(theta) = int_0^1 s^k e^{-i theta s} ds come from their power
series for small theta and from integration by parts otherwise.  Test
infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np


def moments(theta: float, kmax: int = 3) -> np.ndarray:
    """I_k = int_0^1 s^k e^{-i theta s} ds.

    For theta < 2: the power series sum_n (-i theta)^n / (n! (n + k + 1)) (no
    cancellation).  For theta >= 2: integration by parts,
    I_0 = (1 - e^{-i theta}) / (i theta),  I_k = (k I_{k-1} - e^{-i theta}) / (i theta)."""
    out = np.zeros(kmax + 1, dtype=np.complex128)
    if theta >= 2.0:
        e = np.exp(-1j * theta)
        out[0] = (1 - e) / (1j * theta)
        for k in range(1, kmax + 1):
            out[k] = (k * out[k - 1] - e) / (1j * theta)
        return out
    for k in range(kmax + 1):
        term_n = 1.0 + 0j  # (-i theta)^n / n!
        total = 0j
        n = 0
        while True:
            total += term_n / (n + k + 1)
            n += 1
            term_n *= (-1j * theta) / n
            if abs(term_n) < 1e-20 and n > 2:
                break
        out[k] = total
    return out


def hermite_weights(omega: float, dt: float, t_prev: float):
    """(xi00, xi01, xi10, xi11) on the interval [t_prev, t_prev + dt]."""
    I = moments(omega * dt)
    e = dt * np.exp(-1j * omega * t_prev)
    xi00 = e * (I[0] - 3 * I[2] + 2 * I[3])
    xi01 = e * (3 * I[2] - 2 * I[3])
    xi10 = dt * e * (I[1] - 2 * I[2] + I[3])
    xi11 = dt * e * (I[3] - I[2])
    return xi00, xi01, xi10, xi11


def filter_trapezoid(states, omega: float, dt: float, T: float) -> np.ndarray:
    """Eq. filtering_RK2 times 2/T; ``states`` = [U_0, ..., U_M]."""
    acc = 0j
    for m in range(1, len(states)):
        acc = acc + (dt / 2) * (states[m - 1] * np.exp(-1j * omega * (m - 1) * dt)
                                + states[m] * np.exp(-1j * omega * m * dt))
    return (2.0 / T) * acc


def filter_hermite(states, derivs, omega: float, dt: float, T: float) -> np.ndarray:
    """Eq. filtering_RK4 times 2/T; ``states`` = [U_0..U_M], ``derivs`` = [Phi_0..Phi_M]."""
    acc = 0j
    for m in range(1, len(states)):
        xi00, xi01, xi10, xi11 = hermite_weights(omega, dt, (m - 1) * dt)
        acc = acc + states[m - 1] * xi00 + states[m] * xi01 + derivs[m - 1] * xi10 + derivs[m] * xi11
    return (2.0 / T) * acc


def filtered_sweep(stepper, U0, j_re=None, j_im=None) -> np.ndarray:
    """F_{psi,w} U0: one source sweep from U0, filtered (trapezoid for RK2, Hermite for RK4).

    Returns a complex field of shape U0.shape."""
    states, derivs = [], []

    def cb(m, U, K1):
        states.append(U.copy())
        derivs.append(K1.copy())

    UM = stepper.sweep(U0, j_re, j_im, callback=cb)
    states.append(UM)
    if stepper.integrator == "rk2":
        return filter_trapezoid(states, stepper.omega, stepper.dt, stepper.T)
    derivs.append(stepper.phi(j_re, j_im)(stepper.M * stepper.dt, UM))
    return filter_hermite(states, derivs, stepper.omega, stepper.dt, stepper.T)
