"""Explicit time integration and period propagators (oracle).

* Eq. cfl: dt <= c_q min_K sqrt(mu_K eps_K) rho_K.  Section 5.3 prints
  c_1 = 0.24 (RK2 / P1) and c_3 = 0.12 (RK4 / P3), found empirically in 2D; P2
  is unspecified and is read as RK4 with c_2 = 0.12.  On 3D Kuhn meshes the
  printed c_1 is not stable: on the 8^3-cube with a 2x2x2 permittivity block
  partition one period of RK2 at c_1 = 0.24 multiplies the dominant mode by
  about 11 (pinned in tests/test_oracle_time.py), so P1 uses half the printed
  constant, c_1 = 0.12 (PRINTED_CFL keeps the printed values).  dt = T / M with
  M the smallest positive integer satisfying the condition, T = 2 pi / w.
* Algorithm rk2 and Algorithm rk4, literally, on Phi(t, U).
* Section 4.1.2: P_{psi,w} U0 = U(T) with the source, P_w without it, and
  P*_w = Sigma P_w Sigma (same stepper, magnetic sign changed).

Test infrastructure only.
"""
from __future__ import annotations

import math
from typing import Callable, Optional

import numpy as np

from .dg import Phi, apply_B, sigma
from .geometry import Geometry

PRINTED_CFL = {1: 0.24, 3: 0.12}
CFL_CONST = {1: 0.12, 2: 0.12, 3: 0.12}
INTEGRATOR = {1: "rk2", 2: "rk4", 3: "rk4"}


def steps_per_period(geo: Geometry, omega: float, c_q: Optional[float] = None) -> int:
    """M = smallest positive integer with T / M <= c_q min_K sqrt(mu_K eps_K) rho_K."""
    c = CFL_CONST[geo.q] if c_q is None else c_q
    T = 2.0 * math.pi / omega
    dt_max = c * float(np.min(np.sqrt(geo.mu * geo.eps) * geo.rho))
    return max(1, math.ceil(T / dt_max))


def rk2_step(phi: Callable, t: float, U: np.ndarray, dt: float):
    """Algorithm rk2.  Returns (U_{m+1}, K_1)."""
    K1 = phi(t, U)
    K2 = phi(t + dt / 2, U + (dt / 2) * K1)
    return U + dt * K2, K1


def rk4_step(phi: Callable, t: float, U: np.ndarray, dt: float):
    """Algorithm rk4.  Returns (U_{m+1}, K_1)."""
    K1 = phi(t, U)
    K2 = phi(t + dt / 2, U + (dt / 2) * K1)
    K3 = phi(t + dt / 2, U + (dt / 2) * K2)
    K4 = phi(t + dt, U + dt * K3)
    return U + (dt / 6) * (K1 + 2 * K2 + 2 * K3 + K4), K1


class Stepper:
    """The fully discrete scheme of one problem: geometry, w, integrator, M, dt."""

    def __init__(self, geo: Geometry, omega: float, c_q: Optional[float] = None, M: Optional[int] = None,
                 flux: str = "upwind", integrator: Optional[str] = None, g_re=None, g_im=None):
        """g_re, g_im: impedance-face data (nt, 4, 3, Nfp) of the source sweeps (None: none)."""
        self.geo = geo
        self.g_re, self.g_im = g_re, g_im
        self.omega = omega
        self.T = 2.0 * math.pi / omega
        self.M = steps_per_period(geo, omega, c_q) if M is None else M
        self.dt = self.T / self.M
        self.flux = flux
        self.integrator = INTEGRATOR[geo.q] if integrator is None else integrator
        self._step = rk2_step if self.integrator == "rk2" else rk4_step

    def phi(self, j_re=None, j_im=None, adjoint: bool = False) -> Callable:
        if adjoint:
            return lambda t, U: apply_B(U, self.geo, adjoint=True, flux=self.flux)
        if j_re is None:  # source-free sweep: the linear map B (no boundary data either)
            return lambda t, U: Phi(t, U, self.geo, self.omega, None, None, flux=self.flux)
        return lambda t, U: Phi(t, U, self.geo, self.omega, j_re, j_im, flux=self.flux, g_re=self.g_re,
                                g_im=self.g_im)

    def sweep(self, U0: np.ndarray, j_re=None, j_im=None, adjoint: bool = False, callback=None) -> np.ndarray:
        """March M steps from t = 0; ``callback(m, U_m, K1_m)`` sees every step's start state."""
        phi = self.phi(j_re, j_im, adjoint)
        U = np.array(U0, dtype=np.float64, copy=True)
        for m in range(self.M):
            t = m * self.dt
            U_new, K1 = self._step(phi, t, U, self.dt)
            if callback is not None:
                callback(m, U, K1)
            U = U_new
        return U

    # Section 4.1.2
    def P_psi(self, U0, j_re, j_im=None):
        """P_{psi,w} U0: one period with the time-harmonic source."""
        return self.sweep(U0, j_re, j_im)

    def P(self, U0):
        """P_w U0: one period without source (linear)."""
        return self.sweep(U0)

    def P_star(self, WT):
        """P*_w WT = Sigma P_w Sigma WT: back-propagation by the magnetic sign change."""
        return self.sweep(WT, adjoint=True)

    def P_star_via_sigma(self, WT):
        """Same map written literally as Sigma P_w Sigma."""
        return sigma(self.sweep(sigma(WT)))
