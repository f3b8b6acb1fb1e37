"""Several frequencies in one CMCG solve (oracle) -- TEST INFRASTRUCTURE ONLY.

The Conclusion (Section 7) notes that CMCG can compute solutions for several
frequencies "in one shot", at the cost of a single solve.  Reading: with a base
frequency w0, integer harmonics k >= 1 and one current density J_k per harmonic,
the source Re(sum_k J_k e^{i k w0 t}) is periodic with T0 = 2 pi / w0.  Algorithms
init, grad and cmcg (Section 2.2) run unchanged on the period map of T0, and the
filter of Eq. filter taken at the frequency k w0 over T0,

    F_k U = (2 / T0) int_0^T0 U(t) e^{-i k w0 t} dt,

returns the time-harmonic solution of frequency k w0: over a full period T0 the
other harmonics of a T0-periodic solution integrate to zero.  The discrete
filters are those of Section 5.4 (trapezoid for RK2, Hermite for RK4) at the
frequency k w0 with the sweep's dt.  Test infrastructure only.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from .cmcg import CMCGResult, iterate
from .dg import apply_B, source_term
from .filtering import filter_hermite, filter_trapezoid
from .geometry import Geometry
from .timestep import Stepper


class MultiStepper(Stepper):
    """The scheme of one problem driven at the harmonics k w0; sources are stacked (K, nt, 3, Np)."""

    def __init__(self, geo: Geometry, omega0: float, harmonics: Sequence[int], c_q: Optional[float] = None,
                 M: Optional[int] = None):
        super().__init__(geo, omega0, c_q=c_q, M=M)
        self.harmonics = [int(k) for k in harmonics]
        if any(k < 1 for k in self.harmonics):
            raise ValueError("harmonics must be positive integers")

    def phi(self, j_re=None, j_im=None, adjoint: bool = False):
        if adjoint or j_re is None:
            return super().phi(None, None, adjoint)
        jis = [None] * len(self.harmonics) if j_im is None else list(j_im)

        def f(t, U):
            out = apply_B(U, self.geo, flux=self.flux)
            for k, jr, ji in zip(self.harmonics, j_re, jis):
                out = out + source_term(t, k * self.omega, jr, ji, self.geo)
            return out

        return f


def filtered_sweeps(st: MultiStepper, U0, j_re, j_im=None) -> List[np.ndarray]:
    """One sweep of T0 from U0 with every harmonic's source; its filter at each k w0."""
    states, derivs = [], []

    def cb(m, U, K1):
        states.append(U.copy())
        derivs.append(K1.copy())

    UM = st.sweep(U0, j_re, j_im, callback=cb)
    states.append(UM)
    if st.integrator != "rk2":
        derivs.append(st.phi(j_re, j_im)(st.M * st.dt, UM))
    out = []
    for k in st.harmonics:
        w = k * st.omega
        if st.integrator == "rk2":
            out.append(filter_trapezoid(states, w, st.dt, st.T))
        else:
            out.append(filter_hermite(states, derivs, w, st.dt, st.T))
    return out


def solve(st: MultiStepper, j_re, j_im=None, tol: float = 1e-8, max_iter: int = 500) -> List[CMCGResult]:
    """CMCG on the period T0 with the summed source, then one filtered sweep read at every
    harmonic.  Returns one result per harmonic (same U0, iterations and residuals)."""
    zero = np.zeros((st.geo.nt, 6, np.asarray(j_re).shape[-1]))
    G = st.P_psi(zero, j_re, j_im)
    Gstar = G - st.P_star(G)
    U, it, converged, res, funcs, periods = iterate(st, G, Gstar, tol, max_iter)
    Fs = filtered_sweeps(st, U, j_re, j_im)
    return [CMCGResult(U0=U, filtered=F, iters=it, converged=converged, residuals=res, functionals=funcs,
                       periods=periods + 1) for F in Fs]
