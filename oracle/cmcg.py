"""The controllability method with conjugate gradients (oracle).

Section 2.2, Algorithms init, grad and cmcg, with the readings:

* Algorithm grad: J'(U0) = (I - P*)(I - P) U0 - G*  (Eq. functional_gradient;
  the printed "W_T - U_0 - G*" is read as W_0 - W_T - G*).
* Algorithm cmcg is run in residual form R = -J' (with R = +J' the printed
  update U += alpha D would ascend), and the new direction uses the new
  residual, D^{l+1} = R^{l+1} + beta D^l, as in textbook CG (Section 5.1 cites
  Ciarlet, Section 8.5).
* The initial guess is U0 = 0 (Section 6), so R^0 = G* needs no sweep.
* Inner products and norms are the (eps, mu)-weighted L2 ones, V^T M U.

Test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .dg import inner, norm
from .filtering import filtered_sweep
from .timestep import Stepper


@dataclass
class CMCGResult:
    U0: np.ndarray
    filtered: np.ndarray  # complex (nt, 6, Np): e on rows 0..2, h on rows 3..5
    iters: int
    converged: bool
    residuals: List[float] = field(default_factory=list)  # ||R^l|| / ||R^0||
    functionals: List[float] = field(default_factory=list)  # J(U0^l)
    periods: int = 0


def initialise(st: Stepper, j_re, j_im=None):
    """Algorithm init: G = P_{psi,w} 0; G_T = P*_w G; G* = G - G_T."""
    zero = np.zeros(j_re.shape[:-3] + (st.geo.nt, 6, j_re.shape[-1]))
    G = st.P_psi(zero, j_re, j_im)
    GT = st.P_star(G)
    return G, G - GT


def gradient(st: Stepper, U0, Gstar):
    """Algorithm grad: U_T = P U0; W_T = U_T - U0; W_0 = P* W_T; J' = W_0 - W_T - G*."""
    UT = st.P(U0)
    WT = UT - U0
    W0 = st.P_star(WT)
    return W0 - WT - Gstar


def functional(st: Stepper, U0, G) -> float:
    """J(U0) = 1/2 ||(I - P) U0 - G||^2 (Eq. energy_functional_linear)."""
    r = U0 - st.P(U0) - G
    return 0.5 * norm(r, st.geo) ** 2


def solve(st: Stepper, j_re, j_im=None, tol: float = 1e-8, max_iter: int = 500, track_functional: bool = False,
          U0: Optional[np.ndarray] = None) -> CMCGResult:
    G, Gstar = initialise(st, j_re, j_im)
    U, it, converged, res, funcs, periods = iterate(st, G, Gstar, tol, max_iter, track_functional, U0)
    F = filtered_sweep(st, U, j_re, j_im)
    periods += 1
    return CMCGResult(U0=U, filtered=F, iters=it, converged=converged, residuals=res, functionals=funcs,
                      periods=periods)


def iterate(st: Stepper, G, Gstar, tol: float, max_iter: int, track_functional: bool = False,
            U0: Optional[np.ndarray] = None):
    """Algorithm cmcg in residual form from the data G, G* of Algorithm init.  Returns
    (U0, iterations, converged, relative residuals, functionals, periods simulated so far)."""
    geo = st.geo
    periods = 2
    if U0 is None:
        U = np.zeros_like(Gstar)
        R = Gstar.copy()
    else:
        U = np.array(U0, dtype=np.float64, copy=True)
        R = -gradient(st, U, Gstar)
        periods += 2
    D = R.copy()
    rr = float(inner(R, R, geo))
    r0 = np.sqrt(rr)
    res, funcs = [1.0], []
    if track_functional:
        funcs.append(functional(st, U, G))
    it = 0
    converged = r0 == 0.0
    while it < max_iter and not converged:
        if np.sqrt(rr) <= tol * r0:
            converged = True
            break
        # A = J'(D) + G* = (I - P*)(I - P) D
        WT = st.P(D) - D
        A = st.P_star(WT) - WT
        periods += 2
        alpha = rr / float(inner(D, A, geo))
        U = U + alpha * D
        R = R - alpha * A
        rr_new = float(inner(R, R, geo))
        beta = rr_new / rr
        D = R + beta * D
        rr = rr_new
        it += 1
        res.append(np.sqrt(rr) / r0)
        if track_functional:
            funcs.append(functional(st, U, G))
    if not converged and np.sqrt(rr) <= tol * r0:
        converged = True
    return U, it, converged, res, funcs, periods
