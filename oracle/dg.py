"""The semi-discrete DG operator (oracle).

Paper: Eq. DG_semidiscrete (Section 5.2.2) for 2D TM, and Eq. ode_system
Phi(t, U) = Re(J e^{i w t}) + B U with a block-diagonal mass matrix.  The
oracle applies the 3D generalisation with the PDE's own sign convention
eps dE/dt + curl H = J, mu dH/dt - curl E = 0 (Eq. maxwell_time_strong), in
strong form on each tetrahedron K with outward normal n:

  dE/dt = eps^{-1} [ J - sigma E - curl H - M^{-1} oint n x (H^ - H^-) ]
  dH/dt = mu^{-1}  [ curl E + M^{-1} oint n x (E^ - E^-) ]

(sigma: the conductivity of Eq. maxwell_time_strong, Section 1, with the coefficients of
Section 3.1; the discrete term (sigma E_h, v_h) of Section 5.2.2, per tetrahedron; 0 unless the
geometry carries one)

with the upwind (Riemann) numerical traces of Section 5.2.2, the paper's
"avg" read as the mean:

  E^ = (Y^- E^- + Y^+ E^+ - (H^- - H^+) x n) / (Y^- + Y^+)
  H^ = (Z^- H^- + Z^+ H^+ + (E^- - E^+) x n) / (Z^- + Z^+),   Z = sqrt(mu/eps), Y = 1/Z

and the boundary traces
  PEC:        E^ = 0,                       H^ = H^- + Y E^- x n
  impedance:  E^ = (E^- - Z H^- x n) / 2,   H^ = (H^- + Y E^- x n) / 2.

Boundary data on impedance faces (the incident-field datum of Section 5.2.2's
impedance traces): the exterior state of the upwind flux is (E^+, H^+) =
(g(t), 0) with Z^+ = Z^-, i.e. the impedance traces gain g / 2 in E^ and
Y n x g / 2 in H^.  An incident field (E_i, H_i) of the boundary medium is
reproduced exactly by g = E_i - Z n x H_i: its traces then coincide with the
interior upwind traces against (E_i, H_i).

The jump signs are the ones that make the scheme dissipative and the
impedance face transparent to outgoing plane waves (the paper's 2D signs are
not consistent with its own PDE).  ``flux="centred"`` drops the jump terms
(test-only, for the energy identity).  ``adjoint=True`` applies Sigma B Sigma
with Sigma = diag(I, -I) (Section 4.1.2: the adjoint propagator is the same
stepper with the sign of the magnetic field changed).

Fields have shape (..., nt, 6, Np): components Ex, Ey, Ez, Hx, Hy, Hz.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from paper_2106_02858_gb300.inputs import INTERIOR, PEC, IMPEDANCE
from .geometry import Geometry
from .refelem import ref_element


def sigma(U: np.ndarray) -> np.ndarray:
    """Sigma = diag(I, -I): flip the sign of the magnetic components."""
    out = U.copy()
    out[..., 3:, :] *= -1.0
    return out


def _curl(F: np.ndarray, geo: Geometry) -> np.ndarray:
    """curl of a nodal vector field F (..., nt, 3, Np) using D_r, D_s, D_t and d r_b / d x_a."""
    R = ref_element(geo.q)
    Fr = F @ R.Dr.T
    Fs = F @ R.Ds.T
    Ft = F @ R.Dt.T
    Fb = np.stack([Fr, Fs, Ft], axis=-3)  # (..., nt, b, comp, Np)
    # dF[..., k, a, c, n] = d F_c / d x_a = sum_b G[k, b, a] d F_c / d r_b
    dF = np.einsum("kba,...kbcn->...kacn", geo.G, Fb)
    return np.stack([dF[..., 1, 2, :] - dF[..., 2, 1, :],
                     dF[..., 2, 0, :] - dF[..., 0, 2, :],
                     dF[..., 0, 1, :] - dF[..., 1, 0, :]], axis=-2)


def _cross(n: np.ndarray, v: np.ndarray) -> np.ndarray:
    """n x v with the vector index on axis -2 (n broadcast over the node axis)."""
    return np.stack([n[..., 1, :] * v[..., 2, :] - n[..., 2, :] * v[..., 1, :],
                     n[..., 2, :] * v[..., 0, :] - n[..., 0, :] * v[..., 2, :],
                     n[..., 0, :] * v[..., 1, :] - n[..., 1, :] * v[..., 0, :]], axis=-2)


def numerical_traces(U: np.ndarray, geo: Geometry, flux: str = "upwind", G=None):
    """Own traces (E^-, H^-) and numerical traces (E^, H^) on every face node.

    G: boundary data (nt, 4, 3, Nfp) at this time, read on impedance faces only (None = 0).
    Returns (n, Em, Hm, Ehat, Hhat), each (..., nt, 4, 3, Nfp) (n without the batch axes)."""
    R = ref_element(geo.q)
    nt = geo.nt
    E, H = U[..., :3, :], U[..., 3:, :]
    Z = np.sqrt(geo.mu / geo.eps)  # (nt,)
    Y = 1.0 / Z
    Fm = R.Fmask  # (4, Nfp)
    Em = E[..., :, Fm].swapaxes(-3, -2)  # (..., nt, 4, 3, Nfp)
    Hm = H[..., :, Fm].swapaxes(-3, -2)
    # neighbour traces through mapP (boundary faces point at themselves and are not used)
    nb = np.where(geo.nbr >= 0, geo.nbr, np.arange(nt)[:, None])  # (nt, 4)
    Ep = np.swapaxes(np.swapaxes(E, -1, -2)[..., nb[:, :, None], geo.mapP, :], -1, -2)
    Hp = np.swapaxes(np.swapaxes(H, -1, -2)[..., nb[:, :, None], geo.mapP, :], -1, -2)
    n = np.broadcast_to(geo.normals[:, :, :, None], (nt, 4, 3, R.Nfp))
    Zm = Z[:, None, None, None]
    Ym = Y[:, None, None, None]
    Zp = Z[nb][:, :, None, None]
    Yp = Y[nb][:, :, None, None]
    interior = (geo.bc == INTERIOR)[:, :, None, None]
    pec = (geo.bc == PEC)[:, :, None, None]
    if flux == "upwind":
        # -(H^- - H^+) x n = n x (H^- - H^+);  (E^- - E^+) x n = -n x (E^- - E^+)
        E_int = (Ym * Em + Yp * Ep + _cross(n, Hm - Hp)) / (Ym + Yp)
        H_int = (Zm * Hm + Zp * Hp - _cross(n, Em - Ep)) / (Zm + Zp)
        E_pec = np.zeros_like(Em)
        H_pec = Hm - Ym * _cross(n, Em)
        E_imp = 0.5 * (Em + Zm * _cross(n, Hm))
        H_imp = 0.5 * (Hm - Ym * _cross(n, Em))
    elif flux == "centred":
        E_int = (Ym * Em + Yp * Ep) / (Ym + Yp)
        H_int = (Zm * Hm + Zp * Hp) / (Zm + Zp)
        E_pec = np.zeros_like(Em)
        H_pec = Hm.copy()
        E_imp = 0.5 * Em
        H_imp = 0.5 * Hm
    else:
        raise ValueError(flux)
    if G is not None:  # exterior state (G, 0) on impedance faces
        E_imp = E_imp + 0.5 * G
        if flux == "upwind":
            H_imp = H_imp + 0.5 * Ym * _cross(n, G)
    Ehat = np.where(interior, E_int, np.where(pec, E_pec, E_imp))
    Hhat = np.where(interior, H_int, np.where(pec, H_pec, H_imp))
    return n, Em, Hm, Ehat, Hhat


def apply_B(U: np.ndarray, geo: Geometry, adjoint: bool = False, flux: str = "upwind", G=None) -> np.ndarray:
    """B U (or Sigma B Sigma U when ``adjoint``), the source-free part of Phi; with boundary data
    G (see numerical_traces) the affine map B U + b(G)."""
    if adjoint:
        return sigma(apply_B(sigma(U), geo, adjoint=False, flux=flux))
    R = ref_element(geo.q)
    E, H = U[..., :3, :], U[..., 3:, :]
    curlE, curlH = _curl(E, geo), _curl(H, geo)
    n, Em, Hm, Ehat, Hhat = numerical_traces(U, geo, flux, G)
    fE = _cross(n, Hhat - Hm)  # n x (H^ - H^-), enters the E equation with a minus sign
    fH = _cross(n, Ehat - Em)  # n x (E^ - E^-), enters the H equation with a plus sign
    scale = (geo.sJ / geo.J[:, None])[:, :, None, None]  # (nt, 4, 1, 1): face Jacobian / volume Jacobian
    # lift: sum_f LIFT_f (Np, Nfp) applied to (..., nt, f, comp, Nfp)
    L = R.LIFT.reshape(R.Np, 4, R.Nfp)
    liftE = np.einsum("nfj,...kfcj->...kcn", L, fE * scale)
    liftH = np.einsum("nfj,...kfcj->...kcn", L, fH * scale)
    out = np.empty_like(U)
    out[..., :3, :] = (-curlH - liftE) / geo.eps[:, None, None]
    if geo.sigma is not None:
        out[..., :3, :] -= (geo.sigma / geo.eps)[:, None, None] * E
    out[..., 3:, :] = (curlE + liftH) / geo.mu[:, None, None]
    return out


def source_term(t: float, omega: float, j_re: np.ndarray, j_im: np.ndarray, geo: Geometry) -> np.ndarray:
    """Re(J e^{i w t}) with J the nodal interpolant of j / eps on the E rows and 0 on the H rows
    (Eq. ode_system)."""
    jr = np.asarray(j_re)
    ji = np.zeros_like(jr) if j_im is None else np.asarray(j_im)
    out = np.zeros(jr.shape[:-3] + (geo.nt, 6, jr.shape[-1]))
    out[..., :3, :] = (jr * np.cos(omega * t) - ji * np.sin(omega * t)) / geo.eps[:, None, None]
    return out


def boundary_data(t: float, omega: float, g_re, g_im) -> np.ndarray:
    """g(t) = Re((g_re + i g_im) e^{i w t}) at the face nodes, (nt, 4, 3, Nfp)."""
    gr = np.asarray(g_re)
    gi = np.zeros_like(gr) if g_im is None else np.asarray(g_im)
    return gr * np.cos(omega * t) - gi * np.sin(omega * t)


def Phi(t: float, U: np.ndarray, geo: Geometry, omega: float, j_re=None, j_im=None, flux: str = "upwind",
        g_re=None, g_im=None) -> np.ndarray:
    """Phi(t, U) = Re(J e^{i w t}) + B U (Eq. ode_system), with the impedance-face data
    Re(g e^{i w t}) in the traces when g_re is given."""
    G = None if g_re is None else boundary_data(t, omega, g_re, g_im)
    out = apply_B(U, geo, flux=flux, G=G)
    if j_re is not None:
        out = out + source_term(t, omega, j_re, j_im, geo)
    return out


def inner(U: np.ndarray, V: np.ndarray, geo: Geometry) -> np.ndarray:
    """(U, V)_{eps,mu} = V^T M U with the block-diagonal mass matrix (Eq. innerproduct)."""
    R = ref_element(geo.q)
    MU = U @ R.M.T  # (..., nt, 6, Np)
    w = np.concatenate([np.repeat(geo.eps[:, None], 3, 1), np.repeat(geo.mu[:, None], 3, 1)], axis=1) * geo.J[:, None]
    return np.einsum("...kcn,...kcn,kc->...", np.conj(V) if np.iscomplexobj(V) else V, MU, w)


def norm(U: np.ndarray, geo: Geometry) -> float:
    return float(np.sqrt(np.real(inner(U, U, geo))))
