"""Pins of the oracle's reference element against closed forms (no GPU).

* D_r, D_s, D_t differentiate every polynomial of degree <= q exactly.
* The mass matrix integrates products of monomials exactly:
  int over the unit tet of x^a y^b z^c = a! b! c! / (a + b + c + 3)!.
* The face mass matrices integrate barycentric monomials exactly:
  int over a triangle of area A of l1^a l2^b l3^c = a! b! c! 2A / (a + b + c + 2)!.
* Integration by parts (divergence theorem) ties M, D and the face masses.
"""
from math import factorial

import numpy as np
import pytest

from oracle.refelem import FACE_VERTS, ref_element


def _monos(q):
    return [(a, b, c) for a in range(q + 1) for b in range(q + 1 - a) for c in range(q + 1 - a - b)]


@pytest.mark.parametrize("q", [1, 2, 3])
def test_derivative_matrices_exact_on_polynomials(q):
    R = ref_element(q)
    for a, b, c in _monos(q):
        f = R.r**a * R.s**b * R.t**c
        dr = a * R.r ** max(a - 1, 0) * R.s**b * R.t**c
        ds = b * R.r**a * R.s ** max(b - 1, 0) * R.t**c
        dt = c * R.r**a * R.s**b * R.t ** max(c - 1, 0)
        assert np.allclose(R.Dr @ f, dr, atol=1e-12)
        assert np.allclose(R.Ds @ f, ds, atol=1e-12)
        assert np.allclose(R.Dt @ f, dt, atol=1e-12)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_mass_matrix_exact_monomial_integrals(q):
    R = ref_element(q)
    x, y, z = (R.r + 1) / 2, (R.s + 1) / 2, (R.t + 1) / 2  # unit-tet coordinates of the nodes
    for m1 in _monos(q):
        for m2 in _monos(q):
            p = x ** m1[0] * y ** m1[1] * z ** m1[2]
            r = x ** m2[0] * y ** m2[1] * z ** m2[2]
            a, b, c = m1[0] + m2[0], m1[1] + m2[1], m1[2] + m2[2]
            exact = 8.0 * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)  # bi-unit = 8 x unit
            assert abs(p @ R.M @ r - exact) < 1e-13


@pytest.mark.parametrize("q", [1, 2, 3])
def test_face_mass_exact_barycentric_integrals(q):
    R = ref_element(q)
    for f in range(4):
        lam = R.bary[R.Fmask[f]].astype(float) / q  # (Nfp, 4)
        A, B, C = FACE_VERTS[f]
        mon = [(a, b, c) for a in range(q + 1) for b in range(q + 1 - a) for c in range(q + 1 - a - b) if a + b + c == q]
        for m1 in mon:
            for m2 in mon:
                p = lam[:, A] ** m1[0] * lam[:, B] ** m1[1] * lam[:, C] ** m1[2]
                r = lam[:, A] ** m2[0] * lam[:, B] ** m2[1] * lam[:, C] ** m2[2]
                a, b, c = m1[0] + m2[0], m1[1] + m2[1], m1[2] + m2[2]
                exact = factorial(a) * factorial(b) * factorial(c) * 2 * 2.0 / factorial(a + b + c + 2)
                assert abs(p @ R.Mface[f] @ r - exact) < 1e-13


@pytest.mark.parametrize("q", [1, 2, 3])
def test_integration_by_parts_links_mass_derivative_and_lift(q):
    """M D + (M D)^T = sum_f n_f (|F_f| / 2) E_f  for each reference direction (bi-unit tet)."""
    R = ref_element(q)
    verts = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    Ef = []
    nrm = []
    for f in range(4):
        a, b, c = FACE_VERTS[f]
        cr = np.cross(verts[b] - verts[a], verts[c] - verts[a])
        if np.dot(cr, verts[f] - verts[a]) > 0:
            cr = -cr
        area = 0.5 * np.linalg.norm(cr)
        nrm.append((cr / np.linalg.norm(cr), area))
        E = np.zeros((R.Np, R.Np))
        E[np.ix_(R.Fmask[f], R.Fmask[f])] = (R.M @ R.LIFT[:, f * R.Nfp:(f + 1) * R.Nfp])[R.Fmask[f]]
        Ef.append(E)
    for d, D in enumerate((R.Dr, R.Ds, R.Dt)):
        lhs = R.M @ D + (R.M @ D).T
        rhs = sum(nrm[f][0][d] * nrm[f][1] / 2.0 * Ef[f] for f in range(4))
        assert np.allclose(lhs, rhs, atol=1e-12)
