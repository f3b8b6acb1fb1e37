"""Nodal P_q reference element (oracle).

The paper discretises with a nodal basis of P_q on each simplex (Section
5.2.2, "expanded in the nodal basis"); its node set is not specified, and the
boundary layout fixes equispaced nodes.  The oracle builds every reference
matrix from an orthonormal Dubiner basis on the bi-unit tetrahedron
(-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1):

* V[i, n]  = psi_n(x_i)           (generalised Vandermonde)
* M        = (V V^T)^{-1}         (mass matrix of the nodal basis)
* D_r      = V_r V^{-1}           (nodal differentiation, likewise D_s, D_t)
* E_f      = face mass of face f, (V_f V_f^T)^{-1} with a 2D Dubiner basis
* LIFT_f   = M^{-1} E_f           (embedded at the face-node rows)

The oracle is test infrastructure: only tests, the smoke check and the CPU
baseline leg of the benchmark may use it.
"""
from __future__ import annotations

from functools import lru_cache
from math import gamma, sqrt

import numpy as np
from scipy.special import eval_jacobi

from paper_2106_02858_gb300.inputs import n_nodes, node_lattice

# Face f is the face opposite vertex f; its vertices in this order.
FACE_VERTS = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def _jacobi_norm2(n: int, a: float, b: float) -> float:
    """Squared L2 norm of the classical Jacobi polynomial P_n^{(a,b)} for weight (1-x)^a (1+x)^b."""
    return 2.0 ** (a + b + 1) / (2 * n + a + b + 1) * gamma(n + a + 1) * gamma(n + b + 1) / (
        gamma(n + a + b + 1) * gamma(n + 1))


def jacobi(n: int, a: float, b: float, x: np.ndarray) -> np.ndarray:
    """Orthonormal Jacobi polynomial of degree n."""
    return eval_jacobi(n, a, b, x) / sqrt(_jacobi_norm2(n, a, b))


def djacobi(n: int, a: float, b: float, x: np.ndarray) -> np.ndarray:
    """Derivative of the orthonormal Jacobi polynomial: d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}."""
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + a + b + 1) * eval_jacobi(n - 1, a + 1, b + 1, x) / sqrt(_jacobi_norm2(n, a, b))


def modes(q: int):
    """Dubiner mode indices (i, j, k), i + j + k <= q."""
    return [(i, j, k) for i in range(q + 1) for j in range(q + 1 - i) for k in range(q + 1 - i - j)]


def collapse(r, s, t):
    """Collapsed coordinates (a, b, c) of the bi-unit tetrahedron; singular edges mapped to -1."""
    a = np.where(np.abs(s + t) > 1e-14, 2.0 * (1.0 + r) / np.where(np.abs(s + t) > 1e-14, -s - t, 1.0) - 1.0, -1.0)
    b = np.where(np.abs(t - 1.0) > 1e-14, 2.0 * (1.0 + s) / np.where(np.abs(t - 1.0) > 1e-14, 1.0 - t, 1.0) - 1.0, -1.0)
    return a, b, t.copy()


def dubiner(r, s, t, i, j, k):
    """psi_ijk = 2 sqrt(2) P_i(a) P_j^{(2i+1,0)}(b) (1-b)^i P_k^{(2i+2j+2,0)}(c) (1-c)^{i+j}; orthonormal on the bi-unit tet."""
    a, b, c = collapse(r, s, t)
    return (2.0 * sqrt(2.0) * jacobi(i, 0, 0, a) * jacobi(j, 2 * i + 1, 0, b) * (1 - b) ** i
            * jacobi(k, 2 * i + 2 * j + 2, 0, c) * (1 - c) ** (i + j))


def grad_dubiner(r, s, t, i, j, k):
    """(d/dr, d/ds, d/dt) of psi_ijk by the chain rule through the collapsed coordinates,
    written with reduced powers so that it is finite at the collapsed edges."""
    a, b, c = collapse(r, s, t)
    C = 2.0 * sqrt(2.0)
    g, dg = jacobi(i, 0, 0, a), djacobi(i, 0, 0, a)
    pj, dpj = jacobi(j, 2 * i + 1, 0, b), djacobi(j, 2 * i + 1, 0, b)
    pk, dpk = jacobi(k, 2 * i + 2 * j + 2, 0, c), djacobi(k, 2 * i + 2 * j + 2, 0, c)
    one_b, one_c = 1.0 - b, 1.0 - c
    # d/dr: only through a, da/dr = 4 / ((1-b)(1-c)).
    if i >= 1:
        ddr = 4.0 * C * dg * pj * one_b ** (i - 1) * pk * one_c ** (i + j - 1)
    else:
        ddr = np.zeros_like(r)
    # d/db of h(b) = P_j(b) (1-b)^i.
    dh = dpj * one_b**i - (i * pj * one_b ** (i - 1) if i >= 1 else 0.0)
    # term through b: g h'(b) k(c) db/ds, with k(c) 2/(1-c) = 2 P_k (1-c)^{i+j-1}.
    if i + j >= 1:
        tb = 2.0 * C * g * dh * pk * one_c ** (i + j - 1)
    else:
        tb = np.zeros_like(r)
    dds = 0.5 * (1 + a) * ddr + tb
    # d/dc of k(c) = P_k(c) (1-c)^{i+j}.
    dk = dpk * one_c ** (i + j) - ((i + j) * pk * one_c ** (i + j - 1) if i + j >= 1 else 0.0)
    ddt = 0.5 * (1 + a) * ddr + 0.5 * (1 + b) * tb + C * g * pj * one_b**i * dk
    return ddr, dds, ddt


def dubiner2d(r, s, i, j):
    """psi_ij = sqrt(2) P_i(a) P_j^{(2i+1,0)}(b) (1-b)^i on the bi-unit triangle (-1,-1),(1,-1),(-1,1)."""
    a = np.where(np.abs(1 - s) > 1e-14, 2.0 * (1 + r) / np.where(np.abs(1 - s) > 1e-14, 1 - s, 1.0) - 1.0, -1.0)
    b = s
    return sqrt(2.0) * jacobi(i, 0, 0, a) * jacobi(j, 2 * i + 1, 0, b) * (1 - b) ** i


class RefElement:
    """All reference matrices of the order-q nodal element."""

    def __init__(self, q: int):
        self.q = q
        self.Np = n_nodes(q)
        self.Nfp = (q + 1) * (q + 2) // 2
        lat = node_lattice(q)  # (Np, 3) ints (i, j, k) -> unit-tet coords (i,j,k)/q
        self.lattice = lat
        l0 = q - lat.sum(axis=1)
        # barycentric coordinates (lambda_0..lambda_3) times q
        self.bary = np.stack([l0, lat[:, 0], lat[:, 1], lat[:, 2]], axis=1)
        x01 = lat.astype(np.float64) / q
        self.r, self.s, self.t = 2 * x01[:, 0] - 1, 2 * x01[:, 1] - 1, 2 * x01[:, 2] - 1

        md = modes(q)
        V = np.stack([dubiner(self.r, self.s, self.t, *m) for m in md], axis=1)
        g = [grad_dubiner(self.r, self.s, self.t, *m) for m in md]
        Vr = np.stack([x[0] for x in g], axis=1)
        Vs = np.stack([x[1] for x in g], axis=1)
        Vt = np.stack([x[2] for x in g], axis=1)
        Vinv = np.linalg.inv(V)
        self.V = V
        self.M = np.linalg.inv(V @ V.T)
        self.Minv = V @ V.T
        self.Dr, self.Ds, self.Dt = Vr @ Vinv, Vs @ Vinv, Vt @ Vinv

        # Face nodes: lambda_f == 0, in increasing volume-node order.
        self.Fmask = np.stack([np.nonzero(self.bary[:, f] == 0)[0] for f in range(4)])  # (4, Nfp)
        # Face mass matrices on the bi-unit reference triangle (area 2).
        self.Mface = []
        md2 = [(i, j) for i in range(q + 1) for j in range(q + 1 - i)]
        for f in range(4):
            A, B, Cc = FACE_VERTS[f]
            lam = self.bary[self.Fmask[f]].astype(np.float64) / q
            r2 = -lam[:, A] + lam[:, B] - lam[:, Cc]
            s2 = -lam[:, A] - lam[:, B] + lam[:, Cc]
            V2 = np.stack([dubiner2d(r2, s2, *m) for m in md2], axis=1)
            self.Mface.append(np.linalg.inv(V2 @ V2.T))
        # LIFT (Np, 4*Nfp): M^{-1} times the face mass placed at the face-node rows.
        E = np.zeros((self.Np, 4 * self.Nfp))
        for f in range(4):
            E[np.ix_(self.Fmask[f], np.arange(f * self.Nfp, (f + 1) * self.Nfp))] = self.Mface[f]
        self.LIFT = self.Minv @ E


@lru_cache(maxsize=None)
def ref_element(q: int) -> RefElement:
    return RefElement(q)
