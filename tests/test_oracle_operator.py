"""Pins of the oracle's DG operator (no GPU).

* Mesh counts and the inscribed diameter of a Kuhn tetrahedron, rho = h / (1 + sqrt 2).
* Energy: centred flux with PEC walls conserves (U, B U)_M = 0; the upwind
  flux dissipates exactly the face jump terms derived by hand:
    d/dt (1/2)||U||^2 = - sum_int int |[E]_t|^2/(Z-+Z+) + |[H]_t|^2/(Y-+Y+)
                        - sum_PEC int Y |E_t|^2 - sum_imp int (Y|E_t|^2 + Z|H_t|^2)/2.
* Adjoint: (B U, W)_M = (U, Sigma B Sigma W)_M.
* Polynomial exactness: for continuous polynomial fields of degree <= q, B U
  equals (-curl H / eps, curl E / mu) on tetrahedra without boundary faces.
* Transparency: an outgoing plane wave (E tangential, H = -Y n x E) has
  numerical traces equal to its own traces on impedance faces.
* Cavity eigenmode: B applied to the (1,1,0) PEC-cube mode converges to its
  time derivative under refinement.
"""
import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I
from oracle.dg import apply_B, inner, numerical_traces
from oracle.geometry import build_geometry
from oracle.refelem import ref_element


def _geo(n, q, tags="impedance", eps=None, seed=0, removed=None):
    m = I.kuhn_cube_mesh(n, removed=removed)
    if tags == "pec":
        m.tags = np.where(m.tags == I.IMPEDANCE, I.PEC, m.tags).astype(np.uint8)
    rng = np.random.default_rng(seed)
    e = np.ones(m.nt) if eps is None else eps(rng, m)
    return build_geometry(m.verts, m.tets, m.tags, e, np.ones(m.nt), q), m


def test_mesh_counts_and_inradius():
    m = I.kuhn_cube_mesh(4)
    assert m.nt == 384 and int((m.tags == I.IMPEDANCE).sum()) == 192
    g = build_geometry(m.verts, m.tets, m.tags, np.ones(m.nt), np.ones(m.nt), 1)
    assert int((g.nbr >= 0).sum()) == 2 * 672
    assert np.allclose(g.rho, 0.25 / (1 + np.sqrt(2)), rtol=1e-13)
    assert abs(g.volume.sum() - 1.0) < 1e-13
    p = I.scatterer_sphere()
    assert p.nt == 81648
    assert int((p.mesh.tags == I.IMPEDANCE).sum()) == 6912 and int((p.mesh.tags == I.PEC).sum()) == 432


@pytest.mark.parametrize("q", [1, 2, 3])
def test_centred_pec_conserves_energy(q):
    g, m = _geo(2, q, tags="pec", eps=lambda rng, m: rng.uniform(1, 4, m.nt))
    U = I.random_field(np.random.default_rng(1), m.nt, q)
    assert abs(inner(U, apply_B(U, g, flux="centred"), g)) < 1e-13 * inner(U, U, g) * 50


@pytest.mark.parametrize("q", [1, 2])
def test_upwind_dissipation_equals_face_jump_terms(q):
    g, m = _geo(2, q, eps=lambda rng, m: rng.uniform(1, 4, m.nt), removed=None)
    m.tags[0, 3] = I.PEC  # a PEC patch on the impedance boundary, so all three face kinds appear
    g = build_geometry(m.verts, m.tets, m.tags, g.eps, g.mu, q)
    R = ref_element(q)
    U = I.random_field(np.random.default_rng(2), m.nt, q)
    rate = inner(U, apply_B(U, g), g)
    n, Em, Hm, _, _ = numerical_traces(U, g)
    Z = np.sqrt(g.mu / g.eps)
    Y = 1 / Z
    total = 0.0
    for k in range(m.nt):
        for f in range(4):
            nn = g.normals[k, f]
            tang = lambda v: v - np.outer(nn, nn @ v)
            Mf = R.Mface[f] * g.sJ[k, f]
            if g.nbr[k, f] >= 0:
                if g.nbr[k, f] < k:
                    continue  # each interior face once
                kp, fp = g.nbr[k, f], g.nbr_face[k, f]
                Ep = U[kp, :3][:, g.mapP[k, f]]
                Hp = U[kp, 3:][:, g.mapP[k, f]]
                jE = tang(Em[k, f] - Ep)
                jH = tang(Hm[k, f] - Hp)
                total -= sum(jE[c] @ Mf @ jE[c] for c in range(3)) / (Z[k] + Z[kp])
                total -= sum(jH[c] @ Mf @ jH[c] for c in range(3)) / (Y[k] + Y[kp])
            elif g.bc[k, f] == I.PEC:
                Et = tang(Em[k, f])
                total -= Y[k] * sum(Et[c] @ Mf @ Et[c] for c in range(3))
            else:
                Et, Ht = tang(Em[k, f]), tang(Hm[k, f])
                total -= 0.5 * (Y[k] * sum(Et[c] @ Mf @ Et[c] for c in range(3))
                                + Z[k] * sum(Ht[c] @ Mf @ Ht[c] for c in range(3)))
    assert rate < 0
    assert abs(rate - total) < 1e-12 * abs(total)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_operator_adjoint_identity(q):
    g, m = _geo(2, q, eps=lambda rng, m: rng.uniform(1, 4, m.nt))
    rng = np.random.default_rng(3)
    U, W = I.random_field(rng, m.nt, q), I.random_field(rng, m.nt, q)
    a = inner(apply_B(U, g), W, g)
    b = inner(U, apply_B(W, g, adjoint=True), g)
    assert abs(a - b) < 1e-13 * abs(a) * 10


@pytest.mark.parametrize("q", [1, 2, 3])
def test_polynomial_exactness_on_interior_tets(q):
    g, m = _geo(3, q)
    rng = np.random.default_rng(4)
    monos = [(a, b, c) for a in range(q + 1) for b in range(q + 1 - a) for c in range(q + 1 - a - b)]
    coef = rng.standard_normal((6, len(monos)))
    X = g.nodes  # (nt, Np, 3)

    def val(c, x):
        return sum(coef[c, i] * x[..., 0] ** a * x[..., 1] ** b * x[..., 2] ** cc for i, (a, b, cc) in enumerate(monos))

    def d(c, ax, x):
        out = 0.0
        for i, mono in enumerate(monos):
            if mono[ax] == 0:
                continue
            e = list(mono)
            fac = e[ax]
            e[ax] -= 1
            out = out + fac * coef[c, i] * x[..., 0] ** e[0] * x[..., 1] ** e[1] * x[..., 2] ** e[2]
        return out

    U = np.stack([val(c, X) for c in range(6)], axis=1)  # (nt, 6, Np)
    curl = lambda o: np.stack([d(o + 2, 1, X) - d(o + 1, 2, X), d(o + 0, 2, X) - d(o + 2, 0, X),
                               d(o + 1, 0, X) - d(o + 0, 1, X)], axis=1)
    expected = np.concatenate([-curl(3), curl(0)], axis=1)
    BU = apply_B(U, g)
    inner_tets = np.all(g.nbr >= 0, axis=1)
    assert inner_tets.sum() >= 6
    assert np.allclose(BU[inner_tets], expected[inner_tets], atol=1e-10 * np.abs(expected).max())


def test_impedance_face_transparent_to_outgoing_plane_wave():
    g, m = _geo(2, 2)
    rng = np.random.default_rng(5)
    U = np.zeros((m.nt, 6, ref_element(2).Np))
    # per tetrahedron, a constant state that is an outgoing wave through its face 0
    n0 = g.normals[:, 0]
    a = rng.standard_normal((m.nt, 3))
    a -= n0 * np.sum(a * n0, axis=1, keepdims=True)
    H = -np.cross(n0, a)  # Y = 1
    U[:, :3, :] = a[:, :, None]
    U[:, 3:, :] = H[:, :, None]
    n, Em, Hm, Ehat, Hhat = numerical_traces(U, g)
    sm0 = g.bc[:, 0] == I.IMPEDANCE
    assert sm0.sum() > 0
    assert np.allclose(Ehat[sm0, 0], Em[sm0, 0], atol=1e-14)
    assert np.allclose(Hhat[sm0, 0], Hm[sm0, 0], atol=1e-14)
    # an incoming wave (H = +Y n x E) is not passed through
    U[:, 3:, :] = -H[:, :, None]
    _, Em, Hm, Ehat, Hhat = numerical_traces(U, g)
    assert not np.allclose(Hhat[sm0, 0], Hm[sm0, 0], atol=1e-3)


def _cavity_mode(X, t):
    w = np.pi * np.sqrt(2)
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    E = np.stack([0 * x, 0 * x, np.sin(np.pi * x) * np.sin(np.pi * y) * np.cos(w * t)], axis=1)
    H = (np.pi / w) * np.stack([np.sin(np.pi * x) * np.cos(np.pi * y), -np.cos(np.pi * x) * np.sin(np.pi * y), 0 * x],
                               axis=1) * np.sin(w * t)
    dE = np.stack([0 * x, 0 * x, -w * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(w * t)], axis=1)
    dH = np.pi * np.stack([np.sin(np.pi * x) * np.cos(np.pi * y), -np.cos(np.pi * x) * np.sin(np.pi * y), 0 * x],
                          axis=1) * np.cos(w * t)
    return np.concatenate([E, H], axis=1), np.concatenate([dE, dH], axis=1)


@pytest.mark.parametrize("q", [1, 2])
def test_cavity_eigenmode_consistency_converges(q):
    errs = []
    for n in (2, 4):
        g, m = _geo(n, q, tags="pec")
        U, dU = _cavity_mode(g.nodes, 0.3)
        r = apply_B(U, g) - dU
        errs.append(np.sqrt(inner(r, r, g) / inner(dU, dU, g)))
    assert errs[0] / errs[1] > 0.8 * 2.0**q  # O(h^q) consistency in the energy norm
