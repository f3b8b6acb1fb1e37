"""Pins of the oracle's impedance-face data g (no GPU).

* Exterior state: an impedance face with data g contributes exactly what an interior face
  contributes when the neighbour across it holds the field (E, H) = (g, 0): two tetrahedra
  glued on a face, the second holding a constant (g0, 0), give the first the same B U as the
  first alone with that face an impedance boundary carrying g = g0 (same material both sides).
* Plane wave in a box: with g = E_i - Z n x H_i from an incident plane wave on every
  impedance face, the frequency-domain DG solve reproduces the plane wave, with the error
  falling at least like h^q under refinement (P2, 1 and 2 cubes per side, relative errors
  0.26 and 0.038 at w = pi), and the filtered
  CMCG result reaches the same solution up to the time discretisation.
* Zero data changes nothing, and the data enter the affine map linearly.
"""
import math

import numpy as np

from paper_2106_02858_gb300 import inputs as I
from oracle import cmcg, dense
from oracle.dg import apply_B, inner, Phi
from oracle.geometry import build_geometry
from oracle.refelem import ref_element
from oracle.timestep import Stepper


def _rel(a, b, g):
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


def test_impedance_data_equal_an_exterior_neighbour_state():
    q = 2
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], float)
    # tet 0 and tet 1 share the face (1, 2, 3): face 0 of tet 0 (opposite vertex 0)
    t2 = np.array([[0, 1, 2, 3], [4, 1, 2, 3]], np.int32)
    tags2 = np.array([[0, 2, 2, 2], [0, 2, 2, 2]], np.uint8)
    t1 = t2[:1]
    tags1 = np.array([[2, 2, 2, 2]], np.uint8)
    eps2, mu2 = np.array([2.0, 2.0]), np.array([1.5, 1.5])
    g2 = build_geometry(verts, t2, tags2, eps2, mu2, q)
    g1 = build_geometry(verts, t1, tags1, eps2[:1], mu2[:1], q)
    rng = np.random.default_rng(3)
    Np = ref_element(q).Np
    U2 = np.zeros((2, 6, Np))
    U2[0] = rng.standard_normal((6, Np))
    g0 = np.array([0.3, -1.1, 0.7])
    U2[1, :3, :] = g0[:, None]  # constant exterior state (g0, 0)
    G = np.zeros((1, 4, 3, ref_element(q).Nfp))
    G[0, 0] = g0[:, None]
    ref = apply_B(U2, g2)[0]
    got = apply_B(U2[:1], g1, G=G)[0]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # zero data = no data; data enter linearly
    assert np.array_equal(apply_B(U2[:1], g1, G=0 * G), apply_B(U2[:1], g1))
    b1 = apply_B(np.zeros_like(U2[:1]), g1, G=G)
    b2 = apply_B(np.zeros_like(U2[:1]), g1, G=2 * G)
    assert np.allclose(b2, 2 * b1, rtol=1e-14, atol=0)


def plane_wave_problem(n, q, omega=2 * math.pi, d=(1.0, 2.0, 2.0), pol=(2.0, -1.0, 0.0)):
    """All-impedance cube, eps = mu = 1, no volume source, g from the incident plane wave
    E = p e^{-i w d.x}, H = -d x p e^{-i w d.x} (a solution of i w E = -curl H, i w H = curl E)."""
    mesh = I.kuhn_cube_mesh(n)
    eps, mu = np.ones(mesh.nt), np.ones(mesh.nt)
    geo = build_geometry(mesh.verts, mesh.tets, mesh.tags, eps, mu, q)
    d = np.asarray(d, float) / np.linalg.norm(d)
    p = np.asarray(pol, float)
    p = p - d * (p @ d)
    p /= np.linalg.norm(p)
    dxp = np.cross(d, p)

    def fields(x):  # x (..., 3) -> E, H (..., 3) complex
        ph = np.exp(-1j * omega * (x @ d))[..., None]
        return p * ph, -dxp * ph

    E, H = fields(geo.nodes)  # (nt, Np, 3)
    U = np.concatenate([E.transpose(0, 2, 1), H.transpose(0, 2, 1)], axis=1)  # (nt, 6, Np)
    R = ref_element(q)
    xf = geo.nodes[:, R.Fmask, :]  # (nt, 4, Nfp, 3)
    Ef, Hf = fields(xf)
    nrm = geo.normals[:, :, None, :]  # (nt, 4, 1, 3), Z = 1
    g = (Ef - np.cross(np.broadcast_to(nrm, Hf.shape), Hf)).transpose(0, 1, 3, 2)  # (nt, 4, 3, Nfp)
    return mesh, geo, U, g


def test_plane_wave_in_a_box_frequency_domain_and_cmcg():
    omega = math.pi  # wavelength 2: 1 and 2 P2 cubes per side resolve it coarsely and adequately
    errs = []
    for n in (1, 2):
        mesh, geo, U, g = plane_wave_problem(n, 2, omega)
        zero_j = np.zeros((mesh.nt, 3, U.shape[-1]))
        fs = dense.frequency_solve(geo, omega, zero_j, None, g.real, g.imag)
        errs.append(_rel(fs, U, geo))
    assert errs[1] < 0.05
    assert errs[0] / errs[1] > 2 ** 2  # at least O(h^q)
    # CMCG with the same data reaches the frequency-domain solution up to the time discretisation
    st = Stepper(geo, omega, g_re=g.real, g_im=g.imag)
    res = cmcg.solve(st, zero_j, None, tol=1e-10, max_iter=400)
    assert res.converged
    assert _rel(res.filtered, fs, geo) < 1e-3
    assert _rel(res.filtered, U, geo) < 0.05


def test_source_free_sweeps_ignore_the_data():
    mesh, geo, U, g = plane_wave_problem(1, 1)
    st = Stepper(geo, 2 * math.pi, g_re=g.real, g_im=g.imag)
    plain = Stepper(geo, 2 * math.pi)
    V = np.random.default_rng(0).standard_normal((mesh.nt, 6, 4))
    assert np.array_equal(st.P(V), plain.P(V))
    assert np.array_equal(st.P_star(V), plain.P_star(V))
    # Phi with data at t and without: differ by the data term only
    t = 0.1
    d = Phi(t, V, geo, 2 * math.pi, g_re=g.real, g_im=g.imag) - Phi(t, V, geo, 2 * math.pi)
    G = g.real * math.cos(2 * math.pi * t) - g.imag * math.sin(2 * math.pi * t)
    assert np.allclose(d, apply_B(np.zeros_like(V), geo, G=G), rtol=0, atol=1e-12 * np.abs(d).max())
