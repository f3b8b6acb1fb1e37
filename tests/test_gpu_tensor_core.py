"""The tensor-core stage form (stage_variant 7) against the FP64 oracle (GPU).

The volume derivatives D_b F and the lift LIFT . f of the DG operator (Section
5.2.2, Eq. DG_semidiscrete / Eq. ode_system) run as tcgen05 MMAs with three
TF32 products per FP32 product and FP32 accumulation; the fluxes, the chain
rule and the curl stay on the CUDA cores.  Splitting each FP32 value into two
rounded TF32 parts represents it to about 2^-22 relative, so the form keeps the
FP32 tolerances of the other forms: operator and period sweeps 1e-5, filtered
sweeps and converged solves 1e-4 (relative (eps, mu)-weighted L2).

Cases span one tetrahedron, ragged tiles (a CTA covers 64 tetrahedra, two
tiles, of which the last may not exist), PEC and impedance faces, a distorted
mesh, permittivity jumps, all three orders, source stages (nested RK form with
the source combined per stage, source rows prefetched) with the on-the-fly
filter, and a batch whose problems meet inside one CTA.
"""
import math

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TC_FORMS = [7]  # stage_variant of the tensor-core form


@pytest.fixture(scope="module")
def lib():
    from paper_2106_02858_gb300 import build
    build.build()
    from paper_2106_02858_gb300 import cmcg
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return cmcg


def _geo(p):
    from oracle.geometry import build_geometry
    return build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)


def _rel(a, b, g):
    from oracle.dg import inner
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


def _problem(kind, q, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "cube3":
        return I.cube_problem(3, q, 4 * math.pi, (0.4, 0.5, 0.6), (0.2, 1.0, -0.3), 0.2,
                              eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.5, 1.0))
    if kind == "scatterer8":
        return I.cube_problem(8, q, 4 * math.pi, (0.2, 0.3, 0.7), (1.0, 0.0, 0.5), 0.15, removed=(3, 5),
                              eps_fn=lambda c: np.where(np.linalg.norm(c - 0.25, axis=1) < 0.2, 4.0, 1.0))
    if kind == "distorted":
        p = I.cube_problem(3, q, 2 * math.pi, (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 0.3)
        v = p.mesh.verts.copy()
        inner = np.all((v > 1e-9) & (v < 1 - 1e-9), axis=1)
        v[inner] += rng.uniform(-0.04, 0.04, (inner.sum(), 3))
        p.mesh.verts = v
        nodes = I.physical_nodes(v, p.mesh.tets, q)
        p.j_re = I.gaussian_current(nodes, (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 0.3)
        p.j_im = 0.3 * p.j_re
        return p
    if kind == "single":
        verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
        mesh = I.Mesh(verts=verts, tets=np.array([[0, 1, 2, 3]], np.int32),
                      tags=np.array([[2, 1, 2, 1]], np.uint8), h=1.0)
        nodes = I.physical_nodes(verts, mesh.tets, q)
        jr = I.gaussian_current(nodes, (0.2, 0.2, 0.2), (1, 1, 0), 0.5)
        return I.Problem("single", mesh, np.array([2.0]), np.array([1.5]), 2 * math.pi, q, jr, np.zeros_like(jr), 1e-8)
    if kind == "cube4":  # the 384-tet cube of the batched-source workload
        return I.cube_problem(4, q, 4 * math.pi, (0.5, 0.5, 0.5), (1.0, 0.0, 0.0), 0.1)
    raise ValueError(kind)


CASES = [("single", 1), ("single", 3), ("cube3", 1), ("cube3", 2), ("cube3", 3), ("scatterer8", 1),
         ("scatterer8", 2), ("scatterer8", 3), ("distorted", 2), ("distorted", 3), ("cube4", 3)]


@pytest.mark.parametrize("TC", TC_FORMS)
@pytest.mark.parametrize("kind,q", CASES)
def test_tensor_core_operator_matches_oracle(lib, kind, q, TC):
    from oracle.dg import Phi, apply_B
    p = _problem(kind, q)
    g = _geo(p)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP32, stage_variant=TC)
    assert lib.cmcg_get_tuning(h)[0] == TC - 1
    U = I.random_field(np.random.default_rng(7), p.nt, q)
    t = 0.37 * (2 * math.pi / p.omega)
    assert _rel(lib.dgtd_apply(h, t, U, p.j_re, p.j_im), Phi(t, U, g, p.omega, p.j_re, p.j_im), g) < 1e-5
    assert _rel(lib.dgtd_apply(h, 0.0, U, adjoint=True), apply_B(U, g, adjoint=True), g) < 1e-5
    h.close()


@pytest.mark.parametrize("kind,q", [("single", 2), ("cube3", 1), ("cube3", 3), ("scatterer8", 2),
                                    ("distorted", 3), ("cube4", 3)])
@pytest.mark.parametrize("TC", TC_FORMS)
def test_tensor_core_sweeps_match_oracle(lib, kind, q, TC):
    from oracle.timestep import Stepper
    from oracle.filtering import filtered_sweep
    p = _problem(kind, q)
    g = _geo(p)
    st = Stepper(g, p.omega)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP32, stage_variant=TC)
    rng = np.random.default_rng(11)
    U, W = I.random_field(rng, p.nt, q), I.random_field(rng, p.nt, q)
    assert _rel(lib.dgtd_period_forward(h, U), st.P(U), g) < 1e-5
    assert _rel(lib.dgtd_period_adjoint(h, W), st.P_star(W), g) < 1e-5
    uT, fr, fi = lib.dgtd_period_forward(h, U, p.j_re, p.j_im, filtered=True)
    assert _rel(uT, st.P_psi(U, p.j_re, p.j_im), g) < 1e-5
    assert _rel(fr + 1j * fi, filtered_sweep(st, U, p.j_re, p.j_im), g) < 1e-4
    h.close()


@pytest.mark.parametrize("TC", TC_FORMS)
def test_tensor_core_full_size_scatterer_operator(lib, TC):
    """The 81,648-tet P2 scatterer: one operator application of the tensor-core form vs the oracle."""
    from oracle.dg import Phi
    p = I.scatterer_sphere()
    g = _geo(p)
    U = I.random_field(np.random.default_rng(1), p.nt, 2)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP32, stage_variant=TC)
    assert _rel(lib.dgtd_apply(h, 0.1, U, p.j_re, p.j_im), Phi(0.1, U, g, p.omega, p.j_re, p.j_im), g) < 1e-5
    h.close()


@pytest.mark.parametrize("TC", TC_FORMS)
def test_tensor_core_cmcg_converged_matches_oracle(lib, TC):
    from oracle import cmcg as ocmcg
    from oracle.timestep import Stepper
    p = _problem("cube3", 3)
    g = _geo(p)
    ref = ocmcg.solve(Stepper(g, p.omega), p.j_re, p.j_im, tol=1e-8, max_iter=500)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP32, stage_variant=TC)
    e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, tol=1e-5, max_iter=500)
    h.close()
    assert info.status == lib.CMCG_OK
    assert _rel(np.concatenate([e, hh], axis=1), ref.filtered, g) < 1e-4


@pytest.mark.parametrize("TC", TC_FORMS)
def test_tensor_core_batch_alone_vs_in_the_mix(lib, TC):
    """Problems of 162 and 48 tetrahedra (ragged tiles) share CTAs in one handle: each problem's
    result equals its solve alone with the same form (the rows of an MMA are independent)."""
    rng = np.random.default_rng(3)
    probs = []
    for n, omega in ((3, 4 * math.pi), (2, 2 * math.pi), (3, 8 * math.pi)):
        probs.append(I.cube_problem(n, 3, omega, rng.uniform(0.3, 0.7, 3), I.unit_vector(rng), 0.2, tol=1e-6))
    meshes = [lib.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags) for p in probs]
    opt = lib.cmcg_default_options(order=3, precision=lib.CMCG_FP32, stage_variant=TC)
    h = lib.cmcg_create_batch([(m, p.eps, p.mu, p.omega) for m, p in zip(meshes, probs)], opt)
    eb, hb, infos = lib.cmcg_solve_batch(h, [p.j_re for p in probs], [p.j_im for p in probs], 1e-6, 400)
    h.close()
    for k, p in enumerate(probs):
        ha, _ = lib.create_for_problem(p, precision=lib.CMCG_FP32, stage_variant=TC)
        ea, hha, ia = lib.cmcg_solve(ha, p.j_re, p.j_im, 1e-6, 400)
        ha.close()
        assert ia.iters == infos[k].iters
        scale = np.abs(np.concatenate([ea, hha], 1)).max()
        assert np.abs(eb[k] - ea).max() <= 1e-13 * scale
        assert np.abs(hb[k] - hha).max() <= 1e-13 * scale
