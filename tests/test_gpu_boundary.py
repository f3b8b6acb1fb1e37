"""Impedance-face data g on the GPU (through the C ABI) against the FP64 oracle.

The plane wave in an all-impedance box (eps = mu = 1, no volume source, g from the incident
plane wave; see test_oracle_boundary) on 2 and 3 cubes per side:
* one source period from a random state: FP64 1e-12, FP32 1e-5 (as the other sweeps);
* the converged CMCG solve: FP64 1e-9 with the oracle's iteration count, FP32 within 1e-4 of
  FP64, and both within the discretisation error of the exact plane wave;
* a batch holding the plane-wave problem with data and a cube problem without: each result
  equals the same problem solved alone (1e-13, same kernel form);
* clearing the data gives back the handle's results without data, bit for bit.
"""
import math

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I
from test_oracle_boundary import plane_wave_problem

pytestmark = pytest.mark.gpu
OMEGA = math.pi


@pytest.fixture(scope="module")
def lib():
    from paper_2106_02858_gb300 import build
    build.build()
    from paper_2106_02858_gb300 import cmcg
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return cmcg


def _rel(a, b, g):
    from oracle.dg import inner
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


def _handle(lib, mesh, q, precision, form=0):
    m = lib.make_mesh(mesh.verts, mesh.tets, mesh.tags)
    opt = lib.cmcg_default_options(order=q, precision=precision, stage_variant=form)
    return lib.cmcg_create(m, np.ones(mesh.nt), np.ones(mesh.nt), OMEGA, opt), m


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("q", [1, 2])
def test_source_period_with_boundary_data_matches_oracle(lib, prec, q):
    from oracle.timestep import Stepper
    mesh, geo, U, g = plane_wave_problem(3, q, OMEGA)
    P = lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32
    h, _m = _handle(lib, mesh, q, P)
    lib.cmcg_set_boundary_data(h, g.real, g.imag)
    zero_j = np.zeros((mesh.nt, 3, U.shape[-1]))
    V = I.random_field(np.random.default_rng(4), mesh.nt, q)
    st = Stepper(geo, OMEGA, g_re=g.real, g_im=g.imag)
    ref = st.P_psi(V, zero_j)
    got = lib.dgtd_period_forward(h, V, zero_j, None)
    assert _rel(got, ref, geo) < (1e-12 if prec == "fp64" else 1e-5)
    h.close()


def test_plane_wave_cmcg_matches_oracle_and_exact_solution(lib):
    from oracle import cmcg as ocmcg
    from oracle.timestep import Stepper
    q = 2
    mesh, geo, U, g = plane_wave_problem(2, q, OMEGA)
    zero_j = np.zeros((mesh.nt, 3, U.shape[-1]))
    st = Stepper(geo, OMEGA, g_re=g.real, g_im=g.imag)
    ref = ocmcg.solve(st, zero_j, None, tol=1e-9, max_iter=400)
    out = {}
    for prec in ("fp64", "fp32"):
        h, _m = _handle(lib, mesh, q, lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32)
        lib.cmcg_set_boundary_data(h, g.real, g.imag)
        e, hh, info = lib.cmcg_solve(h, zero_j, None, 1e-9 if prec == "fp64" else 1e-5, 400)
        assert info.status == lib.CMCG_OK
        out[prec] = (np.concatenate([e, hh], axis=1), info)
        h.close()
    assert out["fp64"][1].iters == ref.iters
    assert _rel(out["fp64"][0], ref.filtered, geo) < 1e-9
    assert _rel(out["fp32"][0], out["fp64"][0], geo) < 1e-4
    assert _rel(out["fp64"][0], U, geo) < 0.05  # discretisation error of the plane wave (0.038 in FS)


def test_boundary_data_alone_vs_in_a_batch_and_cleared(lib):
    q = 2
    mesh, geo, U, g = plane_wave_problem(2, q, OMEGA)
    other = I.cube_problem(3, q, OMEGA, (0.5, 0.4, 0.6), (1.0, 0.0, 0.0), 0.2, tol=1e-6)
    zero_j = np.zeros((mesh.nt, 3, U.shape[-1]))
    form = 2
    m1 = lib.make_mesh(mesh.verts, mesh.tets, mesh.tags)
    m2 = lib.make_mesh(other.mesh.verts, other.mesh.tets, other.mesh.tags)
    opt = lib.cmcg_default_options(order=q, precision=lib.CMCG_FP64, stage_variant=form)
    hb = lib.cmcg_create_batch([(m1, np.ones(mesh.nt), np.ones(mesh.nt), OMEGA),
                                (m2, other.eps, other.mu, other.omega)], opt)
    lib.cmcg_set_boundary_data(hb, g.real, g.imag, problem=0)
    eb, hhb, ib = lib.cmcg_solve_batch(hb, [zero_j, other.j_re], [None, other.j_im], 1e-8, 400)
    hb.close()
    h1, _a = _handle(lib, mesh, q, lib.CMCG_FP64, form)
    lib.cmcg_set_boundary_data(h1, g.real, g.imag)
    e1, hh1, i1 = lib.cmcg_solve(h1, zero_j, None, 1e-8, 400)
    assert i1.iters == ib[0].iters
    s = np.abs(np.concatenate([e1, hh1], 1)).max()
    assert np.abs(eb[0] - e1).max() <= 1e-13 * s and np.abs(hhb[0] - hh1).max() <= 1e-13 * s
    h2, _b = lib.create_for_problem(other, precision=lib.CMCG_FP64, stage_variant=form)
    e2, hh2, i2 = lib.cmcg_solve(h2, other.j_re, other.j_im, 1e-8, 400)
    s = np.abs(np.concatenate([e2, hh2], 1)).max()
    assert np.abs(eb[1] - e2).max() <= 1e-13 * s and np.abs(hhb[1] - hh2).max() <= 1e-13 * s
    h2.close()
    # cleared data: the same as a handle that never had data
    V = I.random_field(np.random.default_rng(7), mesh.nt, q)
    jr = I.random_field(np.random.default_rng(8), mesh.nt, q)[:, :3, :]
    lib.cmcg_set_boundary_data(h1, None)
    a = lib.dgtd_period_forward(h1, V, jr, None)
    h1.close()
    h3, _c = _handle(lib, mesh, q, lib.CMCG_FP64, form)
    assert np.array_equal(a, lib.dgtd_period_forward(h3, V, jr, None))
    h3.close()
