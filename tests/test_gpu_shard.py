"""Sharded handles on one GPU: parts of an element partition with ghost layers, a halo
exchange after every RK stage and CG reductions summed over the parts, against the
unsharded handle and the FP64 oracle.

The exchange and the summed reductions make every sweep and every CG scalar those of the
whole mesh up to the order of summation, so FP64 sweeps, filtered sweeps and inner products
match the unsharded handle to 1e-12 and the converged FP64 solve to 1e-9 with the same
iteration count (CG rounding, see test_gpu_parity); FP32 sweeps match the oracle to 1e-5.
"""
import math

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2106_02858_gb300 import build
    build.build()
    from paper_2106_02858_gb300 import cmcg
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return cmcg


def _problem(kind, q):
    if kind == "scatterer8":
        return I.cube_problem(8, q, 4 * math.pi, (0.2, 0.3, 0.7), (1.0, 0.0, 0.5), 0.15, removed=(3, 5),
                              eps_fn=lambda c: np.where(np.linalg.norm(c - 0.25, axis=1) < 0.2, 4.0, 1.0))
    return I.cube_problem(3, q, 4 * math.pi, (0.4, 0.5, 0.6), (0.2, 1.0, -0.3), 0.2,
                          eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.5, 1.0))


def _geo(p):
    from oracle.geometry import build_geometry
    return build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)


def _rel(a, b, g):
    from oracle.dg import inner
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


def _sharded(lib, p, nparts, axis, precision, **kw):
    m = lib.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags)
    part = lib.cmcg_partition_slabs(m, nparts, axis)
    opt = lib.cmcg_default_options(order=p.order, precision=precision, **kw)
    return lib.cmcg_create_sharded(m, p.eps, p.mu, p.omega, opt, part), m


@pytest.mark.parametrize("kind,q,nparts,axis", [("scatterer8", 2, 2, 2), ("scatterer8", 1, 3, 0),
                                                ("cube3", 3, 2, 1), ("scatterer8", 2, 5, 2)])
def test_sharded_sweeps_equal_the_unsharded_handle(lib, kind, q, nparts, axis):
    p = _problem(kind, q)
    g = _geo(p)
    hs, _m = _sharded(lib, p, nparts, axis, lib.CMCG_FP64)
    hu, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    assert hs.nt == p.nt and hs.steps == hu.steps
    rng = np.random.default_rng(5)
    U, W = I.random_field(rng, p.nt, q), I.random_field(rng, p.nt, q)
    t = 0.2 * (2 * math.pi / p.omega)
    assert _rel(lib.dgtd_apply(hs, t, U, p.j_re, p.j_im), lib.dgtd_apply(hu, t, U, p.j_re, p.j_im), g) < 1e-12
    assert _rel(lib.dgtd_period_forward(hs, U), lib.dgtd_period_forward(hu, U), g) < 1e-12
    assert _rel(lib.dgtd_period_adjoint(hs, W), lib.dgtd_period_adjoint(hu, W), g) < 1e-12
    a = lib.dgtd_period_forward(hs, U, p.j_re, p.j_im, filtered=True)
    b = lib.dgtd_period_forward(hu, U, p.j_re, p.j_im, filtered=True)
    assert _rel(a[0], b[0], g) < 1e-12
    assert _rel(a[1] + 1j * a[2], b[1] + 1j * b[2], g) < 1e-12
    x, y = lib.cmcg_inner(hs, U, W), lib.cmcg_inner(hu, U, W)
    assert abs(x - y) <= 1e-12 * abs(y)
    hs.close()
    hu.close()


def test_sharded_cmcg_equals_unsharded_and_oracle(lib):
    from oracle import cmcg as ocmcg
    from oracle.timestep import Stepper
    p = _problem("cube3", 1)
    g = _geo(p)
    hs, _m = _sharded(lib, p, 3, 2, lib.CMCG_FP64)
    hu, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    es, hhs, i_s = lib.cmcg_solve(hs, p.j_re, p.j_im, 1e-8, 400)
    eu, hhu, i_u = lib.cmcg_solve(hu, p.j_re, p.j_im, 1e-8, 400)
    assert i_s.status == lib.CMCG_OK and i_s.iters == i_u.iters
    fs, fu = np.concatenate([es, hhs], 1), np.concatenate([eu, hhu], 1)
    assert _rel(fs, fu, g) < 1e-9
    ref = ocmcg.solve(Stepper(g, p.omega), p.j_re, p.j_im, tol=1e-8, max_iter=400)
    assert ref.iters == i_s.iters
    assert _rel(fs, ref.filtered, g) < 1e-9
    hs.close()
    hu.close()


@pytest.mark.parametrize("form", [0, 2, 7])
def test_sharded_fp32_sweeps_match_oracle(lib, form):
    from oracle.timestep import Stepper
    p = _problem("scatterer8", 2)
    g = _geo(p)
    st = Stepper(g, p.omega)
    hs, _m = _sharded(lib, p, 3, 2, lib.CMCG_FP32, stage_variant=form)
    U = I.random_field(np.random.default_rng(7), p.nt, 2)
    assert _rel(lib.dgtd_period_forward(hs, U), st.P(U), g) < 1e-5
    assert _rel(lib.dgtd_period_adjoint(hs, U), st.P_star(U), g) < 1e-5
    hs.close()


def test_sharded_handle_rejects_batch_entry_points(lib):
    p = _problem("cube3", 2)
    hs, _m = _sharded(lib, p, 2, 2, lib.CMCG_FP64)
    with pytest.raises(lib.CMCGError) as ei:
        lib.cmcg_set_conductivity(hs, np.zeros(p.nt))
    assert ei.value.code == lib.CMCG_ERR_INVALID_ARG
    with pytest.raises(lib.CMCGError):
        lib.cmcg_fw_solve(hs, p.j_re, p.j_im, 1)
    hs.close()
