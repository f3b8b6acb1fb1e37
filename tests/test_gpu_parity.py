"""GPU parity: libcmcg (through its C ABI) against the FP64 oracle.

Tolerances (relative, (eps, mu)-weighted L2 unless noted):
* FP64 operator, sweeps, filtered sweeps: 1e-12.  The kernels and the oracle
  evaluate the same polynomial operator with different summation orders, so
  they differ by rounding only; source-free sweeps use the nested RK form (same
  polynomial).
* FP32 operator: 1e-5 (single-rounding errors of ~6e-8 times the operator's
  cancellation); FP32 sweeps 1e-5 per period; FP32 filtered results 1e-4.
* CMCG solves.  CG on the normal operator (I - P*)(I - P) amplifies rounding
  differently along the iteration: perturbing the oracle's own source by 1e-13
  moves its filtered iterate by ~1e-13 after 2-4 iterations, by ~4e-6 after 8
  (a transient where the residual grows), and by ~2e-12 once converged to
  1e-8 (22 iterations on the 384-tet cube).  The checks therefore compare 4
  fixed iterations at 1e-10 and the converged FP64 solve at 1e-9 (same
  iteration count); the FP32 solve to 1e-5 is compared at 1e-4.

Meshes span several 32-tet tiles with ragged tails (27 and 504 cubes per
shape class), a distorted mesh with no repeated shapes (single sorted group),
a single tetrahedron, PEC and impedance faces, and permittivity jumps.
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


def _problem(kind, q, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "cube3":
        p = I.cube_problem(3, q, 4 * math.pi, (0.4, 0.5, 0.6), (0.2, 1.0, -0.3), 0.2,
                           eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.5, 1.0))
    elif kind == "scatterer8":
        p = I.cube_problem(8, q, 4 * math.pi, (0.2, 0.3, 0.7), (1.0, 0.0, 0.5), 0.15, removed=(3, 5),
                           eps_fn=lambda c: np.where(np.linalg.norm(c - 0.25, axis=1) < 0.2, 4.0, 1.0))
    elif kind == "distorted":
        p = I.cube_problem(3, q, 2 * math.pi, (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 0.3)
        v = p.mesh.verts.copy()
        inner = np.all((v > 1e-9) & (v < 1 - 1e-9), axis=1)
        v[inner] += rng.uniform(-0.04, 0.04, (inner.sum(), 3))
        p.mesh.verts = v
        nodes = I.physical_nodes(v, p.mesh.tets, q)
        p.j_re = I.gaussian_current(nodes, (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 0.3)
        p.j_im = 0.3 * p.j_re
    elif kind == "single":
        verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
        mesh = I.Mesh(verts=verts, tets=np.array([[0, 1, 2, 3]], np.int32),
                      tags=np.array([[2, 1, 2, 1]], np.uint8), h=1.0)
        nodes = I.physical_nodes(verts, mesh.tets, q)
        jr = I.gaussian_current(nodes, (0.2, 0.2, 0.2), (1, 1, 0), 0.5)
        p = I.Problem("single", mesh, np.array([2.0]), np.array([1.5]), 2 * math.pi, q, jr, np.zeros_like(jr), 1e-8)
    else:
        raise ValueError(kind)
    return p


def _geo(p):
    from oracle.geometry import build_geometry
    return build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)


def _rel(a, b, g):
    from oracle.dg import inner
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


CASES = [("cube3", 1), ("cube3", 2), ("cube3", 3), ("scatterer8", 1), ("scatterer8", 2), ("distorted", 2),
         ("distorted", 3), ("single", 1), ("single", 3)]


@pytest.mark.parametrize("kind,q", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_operator_parity(lib, kind, q, prec):
    from oracle.dg import Phi, apply_B
    p = _problem(kind, q)
    g = _geo(p)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32)
    tol = 1e-12 if prec == "fp64" else 1e-5
    U = I.random_field(np.random.default_rng(7), p.nt, q)
    t = 0.37 * (2 * math.pi / p.omega)
    assert _rel(lib.dgtd_apply(h, t, U, p.j_re, p.j_im), Phi(t, U, g, p.omega, p.j_re, p.j_im), g) < tol
    assert _rel(lib.dgtd_apply(h, 0.0, U, adjoint=True), apply_B(U, g, adjoint=True), g) < tol
    h.close()


@pytest.mark.parametrize("kind,q", [("cube3", 1), ("cube3", 2), ("scatterer8", 1), ("distorted", 3), ("single", 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_period_sweeps_parity(lib, kind, q, prec):
    from oracle.timestep import Stepper
    from oracle.filtering import filtered_sweep
    p = _problem(kind, q)
    g = _geo(p)
    st = Stepper(g, p.omega)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32)
    assert h.steps == st.M
    tol = 1e-12 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(11)
    U, W = I.random_field(rng, p.nt, q), I.random_field(rng, p.nt, q)
    assert _rel(lib.dgtd_period_forward(h, U), st.P(U), g) < tol
    assert _rel(lib.dgtd_period_adjoint(h, W), st.P_star(W), g) < tol
    uT, fr, fi = lib.dgtd_period_forward(h, U, p.j_re, p.j_im, filtered=True)
    assert _rel(uT, st.P_psi(U, p.j_re, p.j_im), g) < tol
    F = filtered_sweep(st, U, p.j_re, p.j_im)
    assert _rel(fr + 1j * fi, F, g) < (1e-12 if prec == "fp64" else 1e-4)
    h.close()


def test_discrete_adjoint_identity_on_gpu(lib):
    from oracle.dg import inner
    p = _problem("scatterer8", 2)
    g = _geo(p)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    rng = np.random.default_rng(3)
    U, W = I.random_field(rng, p.nt, 2), I.random_field(rng, p.nt, 2)
    a = inner(lib.dgtd_period_forward(h, U), W, g)
    b = inner(U, lib.dgtd_period_adjoint(h, W), g)
    assert abs(a - b) < 1e-12 * abs(a) + 1e-12
    h.close()


def test_cmcg_fixed_iterations_match_oracle(lib):
    from oracle import cmcg as ocmcg
    from oracle.timestep import Stepper
    p = I.plain_fp64_cube()
    g = _geo(p)
    st = Stepper(g, p.omega)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, tol=0.0, max_iter=4)
    assert info.iters == 4 and info.periods == 11
    ref = ocmcg.solve(st, p.j_re, p.j_im, tol=0.0, max_iter=4)
    assert ref.iters == 4
    got = np.concatenate([e, hh], axis=1)
    assert _rel(got, ref.filtered, g) < 1e-10
    assert abs(info.rel_residual - ref.residuals[-1]) < 1e-8 * ref.residuals[-1] + 1e-14
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cmcg_converged_solve_matches_oracle(lib, prec):
    from oracle import cmcg as ocmcg
    from oracle.timestep import Stepper
    p = I.plain_fp64_cube()
    g = _geo(p)
    st = Stepper(g, p.omega)
    ref = ocmcg.solve(st, p.j_re, p.j_im, tol=p.tol, max_iter=500)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32)
    tol = p.tol if prec == "fp64" else 1e-5
    e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, tol=tol, max_iter=500)
    assert info.status == lib.CMCG_OK
    got = np.concatenate([e, hh], axis=1)
    assert _rel(got, ref.filtered, g) < (1e-9 if prec == "fp64" else 1e-4)
    if prec == "fp64":
        assert info.iters == ref.iters
    h.close()


def test_device_entry_points_match_host_entry_points(lib):
    import torch
    p = _problem("cube3", 2)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP32)
    U = I.random_field(np.random.default_rng(5), p.nt, 2)
    host = lib.dgtd_period_forward(h, U, p.j_re, p.j_im)
    dev = torch.device("cuda:0")
    u0 = torch.from_numpy(U).to(dev)
    jr, ji = torch.from_numpy(p.j_re).to(dev), torch.from_numpy(p.j_im).to(dev)
    uT = torch.empty_like(u0)
    lib.dgtd_period_forward_device(h, u0, jr, ji, uT)
    assert np.array_equal(uT.cpu().numpy(), host)
    e, hh, _ = lib.cmcg_solve(h, p.j_re, p.j_im, tol=1e-4, max_iter=50)
    outs = [torch.empty(p.nt, 3, p.np_, dtype=torch.float64, device=dev) for _ in range(4)]
    lib.cmcg_solve_device(h, jr, ji, 1e-4, 50, *outs)
    assert np.array_equal(outs[0].cpu().numpy() + 1j * outs[1].cpu().numpy(), e)
    assert np.array_equal(outs[2].cpu().numpy() + 1j * outs[3].cpu().numpy(), hh)
    h.close()


def test_full_size_scatterer_operator_parity(lib):
    """The 81,648-tet P2 workload of the benchmark: one operator application vs the oracle."""
    from oracle.dg import Phi
    p = I.scatterer_sphere()
    g = _geo(p)
    U = I.random_field(np.random.default_rng(1), p.nt, 2)
    t = 0.1
    ref = Phi(t, U, g, p.omega, p.j_re, p.j_im)
    for prec, tol in ((lib.CMCG_FP32, 1e-5), (lib.CMCG_FP64, 1e-12)):
        h, _ = lib.create_for_problem(p, precision=prec)
        assert h.steps == 242
        assert _rel(lib.dgtd_apply(h, t, U, p.j_re, p.j_im), ref, g) < tol
        h.close()


def test_hbm_budget_is_enforced(lib):
    p = _problem("cube3", 1)
    with pytest.raises(lib.CMCGError) as ei:
        lib.create_for_problem(p, hbm_budget_bytes=1000)
    assert ei.value.code == lib.CMCG_ERR_OUT_OF_MEMORY


@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_stage_kernel_form_matches_oracle(lib, q, prec):
    """Each forced stage-kernel form (two or four threads per tetrahedron, each at several
    occupancies, and the tensor-core form) gives the oracle's sweeps: the autotuner's choice
    cannot change results."""
    from oracle.timestep import Stepper
    p = _problem("scatterer8", q) if q < 3 else _problem("cube3", q)
    g = _geo(p)
    st = Stepper(g, p.omega)
    rng = np.random.default_rng(17)
    U = I.random_field(rng, p.nt, q)
    refF, refA = st.P(U), st.P_star(U)
    tol = 1e-12 if prec == "fp64" else 1e-5
    forms = [1, 2, 3, 4, 5, 6, 7, 8] if prec == "fp32" else [1, 2, 3, 4]
    tried = 0
    for k in forms:
        try:
            h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32,
                                          stage_variant=k)
        except lib.CMCGError as e:
            assert e.code == lib.CMCG_ERR_INVALID_ARG  # form does not fit this order / precision
            continue
        tried += 1
        assert _rel(lib.dgtd_period_forward(h, U), refF, g) < tol, k
        assert _rel(lib.dgtd_period_adjoint(h, U), refA, g) < tol, k
        h.close()
    assert tried == (7 if prec == "fp32" else 3)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_unstable_time_step_is_reported(lib, prec):
    """A step far beyond the CFL limit (M = 3 instead of 16) makes the period map grow the
    (eps, mu)-norm by orders of magnitude (the oracle's P multiplies that of a random field by
    more than 100); the solve stops in its first CG iteration with CMCG_ERR_UNSTABLE instead of
    iterating on garbage, while the CFL step, whose period map is not a contraction either
    (transient growth up to about 3), raises no false alarm."""
    from oracle.timestep import Stepper
    p = _problem("cube3", 1)
    g = _geo(p)
    st = Stepper(g, p.omega, M=3)
    U = I.random_field(np.random.default_rng(5), p.nt, 1)
    from oracle.dg import norm
    assert norm(st.P(U), g) > 100 * norm(U, g)
    P = lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32
    h, _ = lib.create_for_problem(p, precision=P, steps_per_period=3)
    with pytest.raises(lib.CMCGError) as ei:
        lib.cmcg_solve(h, p.j_re, p.j_im, 1e-8, 50)
    assert ei.value.code == lib.CMCG_ERR_UNSTABLE
    h.close()
    h, _ = lib.create_for_problem(p, precision=P)  # the CFL step: no false alarm
    e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, 1e-6, 400)
    assert info.status == lib.CMCG_OK
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fw_baseline_matches_oracle(lib, prec):
    """Limiting-amplitude baseline (Section 6): F_psi(P_psi^l 0) equals the oracle's for l = 0, 3."""
    from oracle import fw as ofw
    from oracle.timestep import Stepper
    p = _problem("scatterer8", 2)
    g = _geo(p)
    st = Stepper(g, p.omega)
    P = lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32
    tol = 1e-12 if prec == "fp64" else 1e-4
    h, _ = lib.create_for_problem(p, precision=P)
    for periods in (0, 3):
        e, hh = lib.cmcg_fw_solve(h, p.j_re, p.j_im, periods)
        ref = ofw.fw_solve(st, p.j_re, p.j_im, periods)
        assert _rel(np.concatenate([e, hh], axis=1), ref, g) < tol, periods
    h.close()


def test_fw_batch_approaches_cmcg_and_matches_single(lib):
    """On the open 3^3 cube FW approaches the CMCG result as the simulated periods grow (the
    oracle gives 3.5e-2, 1.8e-4, 1.6e-7 at 2, 6, 12 periods); the batch entry equals the single."""
    p = _problem("cube3", 1)
    g = _geo(p)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    e_cg, h_cg, info = lib.cmcg_solve(h, p.j_re, p.j_im, 1e-10, 400)
    ref = np.concatenate([e_cg, h_cg], axis=1)
    errs = []
    for periods in (2, 6, 12):
        e, hh = lib.cmcg_fw_solve(h, p.j_re, p.j_im, periods)
        errs.append(_rel(np.concatenate([e, hh], axis=1), ref, g))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6
    eb, hb = lib.cmcg_fw_solve_batch(h, [p.j_re], [p.j_im], 12)
    assert np.array_equal(eb[0], e) and np.array_equal(hb[0], hh)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_and_direct_launches_agree(lib, prec):
    """Sweeps replayed from CUDA graphs (the default) and launched directly give the same
    bits: forward and adjoint periods, a filtered source period and a whole CMCG solve."""
    p = _problem("cube3", 2)
    P = lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32
    U = I.random_field(np.random.default_rng(21), p.nt, 2)
    outs = []
    for graphs in (0, 2):
        h, _ = lib.create_for_problem(p, precision=P, stage_variant=1, launch_graphs=graphs)
        r = [lib.dgtd_period_forward(h, U), lib.dgtd_period_adjoint(h, U)]
        r += list(lib.dgtd_period_forward(h, U, p.j_re, p.j_im, filtered=True))
        e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, 1e-6, 200)
        r += [e, hh]
        r.append(lib.dgtd_period_forward(h, U))  # a replay of the first graph
        outs.append(r)
        h.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert np.array_equal(outs[0][0], outs[0][-1])
