"""The conductivity term (Eq. maxwell_time_strong, Section 1: eps dE/dt + sigma E + curl H = J;
coefficients Section 3.1; the DG term (sigma E_h, v_h) of Section 5.2.2) on the GPU against the
FP64 oracle, whose sigma term is pinned in test_oracle_conductivity (Ohmic energy identity,
adjoint identity, static-mode decay, convergence to the frequency-domain solve).

Tolerances as for sigma = 0 (test_gpu_parity): FP64 operator and sweeps 1e-12, FP32 1e-5 per
operator application and sweep, converged FP64 CMCG 1e-9 with the oracle's iteration count,
FP32 1e-4.  Every FP32 stage form (two threads, four threads, tensor cores) carries the term.
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


def _case(q, seed=0):
    rng = np.random.default_rng(seed)
    p = I.cube_problem(3, q, 4 * math.pi, (0.4, 0.5, 0.6), (0.2, 1.0, -0.3), 0.2,
                       eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.5, 1.0))
    sig = rng.uniform(0.0, 3.0, p.nt)
    from oracle.geometry import build_geometry
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, q, sigma=sig)
    return p, sig, g


def _rel(a, b, g):
    from oracle.dg import inner
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("prec,form", [("fp64", 0), ("fp64", 2), ("fp32", 2), ("fp32", 5), ("fp32", 7)])
def test_operator_and_sweeps_with_conductivity(lib, q, prec, form):
    from oracle.dg import Phi, apply_B
    from oracle.timestep import Stepper
    p, sig, g = _case(q)
    P = lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32
    h, _ = lib.create_for_problem(p, precision=P, stage_variant=form)
    lib.cmcg_set_conductivity(h, sig)
    tol = 1e-12 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(3)
    U, W = I.random_field(rng, p.nt, q), I.random_field(rng, p.nt, q)
    t = 0.3 * (2 * math.pi / p.omega)
    assert _rel(lib.dgtd_apply(h, t, U, p.j_re, p.j_im), Phi(t, U, g, p.omega, p.j_re, p.j_im), g) < tol
    assert _rel(lib.dgtd_apply(h, 0.0, U, adjoint=True), apply_B(U, g, adjoint=True), g) < tol
    st = Stepper(g, p.omega)
    assert h.steps == st.M
    assert _rel(lib.dgtd_period_forward(h, U), st.P(U), g) < tol
    assert _rel(lib.dgtd_period_adjoint(h, W), st.P_star(W), g) < tol
    assert _rel(lib.dgtd_period_forward(h, U, p.j_re, p.j_im), st.P_psi(U, p.j_re, p.j_im), g) < tol
    h.close()


def test_adjoint_identity_and_removal(lib):
    from oracle.dg import inner
    p, sig, g = _case(2, seed=1)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    rng = np.random.default_rng(4)
    U, W = I.random_field(rng, p.nt, 2), I.random_field(rng, p.nt, 2)
    before = lib.dgtd_period_forward(h, U)
    lib.cmcg_set_conductivity(h, sig)
    a = inner(lib.dgtd_period_forward(h, U), W, g)
    b = inner(U, lib.dgtd_period_adjoint(h, W), g)
    assert abs(a - b) < 1e-12 * abs(a)
    lib.cmcg_set_conductivity(h, None)  # back to sigma = 0: the same bits as before
    assert np.array_equal(lib.dgtd_period_forward(h, U), before)
    # rejected values change nothing
    for bad in (-sig, np.full(p.nt, 1e9)):
        with pytest.raises(lib.CMCGError) as ei:
            lib.cmcg_set_conductivity(h, bad)
        assert ei.value.code == lib.CMCG_ERR_INVALID_ARG
    assert np.array_equal(lib.dgtd_period_forward(h, U), before)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cmcg_with_conductivity_matches_oracle(lib, prec):
    from oracle import cmcg as ocmcg
    from oracle.timestep import Stepper
    p, sig, g = _case(1, seed=2)
    ref = ocmcg.solve(Stepper(g, p.omega), p.j_re, p.j_im, tol=1e-8, max_iter=400)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32)
    lib.cmcg_set_conductivity(h, sig)
    e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, tol=1e-8 if prec == "fp64" else 1e-5, max_iter=400)
    h.close()
    assert info.status == lib.CMCG_OK
    got = np.concatenate([e, hh], axis=1)
    if prec == "fp64":
        assert info.iters == ref.iters
        assert _rel(got, ref.filtered, g) < 1e-9
    else:
        assert _rel(got, ref.filtered, g) < 1e-4
