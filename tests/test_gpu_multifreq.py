"""Several frequencies in one solve (cmcg_solve_multifreq) on the GPU against the oracle's
multi-frequency CMCG (oracle.multifreq, pinned in test_oracle_multifreq: one harmonic is the
single-frequency solve, the summed-source sweep is linear in the harmonics, and every harmonic
converges to its frequency-domain solve).

Tolerances as for single solves (test_gpu_parity): converged FP64 1e-9 with the oracle's
iteration count, FP32 1e-4; with one harmonic the result is that of cmcg_solve to rounding.
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


def _case(q, K, seed=0):
    p = I.cube_problem(3, q, 2 * math.pi, (0.5, 0.5, 0.5), (0.3, 1.0, -0.2), 0.25,
                       eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.0, 1.0))
    rng = np.random.default_rng(seed)
    nodes = I.physical_nodes(p.mesh.verts, p.mesh.tets, q)
    J = np.stack([I.gaussian_current(nodes, rng.uniform(0.3, 0.7, 3), I.unit_vector(rng), 0.25) for _ in range(K)])
    Ji = 0.4 * np.roll(J, 1, axis=0)
    from oracle.geometry import build_geometry
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, q)
    return p, J, Ji, g


def _rel(a, b, g):
    from oracle.dg import inner
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


@pytest.mark.parametrize("q,harm", [(1, [1, 2]), (2, [1, 3, 4])])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_multifreq_matches_the_oracle(lib, q, harm, prec):
    from oracle import multifreq as MF
    p, J, Ji, g = _case(q, len(harm))
    tol = 1e-8 if prec == "fp64" else 1e-5
    ref = MF.solve(MF.MultiStepper(g, p.omega, harm), J, Ji, tol=1e-8, max_iter=400)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32)
    e, hh, info = lib.cmcg_solve_multifreq(h, harm, list(J), list(Ji), tol, 400)
    h.close()
    assert info.status == lib.CMCG_OK
    assert info.periods == 3 + 2 * info.iters + len(harm) - 1
    if prec == "fp64":
        assert info.iters == ref[0].iters
    for k in range(len(harm)):
        got = np.concatenate([e[k], hh[k]], axis=1)
        assert _rel(got, ref[k].filtered, g) < (1e-9 if prec == "fp64" else 1e-4), (harm[k], prec)


def test_one_harmonic_is_the_single_solve(lib):
    p, J, Ji, g = _case(2, 1)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    e1, h1, i1 = lib.cmcg_solve_multifreq(h, [1], [J[0]], [Ji[0]], 1e-8, 400)
    e, hh, i = lib.cmcg_solve(h, J[0], Ji[0], 1e-8, 400)
    h.close()
    assert i1.iters == i.iters
    assert _rel(np.concatenate([e1[0], h1[0]], 1), np.concatenate([e, hh], 1), g) < 1e-12


def test_multifreq_arguments_are_checked(lib):
    p, J, Ji, g = _case(1, 2)
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP64)
    with pytest.raises(lib.CMCGError) as ei:
        lib.cmcg_solve_multifreq(h, [1, 0], list(J), None, 1e-6, 10)
    assert ei.value.code == lib.CMCG_ERR_INVALID_ARG
    h.close()
