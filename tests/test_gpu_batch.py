"""Batched solves on the GPU: many sources on one mesh and uneven meshes in one handle.

* Alone vs in the mix: each problem of a batch gives the same filtered result
  as the same problem solved alone.  With the same kernel form both runs do
  the same arithmetic per problem (problem-aligned reductions, per-problem CG
  scalars, converged problems frozen), so FP64 and FP32 results agree to the
  last bits (checked at 1e-13 relative).
* Batched FP32 vs batched FP64: 1e-4 relative L2 on the filtered fields.
* Batched results vs the FP64 oracle for a small problem set (tolerances as
  in test_gpu_parity: converged FP64 solves at 1e-9).
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


def _geo(p):
    from oracle.geometry import build_geometry
    return build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)


def _rel(a, b, g):
    from oracle.dg import inner
    d = a - b
    return math.sqrt(abs(np.real(inner(d, d, g))) / abs(np.real(inner(b, b, g))))


def _create_batch(lib, probs, precision, stage_variant=0):
    meshes = [lib.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags) for p in probs]
    opt = lib.cmcg_default_options(order=probs[0].order, precision=precision, stage_variant=stage_variant)
    h = lib.cmcg_create_batch([(m, p.eps, p.mu, p.omega) for m, p in zip(meshes, probs)], opt)
    return h, meshes


def _uneven(q, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for n, omega in ((3, 2 * math.pi), (5, 4 * math.pi), (2, 4 * math.pi), (4, 8 * math.pi)):
        blocks = rng.uniform(1, 4, 8)
        eps_fn = lambda c, b=blocks: b[(c[:, 0] >= 0.5).astype(int) + 2 * (c[:, 1] >= 0.5) + 4 * (c[:, 2] >= 0.5)]
        out.append(I.cube_problem(n, q, omega, rng.uniform(0.3, 0.7, 3), I.unit_vector(rng), 0.2, eps_fn=eps_fn,
                                  tol=1e-6))
    return out


@pytest.mark.parametrize("threads", [2, 4])
@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_batch_alone_vs_in_the_mix(lib, q, prec, threads):
    probs = _uneven(q)
    P = lib.CMCG_FP64 if prec == "fp64" else lib.CMCG_FP32
    # the same kernel form alone and in the mix: two or four threads per tetrahedron
    form = {("fp32", 2): 2, ("fp32", 4): 5, ("fp64", 2): 1, ("fp64", 4): 2}[prec, threads]
    h, _m = _create_batch(lib, probs, P, stage_variant=form)
    assert lib.cmcg_batch_size(h) == len(probs)
    steps = [lib.cmcg_get_problem(h, p)[1] for p in range(len(probs))]
    assert len(set(steps)) > 1  # genuinely uneven step counts
    tol = 1e-6
    eb, hb, infos = lib.cmcg_solve_batch(h, [p.j_re for p in probs], [p.j_im for p in probs], tol, 400)
    h.close()
    assert len({i.iters for i in infos}) > 1  # problems converge at different iterations
    for k, p in enumerate(probs):
        ha, _ = lib.create_for_problem(p, precision=P, stage_variant=form)
        ea, hha, ia = lib.cmcg_solve(ha, p.j_re, p.j_im, tol, 400)
        ha.close()
        assert ia.iters == infos[k].iters
        scale = np.abs(np.concatenate([ea, hha], 1)).max()
        assert np.abs(eb[k] - ea).max() <= 1e-13 * scale
        assert np.abs(hb[k] - hha).max() <= 1e-13 * scale


def test_many_sources_on_one_mesh_fp32_vs_fp64_and_oracle(lib):
    from oracle import cmcg as ocmcg
    from oracle.timestep import Stepper
    base = I.batched_rhs(nrhs=6, n=3, order=3)
    probs = []
    for r in range(6):
        p = I.Problem(f"rhs{r}", base.mesh, base.eps, base.mu, base.omega, 3, base.j_re[r], base.j_im[r], 1e-6)
        probs.append(p)
    tol = 1e-6
    h64, _a = _create_batch(lib, probs, lib.CMCG_FP64)
    e64, h64f, i64 = lib.cmcg_solve_batch(h64, [p.j_re for p in probs], None, tol, 400)
    h64.close()
    h32, _b = _create_batch(lib, probs, lib.CMCG_FP32)
    e32, h32f, i32 = lib.cmcg_solve_batch(h32, [p.j_re for p in probs], None, tol, 400)
    h32.close()
    g = _geo(probs[0])
    for k in range(6):
        f64 = np.concatenate([e64[k], h64f[k]], 1)
        f32 = np.concatenate([e32[k], h32f[k]], 1)
        assert i64[k].status == lib.CMCG_OK and i32[k].status == lib.CMCG_OK
        assert _rel(f32, f64, g) < 1e-4
    st = Stepper(g, probs[0].omega)
    for k in (0, 5):
        ref = ocmcg.solve(st, probs[k].j_re, None, tol=tol, max_iter=400)
        assert ref.iters == i64[k].iters
        assert _rel(np.concatenate([e64[k], h64f[k]], 1), ref.filtered, g) < 1e-9
