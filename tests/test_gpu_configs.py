"""The batched workloads at their stated shapes, through the C ABI, against the FP64 oracle (GPU).

* Batched sources: 32 seeded Gaussian sources on the 384-tet cube at P3 (omega = 4 pi,
  CG to 1e-6), FP32 sweeps with the kernel form chosen by timing (the tensor-core
  form on this shape), in one handle.  Every source's filtered field is compared
  with the FP64 GPU solve of the same batch (1e-4); source 0 is solved to
  convergence by the oracle (FP32 1e-4; FP64 1e-9 with the same iteration count).
* Uneven problems: meshes of the uneven-batch recipe (n^3 Kuhn cubes, eps on a
  seeded 2x2x2 block partition drawn U[1,4], impedance outer boundary, one seeded
  Gaussian source) at n in {6, 7, 8}, q = 1..3, omega in {2, 4, 8} pi, one handle
  per order.  Four CG iterations against the oracle's four (FP64 1e-10, FP32 in the
  mix 1e-4: the CG transient amplifies rounding, see test_gpu_parity), and the
  converged FP32 batch against the converged FP64 GPU solves (1e-4).
* The full 64-problem uneven batch (n ~ U{6..20}, about 1.1e8 dofs), one handle per
  order: every problem converges, and sampled problems give the same result alone
  and in the mix (1e-13 relative, same kernel form).

Oracle solves run in spawned worker processes while the GPU works.
"""
import concurrent.futures as cf
import math
import multiprocessing as mp

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I

import oracle_jobs as J

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oracle_results():
    """Starts every oracle job of this module at once (spawned workers)."""
    jobs = {("rhs", 0): (1e-6, 400)}
    for k in range(len(J.BLOCK_SHAPES)):
        jobs[("block", k)] = (0.0, 4)
    ex = cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn"))
    futs = {spec: ex.submit(J.cmcg_solve, spec, tol, it) for spec, (tol, it) in jobs.items()}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def lib(oracle_results):
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


def _batch(lib, probs, precision, **kw):
    meshes = [lib.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags) for p in probs]
    opt = lib.cmcg_default_options(order=probs[0].order, precision=precision, **kw)
    return lib.cmcg_create_batch([(m, p.eps, p.mu, p.omega) for m, p in zip(meshes, probs)], opt), meshes


def test_batched_sources_32_on_the_384_tet_cube(lib, oracle_results):
    b = I.batched_rhs(nrhs=32)
    assert b.nt == 384 and b.order == 3 and b.j_re.shape[0] == 32
    probs = [I.Problem(f"rhs{k}", b.mesh, b.eps, b.mu, b.omega, 3, b.j_re[k], b.j_im[k], b.tol) for k in range(32)]
    h32, _a = _batch(lib, probs, lib.CMCG_FP32)
    form = lib.cmcg_get_tuning(h32)[0]
    e32, hh32, i32 = lib.cmcg_solve_batch(h32, list(b.j_re), list(b.j_im), b.tol, 400)
    h32.close()
    h64, _b = _batch(lib, probs, lib.CMCG_FP64)
    e64, hh64, i64 = lib.cmcg_solve_batch(h64, list(b.j_re), list(b.j_im), b.tol, 400)
    h64.close()
    g = _geo(probs[0])
    for k in range(32):
        assert i32[k].status == lib.CMCG_OK and i64[k].status == lib.CMCG_OK
        f32 = np.concatenate([e32[k], hh32[k]], 1)
        f64 = np.concatenate([e64[k], hh64[k]], 1)
        assert _rel(f32, f64, g) < 1e-4, (k, form)
    ref, iters = oracle_results[("rhs", 0)].result()
    assert iters == i64[0].iters
    assert _rel(np.concatenate([e64[0], hh64[0]], 1), ref, g) < 1e-9
    assert _rel(np.concatenate([e32[0], hh32[0]], 1), ref, g) < 1e-4


def test_uneven_shapes_against_the_oracle(lib, oracle_results):
    probs = I.block_eps_subset(J.BLOCK_SHAPES, seed=J.BLOCK_SEED)
    by_order = {}
    for k, p in enumerate(probs):
        by_order.setdefault(p.order, []).append(k)
    got32, conv32 = {}, {}
    for q, ks in by_order.items():
        sub = [probs[k] for k in ks]
        h, _m = _batch(lib, sub, lib.CMCG_FP32)
        e, hh, infos = lib.cmcg_solve_batch(h, [p.j_re for p in sub], [p.j_im for p in sub], 0.0, 4)
        for i, k in enumerate(ks):
            assert infos[i].iters == 4
            got32[k] = np.concatenate([e[i], hh[i]], 1)
        e, hh, infos = lib.cmcg_solve_batch(h, [p.j_re for p in sub], [p.j_im for p in sub], 1e-5, 600)
        for i, k in enumerate(ks):
            assert infos[i].status == lib.CMCG_OK
            conv32[k] = np.concatenate([e[i], hh[i]], 1)
        h.close()
    for k, p in enumerate(probs):
        g = _geo(p)
        h, _m = lib.create_for_problem(p, precision=lib.CMCG_FP64)
        e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, tol=0.0, max_iter=4)
        four64 = np.concatenate([e, hh], 1)
        e, hh, info = lib.cmcg_solve(h, p.j_re, p.j_im, tol=1e-5, max_iter=600)
        assert info.status == lib.CMCG_OK
        conv64 = np.concatenate([e, hh], 1)
        h.close()
        assert _rel(conv32[k], conv64, g) < 1e-4, k
        ref, iters = oracle_results[("block", k)].result()
        assert iters == 4
        assert _rel(four64, ref, g) < 1e-10, k
        assert _rel(got32[k], ref, g) < 1e-4, k


def test_full_uneven_batch_of_64(lib):
    probs = I.uneven_batch()
    assert len(probs) == 64
    assert {p.meta["n"] for p in probs} <= set(range(6, 21)) and {p.order for p in probs} == {1, 2, 3}
    checked = 0
    for q in (1, 2, 3):
        sub = [p for p in probs if p.order == q]
        h, _m = _batch(lib, sub, lib.CMCG_FP32)
        form = lib.cmcg_get_tuning(h)[0]
        e, hh, infos = lib.cmcg_solve_batch(h, [p.j_re for p in sub], [p.j_im for p in sub], 1e-5, 600)
        h.close()
        assert all(i.status == lib.CMCG_OK for i in infos), [i.status for i in infos]
        assert len({i.steps_per_period for i in infos}) > 1
        # the smallest and the largest problem of this order, alone with the same form
        for k in (min(range(len(sub)), key=lambda i: sub[i].nt), max(range(len(sub)), key=lambda i: sub[i].nt)):
            ha, _ = lib.create_for_problem(sub[k], precision=lib.CMCG_FP32, stage_variant=form + 1)
            ea, hha, ia = lib.cmcg_solve(ha, sub[k].j_re, sub[k].j_im, 1e-5, 600)
            ha.close()
            assert ia.iters == infos[k].iters
            scale = np.abs(np.concatenate([ea, hha], 1)).max()
            assert np.abs(e[k] - ea).max() <= 1e-13 * scale
            assert np.abs(hh[k] - hha).max() <= 1e-13 * scale
            checked += 1
    assert checked == 6
