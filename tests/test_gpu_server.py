"""The serving runtime on the GPU: continuous batching, HBM admission, alone vs in the mix.

Requests of two models (a P3 cube and a P2 cube with a PEC scatterer) are
submitted from three host threads at seeded, staggered times, so batches form
while other batches are on the GPU.  Every result must equal the same request
solved alone on a one-problem handle with the same kernel form (the batched
arithmetic per problem is that of a solve alone; checked at 1e-13 relative),
whatever shared its batch.  A server whose HBM budget only admits the first
handle of each model must still serve every request (batches wait for pooled
handles instead of allocating).
"""
import math
import threading
import time

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORM = 2  # scalar kernel, at least 3 resident blocks per SM


@pytest.fixture(scope="module")
def lib():
    from paper_2106_02858_gb300 import build
    build.build()
    from paper_2106_02858_gb300 import cmcg
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return cmcg


def _models():
    small = I.cube_problem(3, 3, 4 * math.pi, (0.5, 0.5, 0.5), (1, 0, 0), 0.2, tol=1e-6)
    large = I.cube_problem(6, 2, 4 * math.pi, (0.3, 0.3, 0.3), (0, 0, 1), 0.15, removed=(2, 4), tol=1e-6)
    return small, large


def _sources(p, rng, count):
    nodes = I.physical_nodes(p.mesh.verts, p.mesh.tets, p.order)
    return [I.gaussian_current(nodes, rng.uniform(0.15, 0.85, 3), I.unit_vector(rng), 0.15) for _ in range(count)]


def _serve(lib, budget, tol=1e-6):
    small, large = _models()
    opt = lib.cmcg_server_default_options(precision=lib.CMCG_FP32, max_batch=3, workers=2, max_wait_ms=3.0, tol=tol,
                                          max_iter=500, hbm_budget_bytes=budget, stage_variant=FORM)
    srv = lib.cmcg_server_create(opt)
    ms = lib.make_mesh(small.mesh.verts, small.mesh.tets, small.mesh.tags)
    ml = lib.make_mesh(large.mesh.verts, large.mesh.tets, large.mesh.tags)
    m_small = lib.cmcg_server_add_model(srv, ms, small.eps, small.mu, small.omega, small.order)
    m_large = lib.cmcg_server_add_model(srv, ml, large.eps, large.mu, large.omega, large.order, max_batch=2)
    rng = np.random.default_rng(11)
    jobs = [(m_small, j) for j in _sources(small, rng, 8)] + [(m_large, j) for j in _sources(large, rng, 4)]
    order = rng.permutation(len(jobs))
    delays = rng.uniform(0.0, 0.05, len(jobs))
    tickets = [None] * len(jobs)

    def submitter(part):
        for k in part:
            time.sleep(delays[k])
            m, j = jobs[k]
            tickets[k] = lib.cmcg_server_submit(srv, m, j)

    threads = [threading.Thread(target=submitter, args=(order[i::3],)) for i in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    results = [lib.cmcg_server_poll(srv, tickets[k], jobs[k][0], wait=True) for k in range(len(jobs))]
    stats = lib.cmcg_server_stats(srv)
    srv.close()
    return (small, large), (m_small, m_large), jobs, results, stats


def _alone(lib, p, j, tol):
    h, _ = lib.create_for_problem(p, precision=lib.CMCG_FP32, stage_variant=FORM)
    e, hh, info = lib.cmcg_solve(h, j, None, tol, 500)
    h.close()
    return e, hh, info


def test_server_results_equal_solves_alone(lib):
    probs, mids, jobs, results, stats = _serve(lib, budget=0)
    assert stats["completed"] == len(jobs) and stats["queued"] == 0
    for (m, j), res in zip(jobs, results):
        status, e, hh, info, latency, queued = res
        assert status == lib.CMCG_OK
        assert latency >= queued >= 0.0
        p = probs[mids.index(m)]
        ea, hha, ia = _alone(lib, p, j, 1e-6)
        assert ia.iters == info.iters
        scale = np.abs(np.concatenate([ea, hha], 1)).max()
        assert np.abs(e - ea).max() <= 1e-13 * scale
        assert np.abs(hh - hha).max() <= 1e-13 * scale


def test_server_respects_hbm_budget(lib):
    small, large = _models()
    # Room for the first handle of each model only (sizes measured on real handles).
    sizes = []
    for p, cap in ((small, 3), (large, 2)):
        meshes = [lib.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags)] * cap
        h = lib.cmcg_create_batch([(m, p.eps, p.mu, p.omega) for m in meshes],
                                  lib.cmcg_default_options(order=p.order, precision=lib.CMCG_FP32, stage_variant=FORM))
        sizes.append(lib.cmcg_device_bytes(h))
        h.close()
    budget = sum(sizes) + 1024
    probs, mids, jobs, results, stats = _serve(lib, budget=budget)
    assert stats["handles"] == 2 and stats["bytes_in_use"] <= budget
    assert all(r[0] == lib.CMCG_OK for r in results)
