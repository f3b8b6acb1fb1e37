"""Continuous batching at the slot level (cmcg_slot_*) on the GPU.

A batch handle's problems are slots; requests are admitted into free slots between rounds
while other requests are mid-solve, and a slot freed by a finished request takes the next
one.  Each slot runs the operations of a solve alone (Algorithms init, grad, cmcg, the final
filter of Section 5.4) with the same kernel form, so every result equals the same request
solved alone with cmcg_solve to 1e-13 relative (max-abs over the field), with the same
iteration count, in FP32 and FP64.
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


@pytest.mark.parametrize("prec,form", [("fp32", 2), ("fp32", 7), ("fp64", 1)])
def test_requests_admitted_mid_solve_equal_their_alone_solves(lib, prec, form):
    b = I.batched_rhs(nrhs=6, n=3, order=2, tol=1e-6)
    P = lib.CMCG_FP32 if prec == "fp32" else lib.CMCG_FP64
    mesh = lib.make_mesh(b.mesh.verts, b.mesh.tets, b.mesh.tags)
    opt = lib.cmcg_default_options(order=2, precision=P, stage_variant=form)
    h = lib.cmcg_create_batch([(mesh, b.eps, b.mu, b.omega)] * 3, opt)
    tol, max_iter = 1e-6, 400
    queue = list(range(6))
    where = {}      # slot -> request
    results = {}
    rounds = 0
    admitted_mid = 0
    while queue or where:
        # admit into free slots, one per round so that requests start at different times
        free = [s for s in range(3) if lib.cmcg_slot_state(h, s) == 0]
        if queue and free:
            r = queue.pop(0)
            lib.cmcg_slot_admit(h, free[0], b.j_re[r], b.j_im[r])
            if where:
                admitted_mid += 1
            where[free[0]] = r
        for s in lib.cmcg_slot_round(h, tol, max_iter):
            e, hh, info = lib.cmcg_slot_take(h, s)
            results[where.pop(s)] = (e, hh, info)
        rounds += 1
        assert rounds < 2000
    h.close()
    assert admitted_mid >= 4  # most requests joined while others were iterating
    for r in range(6):
        ha, _ = lib.create_for_problem(
            I.Problem("one", b.mesh, b.eps, b.mu, b.omega, 2, b.j_re[r], b.j_im[r], tol), precision=P,
            stage_variant=form)
        ea, hha, ia = lib.cmcg_solve(ha, b.j_re[r], b.j_im[r], tol, max_iter)
        ha.close()
        e, hh, info = results[r]
        assert info.status == lib.CMCG_OK and info.iters == ia.iters
        scale = np.abs(np.concatenate([ea, hha], 1)).max()
        assert np.abs(e - ea).max() <= 1e-13 * scale
        assert np.abs(hh - hha).max() <= 1e-13 * scale


def test_slot_state_machine_rejects_misuse(lib):
    b = I.batched_rhs(nrhs=2, n=2, order=1)
    mesh = lib.make_mesh(b.mesh.verts, b.mesh.tets, b.mesh.tags)
    opt = lib.cmcg_default_options(order=1, precision=lib.CMCG_FP64)
    h = lib.cmcg_create_batch([(mesh, b.eps, b.mu, b.omega)] * 2, opt)
    assert lib.cmcg_slot_state(h, 0) == 0
    lib.cmcg_slot_admit(h, 0, b.j_re[0])
    assert lib.cmcg_slot_state(h, 0) == 1
    with pytest.raises(lib.CMCGError):
        lib.cmcg_slot_admit(h, 0, b.j_re[1])  # busy
    with pytest.raises(lib.CMCGError):
        lib.cmcg_slot_take(h, 0)  # not ready
    lib.cmcg_slot_round(h, 1e-6, 100)
    assert lib.cmcg_slot_state(h, 0) == 2
    h.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_checkpoint_and_resume_in_another_handle(lib, prec):
    """A request saved mid-solve (after a few CG iterations), restored into another slot of
    another handle of the same model and finished there, gives the bits of an uninterrupted solve;
    a state of another model is rejected."""
    b = I.batched_rhs(nrhs=2, n=3, order=2, tol=1e-6)
    P = lib.CMCG_FP32 if prec == "fp32" else lib.CMCG_FP64
    mesh = lib.make_mesh(b.mesh.verts, b.mesh.tets, b.mesh.tags)
    opt = lib.cmcg_default_options(order=2, precision=P, stage_variant=2 if prec == "fp32" else 1)
    h1 = lib.cmcg_create_batch([(mesh, b.eps, b.mu, b.omega)] * 2, opt)
    h2 = lib.cmcg_create_batch([(mesh, b.eps, b.mu, b.omega)] * 3, opt)

    def finish(h, slot):
        for _ in range(2000):
            if slot in lib.cmcg_slot_round(h, 1e-6, 400):
                return lib.cmcg_slot_take(h, slot)
        raise AssertionError("no result")

    lib.cmcg_slot_admit(h1, 0, b.j_re[0], b.j_im[0])
    ref = finish(h1, 0)
    lib.cmcg_slot_admit(h1, 1, b.j_re[0], b.j_im[0])
    for _ in range(5):
        lib.cmcg_slot_round(h1, 1e-6, 400)
    assert lib.cmcg_slot_state(h1, 1) == 2
    state = lib.cmcg_slot_save(h1, 1)
    assert lib.cmcg_slot_state(h1, 1) == 0
    lib.cmcg_slot_admit(h2, 0, b.j_re[1], b.j_im[1])  # other work in the target handle
    lib.cmcg_slot_round(h2, 1e-6, 400)
    lib.cmcg_slot_restore(h2, 2, state)
    assert lib.cmcg_slot_state(h2, 2) == 2
    got = finish(h2, 2)
    assert got[2].iters == ref[2].iters
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    other = I.batched_rhs(nrhs=1, n=2, order=2)
    m2 = lib.make_mesh(other.mesh.verts, other.mesh.tets, other.mesh.tags)
    h3 = lib.cmcg_create_batch([(m2, other.eps, other.mu, other.omega)], opt)
    with pytest.raises(lib.CMCGError):
        lib.cmcg_slot_restore(h3, 0, state)
    for h in (h1, h2, h3):
        h.close()
