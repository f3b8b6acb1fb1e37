"""The sharded path with two CPU ranks (gloo): halo exchange and the CG's scalar all-reduce.

Each rank owns one part of a slab partition of a mesh with PEC and impedance faces and a
permittivity jump, and builds its plan through the library (host only).  Rank r holds only
its owned values of a seeded field; one halo exchange (each rank sends the owned values the
other rank's ghosts need, in the order of that rank's plan) fills its ghosts, after which
the FP64 oracle's operator on the local mesh equals the global operator on every owned
tetrahedron (Section 5.2.2: the face fluxes need only the neighbours' traces), and an
all-reduce of the owned-only inner products (FP64, as the sharded CG does per iteration)
gives the global inner product (Eq. innerproduct).  A second test runs a whole CMCG solve on
the two ranks (a halo exchange before every RK stage, all-reduced inner products) and checks it
against the oracle's solve of the whole mesh.
"""
import json
import dataclasses
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2106_02858_gb300 import build, inputs as I
    build.build()
    from paper_2106_02858_gb300 import cmcg
    from oracle.dg import apply_B, inner
    from oracle.geometry import build_geometry
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = I.cube_problem(5, 1, 4 * math.pi, (0.3, 0.5, 0.6), (0, 1, 0), 0.2, removed=(2, 3),
                           eps_fn=lambda c: np.where(c[:, 0] > 0.45, 2.0, 1.0))
        m = cmcg.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags)
        part = cmcg.cmcg_partition_slabs(m, world, 2)
        plans = [cmcg.cmcg_shard_plan(m, part, world, q) for q in range(world)]
        me = plans[rank]
        sel, no = me["global_of_local"], me["n_owned"]
        rng = np.random.default_rng(0)
        U, V = I.random_field(rng, p.nt, 1), I.random_field(rng, p.nt, 1)  # the same seed on every rank
        loc = np.full((len(sel),) + U.shape[1:], np.nan)
        loc[:no] = U[sel[:no]]  # only the owned values are known here
        # halo exchange: send what the other rank's ghosts need (in its order), receive ours
        other = 1 - rank
        op = plans[other]
        need = op["ghost_owner_local"][op["ghost_owner_part"] == rank]
        send = torch.from_numpy(np.ascontiguousarray(loc[need]))
        mine = me["ghost_owner_part"] == other
        recv = torch.empty((int(mine.sum()),) + U.shape[1:], dtype=torch.float64)
        if rank == 0:
            dist.send(send, other)
            dist.recv(recv, other)
        else:
            dist.recv(recv, other)
            dist.send(send, other)
        loc[no:][mine] = recv.numpy()
        ghosts_exact = bool(np.array_equal(loc, U[sel]))
        g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 1)
        gl = build_geometry(p.mesh.verts, p.mesh.tets[sel], me["local_tags"], p.eps[sel], p.mu[sel], 1)
        err = float(np.abs(apply_B(loc, gl)[:no] - apply_B(U, g)[sel[:no]]).max() / np.abs(apply_B(U, g)).max())
        w = np.zeros(len(sel))
        w[:no] = 1.0
        gw = dataclasses.replace(gl, J=gl.J * w)
        s = torch.tensor([float(inner(loc, V[sel], gw))], dtype=torch.float64)
        dist.all_reduce(s)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ghosts_exact": ghosts_exact, "op_err": err, "dot": float(s.item()),
                       "ref": float(inner(U, V, g)), "n_ghost": int(len(sel) - no)}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_halo_exchange_and_scalar_all_reduce(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["n_ghost"] > 0
        assert r["ghosts_exact"]
        assert r["op_err"] <= 1e-13
        assert r["dot"] == pytest.approx(r["ref"], rel=1e-12)
    assert res[0]["dot"] == res[1]["dot"]  # the same reduced scalar on every rank


def _rank_cmcg(rank, world, port, out_dir):
    """A whole CMCG solve (Algorithms init, grad, cmcg and the filter, Sections 2.2 and 5.4) on
    two ranks: every RK stage exchanges the ghosts of its input (the oracle's operator on the
    local mesh, the global step count), every inner product is an all-reduce of owned-only
    sums.  Each rank writes its owned rows of the filtered field."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2106_02858_gb300 import build, inputs as I
    build.build()
    from paper_2106_02858_gb300 import cmcg
    from oracle import cmcg as ocmcg
    from oracle.dg import inner
    from oracle.filtering import filtered_sweep
    from oracle.geometry import build_geometry
    from oracle.timestep import Stepper
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = I.cube_problem(3, 1, 4 * math.pi, (0.4, 0.5, 0.6), (0, 1, 0), 0.2,
                           eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.0, 1.0))
        m = cmcg.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags)
        part = cmcg.cmcg_partition_slabs(m, world, 2)
        plans = [cmcg.cmcg_shard_plan(m, part, world, q) for q in range(world)]
        me, other = plans[rank], plans[1 - rank]
        sel, no = me["global_of_local"], me["n_owned"]
        need = other["ghost_owner_local"][other["ghost_owner_part"] == rank]
        mine = me["ghost_owner_part"] == 1 - rank
        g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 1)
        gl = build_geometry(p.mesh.verts, p.mesh.tets[sel], me["local_tags"], p.eps[sel], p.mu[sel], 1)
        M = Stepper(g, p.omega).M  # every part steps with the M of the whole mesh

        def exchange(X):
            X = np.array(X, copy=True)
            send = torch.from_numpy(np.ascontiguousarray(X[need]))
            recv = torch.empty((int(mine.sum()),) + X.shape[1:], dtype=torch.float64)
            if rank == 0:
                dist.send(send, 1)
                dist.recv(recv, 1)
            else:
                dist.recv(recv, 0)
                dist.send(send, 0)
            X[no:][mine] = recv.numpy()
            return X

        class ShardStepper(Stepper):
            def phi(self, j_re=None, j_im=None, adjoint=False):
                f = super().phi(j_re, j_im, adjoint)
                return lambda t, U: f(t, exchange(U))

        st = ShardStepper(gl, p.omega, M=M)
        w = np.zeros(len(sel))
        w[:no] = 1.0
        gw = dataclasses.replace(gl, J=gl.J * w)

        def dot(X, Y):
            s = torch.tensor([float(inner(X, Y, gw))], dtype=torch.float64)
            dist.all_reduce(s)
            return float(s.item())

        jr = p.j_re[sel]
        G, Gs = ocmcg.initialise(st, jr)
        U, R = np.zeros_like(Gs), Gs.copy()
        D = R.copy()
        rr = dot(R, R)
        r0 = math.sqrt(rr)
        it = 0
        while it < 200 and math.sqrt(rr) > 1e-8 * r0:
            WT = st.P(D) - D
            A = st.P_star(WT) - WT
            alpha = rr / dot(D, A)
            U, R = U + alpha * D, R - alpha * A
            rr_new = dot(R, R)
            D, rr = R + (rr_new / rr) * D, rr_new
            it += 1
        F = filtered_sweep(st, U, jr, None)
        np.save(os.path.join(out_dir, f"f{rank}.npy"), F[:no])
        np.save(os.path.join(out_dir, f"sel{rank}.npy"), sel[:no])
        with open(os.path.join(out_dir, f"c{rank}.json"), "w") as f:
            json.dump({"iters": it}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_sharded_cmcg_equals_the_whole_mesh_solve(tmp_path):
    """Halo exchange per RK stage and all-reduced FP64 inner products give the CMCG solve of the
    whole mesh: the ranks' filtered fields, put together, equal the oracle's unsharded solve to
    1e-9 (converged FP64 CG, summation order only) with the same iteration count."""
    world = 2
    mp.spawn(_rank_cmcg, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    sys.path.insert(0, ROOT)
    from paper_2106_02858_gb300 import inputs as I
    from oracle import cmcg as ocmcg
    from oracle.dg import inner
    from oracle.geometry import build_geometry
    from oracle.timestep import Stepper
    p = I.cube_problem(3, 1, 4 * math.pi, (0.4, 0.5, 0.6), (0, 1, 0), 0.2,
                       eps_fn=lambda c: np.where(c[:, 0] > 0.5, 2.0, 1.0))
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 1)
    ref = ocmcg.solve(Stepper(g, p.omega), p.j_re, None, tol=1e-8, max_iter=200)
    got = np.full_like(ref.filtered, np.nan)
    iters = []
    for r in range(world):
        got[np.load(tmp_path / f"sel{r}.npy")] = np.load(tmp_path / f"f{r}.npy")
        iters.append(json.load(open(tmp_path / f"c{r}.json"))["iters"])
    assert not np.isnan(got.real).any()
    assert iters[0] == iters[1] == ref.iters
    d = got - ref.filtered
    rel = math.sqrt(abs(inner(d, d, g)) / abs(inner(ref.filtered, ref.filtered, g)))
    assert rel <= 1e-9, rel
