"""The sharded path with two CPU ranks (gloo): halo exchange and the CG's scalar all-reduce.

Each rank owns one part of a slab partition of a mesh with PEC and impedance faces and a
permittivity jump, and builds its plan through the library (host only).  Rank r holds only
its owned values of a seeded field; one halo exchange (each rank sends the owned values the
other rank's ghosts need, in the order of that rank's plan) fills its ghosts, after which
the FP64 oracle's operator on the local mesh equals the global operator on every owned
tetrahedron (Section 5.2.2: the face fluxes need only the neighbours' traces), and an
all-reduce of the owned-only inner products (FP64, as the sharded CG does per iteration)
gives the global inner product (Eq. innerproduct).
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
