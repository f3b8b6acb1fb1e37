"""Element partition and ghost layers of the sharded path, host only (no GPU).

The DG operator couples tetrahedra only through face fluxes (Section 5.2.2, Eq.
DG_semidiscrete), so a part needs the stage values of its ghosts (the other parts'
tetrahedra across its cut faces), and CMCG's inner products (Eq. innerproduct) split
into per-part sums over owned tetrahedra.  Checked here: the slab partition, the plans
(owned sets partition the mesh, ghosts are exactly the cut-face neighbours, owners and
owner-local indices agree between plans, local meshes validate), and with the FP64
oracle that the operator of a local mesh reproduces the global operator on every owned
tetrahedron once the ghosts hold their owners' values, while the owned-only inner
products add up to the global one.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    from paper_2106_02858_gb300 import build
    build.build()
    from paper_2106_02858_gb300 import cmcg
    return cmcg


def _mesh(lib):
    p = I.cube_problem(6, 2, 4 * math.pi, (0.3, 0.5, 0.6), (0, 1, 0), 0.2, removed=(2, 4),
                       eps_fn=lambda c: np.where(c[:, 2] > 0.55, 3.0, 1.0))
    return p, lib.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags)


def _face_neighbours(tets):
    from collections import defaultdict
    faces = defaultdict(list)
    for k, t in enumerate(tets):
        for f in range(4):
            faces[tuple(sorted(np.delete(t, f)))].append(k)
    nb = [set() for _ in range(len(tets))]
    for ks in faces.values():
        if len(ks) == 2:
            nb[ks[0]].add(ks[1])
            nb[ks[1]].add(ks[0])
    return nb


@pytest.mark.parametrize("nparts,axis", [(2, 2), (3, 0), (5, 1)])
def test_slab_partition_and_plans(lib, nparts, axis):
    p, m = _mesh(lib)
    part = lib.cmcg_partition_slabs(m, nparts, axis)
    counts = np.bincount(part, minlength=nparts)
    assert counts.max() - counts.min() <= 1
    cen = p.mesh.centroids()[:, axis]
    for q in range(nparts - 1):
        assert cen[part == q].max() <= cen[part == q + 1].min() + 1e-12
    nb = _face_neighbours(p.mesh.tets)
    plans = [lib.cmcg_shard_plan(m, part, nparts, q) for q in range(nparts)]
    owned = np.concatenate([pl["global_of_local"][:pl["n_owned"]] for pl in plans])
    assert np.array_equal(np.sort(owned), np.arange(p.nt))  # every tetrahedron owned exactly once
    for q, pl in enumerate(plans):
        own = pl["global_of_local"][:pl["n_owned"]]
        ghosts = pl["global_of_local"][pl["n_owned"]:]
        assert np.all(part[own] == q) and np.all(np.diff(own) > 0)
        expect = sorted({k2 for k in own for k2 in nb[k] if part[k2] != q})
        assert list(ghosts) == expect
        for g, o, ol in zip(ghosts, pl["ghost_owner_part"], pl["ghost_owner_local"]):
            assert part[g] == o and plans[o]["global_of_local"][ol] == g
        # the local mesh is a valid mesh of its own (ghosts' outer faces tagged PEC)
        loc = lib.make_mesh(p.mesh.verts, p.mesh.tets[pl["global_of_local"]], pl["local_tags"])
        opt = lib.cmcg_default_options(order=2)
        sel = pl["global_of_local"]
        rc, steps = lib.cmcg_validate(loc, p.eps[sel], p.mu[sel], p.omega, opt)
        assert rc == lib.CMCG_OK and steps > 0
        # owned tetrahedra keep their faces' tags
        assert np.array_equal(pl["local_tags"][:pl["n_owned"]], p.mesh.tags[own])


def test_plans_of_an_arbitrary_partition_and_of_one_part(lib):
    """The plan does not rely on slabs: a seeded random partition (parts interleaved, many cut
    faces, some parts without a cut face to a given other part) gives the same invariants, and a
    single part owns the whole mesh with no ghosts."""
    p, m = _mesh(lib)
    nb = _face_neighbours(p.mesh.tets)
    nparts = 4
    part = np.random.default_rng(11).integers(0, nparts, p.nt).astype(np.int32)
    plans = [lib.cmcg_shard_plan(m, part, nparts, q) for q in range(nparts)]
    for q, pl in enumerate(plans):
        own = pl["global_of_local"][:pl["n_owned"]]
        ghosts = pl["global_of_local"][pl["n_owned"]:]
        assert np.array_equal(own, np.flatnonzero(part == q))
        assert list(ghosts) == sorted({k2 for k in own for k2 in nb[k] if part[k2] != q})
        for g, o, ol in zip(ghosts, pl["ghost_owner_part"], pl["ghost_owner_local"]):
            assert part[g] == o and plans[o]["global_of_local"][ol] == g
    one = lib.cmcg_shard_plan(m, np.zeros(p.nt, dtype=np.int32), 1, 0)
    assert one["n_owned"] == p.nt and len(one["global_of_local"]) == p.nt
    assert np.array_equal(one["global_of_local"], np.arange(p.nt))
    assert np.array_equal(one["local_tags"], p.mesh.tags)


def test_local_operator_equals_global_operator_on_owned_tetrahedra(lib):
    from oracle.dg import apply_B, inner
    from oracle.geometry import build_geometry
    p, m = _mesh(lib)
    nparts = 3
    part = lib.cmcg_partition_slabs(m, nparts, 2)
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, 2)
    rng = np.random.default_rng(0)
    U, V = I.random_field(rng, p.nt, 2), I.random_field(rng, p.nt, 2)
    BU = apply_B(U, g)
    total = 0.0
    for q in range(nparts):
        pl = lib.cmcg_shard_plan(m, part, nparts, q)
        sel, no = pl["global_of_local"], pl["n_owned"]
        gl = build_geometry(p.mesh.verts, p.mesh.tets[sel], pl["local_tags"], p.eps[sel], p.mu[sel], 2)
        BUl = apply_B(U[sel], gl)
        assert np.abs(BUl[:no] - BU[sel[:no]]).max() <= 1e-12 * np.abs(BU).max()
        w = np.zeros(len(sel))
        w[:no] = 1.0
        gw = dataclasses.replace(gl, J=gl.J * w)  # ghosts carry no weight in the part's inner product
        total += float(inner(U[sel], V[sel], gw))
    ref = float(inner(U, V, g))
    assert abs(total - ref) <= 1e-12 * abs(ref)


def test_partition_arguments_are_checked(lib):
    p, m = _mesh(lib)
    with pytest.raises(lib.CMCGError):
        lib.cmcg_partition_slabs(m, 0, 2)
    with pytest.raises(lib.CMCGError):
        lib.cmcg_partition_slabs(m, 2, 3)
    part = lib.cmcg_partition_slabs(m, 2, 2)
    with pytest.raises(lib.CMCGError):
        lib.cmcg_shard_plan(m, part, 2, 2)
    bad = part.copy()
    bad[0] = 7
    with pytest.raises(lib.CMCGError):
        lib.cmcg_shard_plan(m, bad, 2, 0)
