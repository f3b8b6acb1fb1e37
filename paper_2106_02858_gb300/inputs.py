"""Seeded synthetic workloads for the CMCG hot path.

This module builds the *inputs* of a controllability solve and nothing else:
tetrahedral meshes (cubes split into Kuhn tetrahedra), boundary tags, element
permittivity / permeability, angular frequency, polynomial order and nodal
Gaussian current densities.  It holds none of the method's arithmetic (no DG
operator, no time stepping, no conjugate gradient, no filter), so both the
FP64 oracle and the CUDA path can consume it without sharing any numerics.

Boundary data layout (shared by every consumer, and documented in
``include/cmcg.h``):

* a tetrahedron's nodal field is stored ``[tet][component][node]``;
* nodes of order ``q`` are the equispaced lattice points ``(i, j, k)/q`` with
  ``i, j, k >= 0`` and ``i + j + k <= q`` of the unit reference tetrahedron
  ``(0,0,0), (1,0,0), (0,1,0), (0,0,1)``, enumerated with ``k`` outermost,
  then ``j``, then ``i`` fastest; the physical node is
  ``v0 + r (v1 - v0) + s (v2 - v0) + t (v3 - v0)``;
* face ``f`` of a tetrahedron is the face opposite its vertex ``f``;
* boundary tags: 0 interior, 1 perfectly conducting (PEC), 2 impedance
  (Silver-Mueller).

Workload shapes follow the paper's experiments (Section 6): Gaussian volume
currents ``exp(-|x - c|^2 / s^2)`` as in the trapping-medium test, piecewise
constant permittivity, impedance outer boundaries, perfectly conducting
scatterers, and Cartesian meshes cut into simplices.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

INTERIOR, PEC, IMPEDANCE = 0, 1, 2

# The six Kuhn tetrahedra of a unit cube, one per permutation of the axes:
# 0 -> e_p0 -> e_p0 + e_p1 -> (1,1,1).
KUHN_PERMS: Tuple[Tuple[int, int, int], ...] = tuple(itertools.permutations(range(3)))


def n_nodes(q: int) -> int:
    """Number of nodes of the order-q simplex lattice, (q+1)(q+2)(q+3)/6."""
    return (q + 1) * (q + 2) * (q + 3) // 6


def node_lattice(q: int) -> np.ndarray:
    """Integer lattice (i, j, k) of the order-q nodes in boundary order."""
    pts = [(i, j, k) for k in range(q + 1) for j in range(q + 1 - k) for i in range(q + 1 - k - j)]
    return np.array(pts, dtype=np.int64)


def physical_nodes(verts: np.ndarray, tets: np.ndarray, q: int) -> np.ndarray:
    """Physical coordinates of every node, shape (nt, Np, 3)."""
    rst = node_lattice(q).astype(np.float64) / q
    v = verts[tets]  # (nt, 4, 3)
    e = v[:, 1:, :] - v[:, :1, :]  # (nt, 3, 3) rows: v1-v0, v2-v0, v3-v0
    return v[:, None, 0, :] + np.einsum("nb,kbx->knx", rst, e)


@dataclass
class Mesh:
    """A conforming tetrahedral mesh with per-face boundary tags."""

    verts: np.ndarray  # (nv, 3) float64
    tets: np.ndarray  # (nt, 4) int32
    tags: np.ndarray  # (nt, 4) uint8, face f opposite vertex f
    h: float  # cube edge length

    @property
    def nt(self) -> int:
        return int(self.tets.shape[0])

    def centroids(self) -> np.ndarray:
        return self.verts[self.tets].mean(axis=1)


def kuhn_cube_mesh(n: int, removed: Optional[Tuple[int, int]] = None) -> Mesh:
    """[0,1]^3 as n^3 cubes, each cut into 6 Kuhn tetrahedra.

    Cubes are enumerated x fastest, then y, then z; each cube contributes its
    six tetrahedra in ``KUHN_PERMS`` order.  ``removed = (lo, hi)`` deletes the
    cubes whose three indices all lie in ``[lo, hi)``; faces left bare by the
    deletion are tagged PEC, the outer boundary is tagged impedance.
    """
    g = np.arange(n + 1, dtype=np.float64) / n
    vx, vy, vz = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([vx.ravel(order="F"), vy.ravel(order="F"), vz.ravel(order="F")], axis=1)

    idx = np.arange(n**3, dtype=np.int64)
    cube = np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1)  # (nc, 3), x fastest

    def is_removed(c):
        if removed is None:
            return np.zeros(c.shape[0], dtype=bool)
        lo, hi = removed
        return np.all((c >= lo) & (c < hi), axis=1)

    cube = cube[~is_removed(cube)]
    nc = cube.shape[0]

    def vid(c):
        return c[:, 0] + (n + 1) * (c[:, 1] + (n + 1) * c[:, 2])

    tets = np.empty((nc, 6, 4), dtype=np.int64)
    tags = np.zeros((nc, 6, 4), dtype=np.uint8)
    for pi, p in enumerate(KUHN_PERMS):
        a = cube.copy()
        tets[:, pi, 0] = vid(a)
        for s in range(3):
            a[:, p[s]] += 1
            tets[:, pi, s + 1] = vid(a)
        # face 0 (opposite v0) lies on the plane x_{p0} = c_{p0} + 1,
        # face 3 (opposite v3) on x_{p2} = c_{p2}; faces 1, 2 are inside the cube.
        up = cube.copy()
        up[:, p[0]] += 1
        tags[:, pi, 0] = np.where(cube[:, p[0]] + 1 == n, IMPEDANCE, np.where(is_removed(up), PEC, INTERIOR))
        dn = cube.copy()
        dn[:, p[2]] -= 1
        tags[:, pi, 3] = np.where(cube[:, p[2]] == 0, IMPEDANCE, np.where(is_removed(dn), PEC, INTERIOR))
    return Mesh(verts=verts, tets=tets.reshape(-1, 4).astype(np.int32), tags=tags.reshape(-1, 4), h=1.0 / n)


def gaussian_current(nodes: np.ndarray, centre: Sequence[float], pol: Sequence[float], width: float) -> np.ndarray:
    """Nodal values of j(x) = pol * exp(-|x - c|^2 / s^2), shape (nt, 3, Np)."""
    d2 = np.sum((nodes - np.asarray(centre)[None, None, :]) ** 2, axis=-1)  # (nt, Np)
    g = np.exp(-d2 / width**2)
    return np.asarray(pol, dtype=np.float64)[None, :, None] * g[:, None, :]


def unit_vector(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


@dataclass
class Problem:
    """One controllability solve: mesh, materials, frequency, order, source."""

    name: str
    mesh: Mesh
    eps: np.ndarray  # (nt,)
    mu: np.ndarray  # (nt,)
    omega: float
    order: int
    j_re: np.ndarray  # (nt, 3, Np) or (nrhs, nt, 3, Np)
    j_im: np.ndarray
    tol: float
    max_iter: int = 2000
    meta: dict = field(default_factory=dict)

    @property
    def nt(self) -> int:
        return self.mesh.nt

    @property
    def np_(self) -> int:
        return n_nodes(self.order)

    @property
    def ndof(self) -> int:
        return 6 * self.np_ * self.nt


def cube_problem(n: int, order: int, omega: float, centre, pol, width: float = 0.1, tol: float = 1e-8,
                 eps_fn=None, removed=None, name: str = "cube") -> Problem:
    """A Kuhn-cube problem with impedance outer boundary and one Gaussian source."""
    mesh = kuhn_cube_mesh(n, removed=removed)
    cen = mesh.centroids()
    eps = np.ones(mesh.nt) if eps_fn is None else eps_fn(cen)
    mu = np.ones(mesh.nt)
    nodes = physical_nodes(mesh.verts, mesh.tets, order)
    j_re = gaussian_current(nodes, centre, pol, width)
    return Problem(name=name, mesh=mesh, eps=eps, mu=mu, omega=omega, order=order, j_re=j_re,
                   j_im=np.zeros_like(j_re), tol=tol,
                   meta={"n": n, "centre": list(map(float, centre)), "pol": list(map(float, pol)), "width": width})


# --------------------------------------------------------------------------------------------
# The five workloads.
# --------------------------------------------------------------------------------------------

def plain_fp64_cube(n: int = 4, order: int = 1) -> Problem:
    """[0,1]^3 as 4^3 cubes x 6 Kuhn tets (384 tets), P1, eps = mu = 1, omega = 2 pi,
    impedance on every outer face, x-polarised Gaussian (width 0.1) at the centre,
    CG to relative residual 1e-8."""
    return cube_problem(n, order, 2 * np.pi, (0.5, 0.5, 0.5), (1.0, 0.0, 0.0), 0.1, tol=1e-8,
                        name=f"cube{n}_P{order}_omega2pi")


def scatterer_sphere(seed: int = 0, n: int = 24, order: int = 2, tol: float = 1e-5) -> Problem:
    """Cube 24^3 x 6 Kuhn tets minus a centred 0.25-side PEC cube (81,648 tets), P2,
    eps = 4 in a seeded sphere of radius 0.15 (elsewhere 1), mu = 1, omega = 4 pi,
    impedance outer boundary, seeded Gaussian source of width 0.1 inside the sphere."""
    rng = np.random.default_rng(seed)
    lo, hi = (3 * n) // 8, n - (3 * n) // 8  # 9..15 for n = 24: side 6/24 = 0.25
    box_lo, box_hi = lo / n, hi / n
    r = 0.15
    while True:
        c = rng.uniform(r, 1.0 - r, 3)
        d = np.linalg.norm(np.maximum(0.0, np.maximum(box_lo - c, c - box_hi)))
        if d > r:
            break
    while True:
        src = c + rng.uniform(-0.5 * r, 0.5 * r, 3)
        if np.linalg.norm(src - c) <= 0.5 * r:
            break
    pol = unit_vector(rng)

    def eps_fn(cen):
        return np.where(np.linalg.norm(cen - c[None, :], axis=1) < r, 4.0, 1.0)

    p = cube_problem(n, order, 4 * np.pi, src, pol, 0.1, tol=tol, eps_fn=eps_fn, removed=(lo, hi),
                     name=f"scatterer{n}_P{order}_omega4pi")
    p.meta.update({"sphere_centre": c.tolist(), "sphere_radius": r, "scatterer": [box_lo, box_hi], "seed": seed})
    return p


def batched_rhs(seed: int = 0, nrhs: int = 32, n: int = 4, order: int = 3, tol: float = 1e-6) -> Problem:
    """The 384-tet cube at P3, omega = 4 pi, ``nrhs`` Gaussian sources (width 0.1) at
    seeded positions with seeded unit polarisations; j has shape (nrhs, nt, 3, Np)."""
    rng = np.random.default_rng(seed)
    base = cube_problem(n, order, 4 * np.pi, (0.5, 0.5, 0.5), (1.0, 0.0, 0.0), 0.1, tol=tol,
                        name=f"cube{n}_P{order}_omega4pi_x{nrhs}")
    nodes = physical_nodes(base.mesh.verts, base.mesh.tets, order)
    centres = rng.uniform(0.2, 0.8, (nrhs, 3))
    pols = np.stack([unit_vector(rng) for _ in range(nrhs)])
    base.j_re = np.stack([gaussian_current(nodes, centres[i], pols[i], 0.1) for i in range(nrhs)])
    base.j_im = np.zeros_like(base.j_re)
    base.meta.update({"centres": centres.tolist(), "pols": pols.tolist(), "seed": seed})
    return base


def uneven_batch(seed: int = 0, count: int = 64, n_range=(6, 20), tol: float = 1e-5) -> List[Problem]:
    """``count`` independent cubes: n ~ U{6..20}, q ~ U{1,2,3}, omega ~ U{2pi, 4pi, 8pi},
    eps constant on a seeded 2x2x2 block partition drawn U[1,4], impedance outer
    boundary, one seeded Gaussian source each."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        q = int(rng.integers(1, 4))
        omega = float(rng.choice([2 * np.pi, 4 * np.pi, 8 * np.pi]))
        out.append(block_eps_problem(n, q, omega, rng, tol=tol, name=f"uneven{p}_n{n}_P{q}"))
    return out


def block_eps_problem(n: int, q: int, omega: float, rng: np.random.Generator, tol: float = 1e-5,
                      name: str = "blocks") -> Problem:
    """One problem of the uneven batch: the n^3 Kuhn cube at order q and frequency omega, eps
    constant on the 2x2x2 block partition with values drawn U[1,4] from ``rng``, impedance outer
    boundary, one Gaussian source (width 0.1) at a drawn centre with a drawn unit polarisation."""
    blocks = rng.uniform(1.0, 4.0, 8)
    centre = rng.uniform(0.2, 0.8, 3)
    pol = unit_vector(rng)

    def eps_fn(cen, blocks=blocks):
        idx = (cen[:, 0] >= 0.5).astype(int) + 2 * (cen[:, 1] >= 0.5) + 4 * (cen[:, 2] >= 0.5)
        return blocks[idx]

    prob = cube_problem(n, q, omega, centre, pol, 0.1, tol=tol, eps_fn=eps_fn, name=name)
    prob.meta.update({"blocks": blocks.tolist()})
    return prob


def block_eps_subset(shapes, seed: int = 1, tol: float = 1e-5) -> List[Problem]:
    """Problems of the uneven batch's recipe at chosen (n, q, omega) shapes, drawn from one seed."""
    rng = np.random.default_rng(seed)
    return [block_eps_problem(n, q, w, rng, tol=tol, name=f"blocks_n{n}_P{q}") for n, q, w in shapes]


@dataclass
class Request:
    arrival_s: float
    kind: str  # "small" (one P3 RHS on the 384-tet cube) or "large" (64^3 cube, P2)
    seed: int


def request_stream(seed: int = 0, count: int = 2000, rate_hz: float = 100.0, large_frac: float = 0.05) -> List[Request]:
    """Poisson arrivals: ``large_frac`` large requests, the rest batched-RHS shaped."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, count)
    t = np.cumsum(gaps)
    kinds = np.where(rng.uniform(size=count) < large_frac, "large", "small")
    seeds = rng.integers(0, 2**31 - 1, count)
    return [Request(float(t[i]), str(kinds[i]), int(seeds[i])) for i in range(count)]


def cavity_cube(n: int, order: int, omega: float) -> Problem:
    """[0,1]^3 with every outer face perfectly conducting (closed cavity), eps = mu = 1,
    no source; used for closed-form eigenmode checks."""
    mesh = kuhn_cube_mesh(n)
    mesh.tags = np.where(mesh.tags == IMPEDANCE, PEC, mesh.tags).astype(np.uint8)
    z = np.zeros((mesh.nt, 3, n_nodes(order)))
    return Problem(name=f"cavity{n}_P{order}", mesh=mesh, eps=np.ones(mesh.nt), mu=np.ones(mesh.nt),
                   omega=omega, order=order, j_re=z, j_im=z.copy(), tol=1e-8)


def random_field(rng: np.random.Generator, nt: int, q: int, batch: Tuple[int, ...] = ()) -> np.ndarray:
    """A seeded random nodal field, shape (*batch, nt, 6, Np), entries N(0,1)."""
    return rng.standard_normal(batch + (nt, 6, n_nodes(q)))
