"""Mesh geometry and connectivity (oracle).

Section 5.2.2 of the paper: a conforming simplicial mesh T_h, its faces F_h
split into interior faces, PEC faces and impedance faces, a normal per face
that is outward on the boundary, and rho_K, the diameter of the largest ball
inscribed in K (used by the CFL condition, Eq. cfl).

Everything here is done the plain way: faces are matched by their sorted
global vertex triples, face nodes are matched by their physical coordinates,
normals come from cross products oriented away from the opposite vertex.
Test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

from paper_2106_02858_gb300.inputs import INTERIOR, PEC, IMPEDANCE, physical_nodes
from .refelem import FACE_VERTS, ref_element


@dataclass
class Geometry:
    q: int
    nt: int
    J: np.ndarray  # (nt,) |d x / d (r,s,t)| for the bi-unit reference map
    G: np.ndarray  # (nt, 3, 3) G[k, b, a] = d r_b / d x_a
    normals: np.ndarray  # (nt, 4, 3) outward unit normals
    area: np.ndarray  # (nt, 4) face areas
    sJ: np.ndarray  # (nt, 4) face area / reference face area (2)
    volume: np.ndarray  # (nt,)
    rho: np.ndarray  # (nt,) inscribed-ball diameter
    nbr: np.ndarray  # (nt, 4) neighbour tet or -1
    nbr_face: np.ndarray  # (nt, 4) neighbour's face index or -1
    mapP: np.ndarray  # (nt, 4, Nfp) neighbour's volume node matching each own face node (or own node on boundary)
    bc: np.ndarray  # (nt, 4) INTERIOR / PEC / IMPEDANCE
    eps: np.ndarray
    mu: np.ndarray
    nodes: np.ndarray  # (nt, Np, 3)
    sigma: Optional[np.ndarray] = None  # (nt,) conductivity (Eq. maxwell_time_strong, Section 1; coefficients Section 3.1); None = 0


class MeshError(ValueError):
    pass


def build_geometry(verts, tets, tags, eps, mu, q: int, sigma=None) -> Geometry:
    R = ref_element(q)
    verts = np.asarray(verts, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    tags = np.asarray(tags, dtype=np.int64)
    nt = tets.shape[0]
    v = verts[tets]  # (nt, 4, 3)
    A = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)  # columns are edges
    detA = np.linalg.det(A)
    if np.any(np.abs(detA) <= 0):
        raise MeshError("degenerate tetrahedron")
    volume = np.abs(detA) / 6.0
    # bi-unit map x = v0 + (1+r)/2 (v1-v0) + ...: dx/d(r,s,t) = A/2
    J = np.abs(detA) / 8.0
    G = np.linalg.inv(A / 2.0)  # G[k, b, a] = d r_b / d x_a

    normals = np.zeros((nt, 4, 3))
    area = np.zeros((nt, 4))
    for f in range(4):
        a, b, c = FACE_VERTS[f]
        cr = np.cross(v[:, b] - v[:, a], v[:, c] - v[:, a])
        ar = 0.5 * np.linalg.norm(cr, axis=1)
        sgn = np.sign(np.einsum("kx,kx->k", cr, v[:, f] - v[:, a]))
        normals[:, f] = -sgn[:, None] * cr / (2.0 * ar[:, None])
        area[:, f] = ar
    rho = 6.0 * volume / area.sum(axis=1)

    # Face matching by sorted vertex triples.
    keys = np.sort(np.stack([tets[:, list(FACE_VERTS[f])] for f in range(4)], axis=1), axis=2)  # (nt,4,3)
    flat = keys.reshape(-1, 3)
    order = np.lexsort((flat[:, 2], flat[:, 1], flat[:, 0]))
    sk = flat[order]
    same = np.all(sk[1:] == sk[:-1], axis=1)
    if np.any(same[1:] & same[:-1]):
        raise MeshError("a face is shared by more than two tetrahedra")
    nbr = -np.ones(nt * 4, dtype=np.int64)
    pair = np.nonzero(same)[0]
    i0, i1 = order[pair], order[pair + 1]
    nbr[i0], nbr[i1] = i1, i0
    nbr_tet = np.where(nbr >= 0, nbr // 4, -1).reshape(nt, 4)
    nbr_face = np.where(nbr >= 0, nbr % 4, -1).reshape(nt, 4)

    bc = np.where(nbr_tet >= 0, INTERIOR, tags)
    if np.any((nbr_tet >= 0) & (tags != INTERIOR)):
        raise MeshError("boundary tag on an interior face")
    if np.any((nbr_tet < 0) & (tags != PEC) & (tags != IMPEDANCE)):
        raise MeshError("unmatched face without a boundary tag")

    # Node matching across interior faces by physical coordinates.
    nodes = physical_nodes(verts, tets, q)
    Fm = R.Fmask
    mapP = np.broadcast_to(Fm[None], (nt, 4, R.Nfp)).copy()
    kk, ff = np.nonzero(nbr_tet >= 0)
    own = nodes[kk[:, None], Fm[ff]]  # (nf, Nfp, 3)
    oth = nodes[nbr_tet[kk, ff][:, None], Fm[nbr_face[kk, ff]]]  # (nf, Nfp, 3)
    d = np.linalg.norm(own[:, :, None, :] - oth[:, None, :, :], axis=-1)  # (nf, Nfp, Nfp)
    j = np.argmin(d, axis=2)
    if np.any(np.take_along_axis(d, j[:, :, None], axis=2) > 1e-9):
        raise MeshError("non-conforming face nodes")
    mapP[kk, ff] = Fm[nbr_face[kk, ff]][np.arange(len(kk))[:, None], j]

    return Geometry(q=q, nt=nt, J=J, G=G, normals=normals, area=area, sJ=area / 2.0, volume=volume, rho=rho,
                    nbr=nbr_tet, nbr_face=nbr_face, mapP=mapP, bc=bc, eps=np.asarray(eps, np.float64),
                    mu=np.asarray(mu, np.float64), nodes=nodes,
                    sigma=None if sigma is None else np.asarray(sigma, np.float64))
