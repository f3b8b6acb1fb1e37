"""The allocation-free inner product against the handle-based one (GPU).

``cmcg_inner_noalloc`` is for callers that cannot call cudaMalloc where they
need the (eps, mu) inner product: their device memory belongs to their own pool
allocator, an allocation would synchronise their stream-ordered pipeline, or
they hold no handle (``cmcg_create`` allocates).  It reduces through a static
device array instead of an allocated buffer.  Two calls in a row on the same
stream, on meshes of different sizes (the larger first, so the second finds
the first's partial sums in the shared array), must agree with ``cmcg_inner``
and with the FP64 oracle's inner product (Eq. innerproduct, on meshes with
permittivity jumps) to the rounding of an FP64 reduction (1e-12 relative).
Sizes beyond the array are rejected before anything is launched.
"""
import math

import numpy as np
import pytest

from paper_2106_02858_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _weights(p):
    """(eps, mu) times |det(v1 - v0, v2 - v0, v3 - v0)| per tetrahedron."""
    v = p.mesh.verts[p.mesh.tets]
    A = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    d = np.abs(np.linalg.det(A))
    return np.ascontiguousarray(np.stack([d * p.eps, d * p.mu], axis=1))


def test_noalloc_inner_matches_handle_inner_on_two_calls():
    from paper_2106_02858_gb300 import build
    build.build()
    import torch
    from paper_2106_02858_gb300 import cmcg
    assert torch.cuda.is_available(), "needs a CUDA device"
    dev = torch.device("cuda:0")
    probs = [I.cube_problem(7, 2, 4 * math.pi, (0.5, 0.5, 0.5), (1, 0, 0), 0.2,
                            eps_fn=lambda c: np.where(c[:, 2] > 0.4, 3.0, 1.0)),
             I.cube_problem(3, 3, 2 * math.pi, (0.5, 0.5, 0.5), (0, 1, 0), 0.2,
                            eps_fn=lambda c: 1.0 + c[:, 0])]
    from oracle.dg import inner as oracle_inner
    from oracle.geometry import build_geometry
    rng = np.random.default_rng(4)
    args, expected, oracle_vals = [], [], []
    for p in probs:
        u = I.random_field(rng, p.nt, p.order)
        v = I.random_field(rng, p.nt, p.order)
        h, _m = cmcg.create_for_problem(p, precision=cmcg.CMCG_FP64)
        expected.append(cmcg.cmcg_inner(h, u, v))
        h.close()
        g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)
        oracle_vals.append(float(oracle_inner(u, v, g)))
        args.append((p.order, p.nt, torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev),
                     torch.from_numpy(_weights(p)).to(dev), torch.zeros(1, dtype=torch.float64, device=dev)))
    stream = torch.cuda.current_stream(dev)
    for order, nt, u, v, w, out in args:  # two calls in a row on one stream
        cmcg.cmcg_inner_noalloc(order, nt, u, v, w, out, stream)
    torch.cuda.synchronize(dev)
    for (order, nt, u, v, w, out), ref, orc in zip(args, expected, oracle_vals):
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
        # both entry points against the oracle's (eps, mu) inner product
        assert abs(got - orc) <= 1e-12 * abs(orc), (got, orc)
        assert abs(ref - orc) <= 1e-12 * abs(orc), (ref, orc)

    order, nt, u, v, w, out = args[1]
    with pytest.raises(cmcg.CMCGError) as ei:
        cmcg.cmcg_inner_noalloc(order, cmcg.CMCG_NOALLOC_MAX_TETS + 1, u, v, w, out, stream)
    assert ei.value.code == cmcg.CMCG_ERR_INVALID_ARG
    assert "static scratch" in str(ei.value)
