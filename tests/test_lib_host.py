"""Host-side checks of libcmcg that need no GPU.

* The library loads and exports every function that ``include/cmcg.h`` declares.
* ``cmcg_validate`` rejects broken meshes and computes the same number of
  steps per period (Eq. cfl) as the oracle, bit for bit.
* ``cmcg_reference_matrices`` (monomial basis, exact simplex integrals, Duffy
  quadrature on the unit tetrahedron) equals the oracle's Dubiner-based
  matrices after the change of reference tetrahedron.
* Without a GPU, ``cmcg_create`` and ``cmcg_server_create`` fail cleanly with
  CMCG_ERR_NO_DEVICE; every entry rejects a NULL handle or server, bad options
  and empty inputs with CMCG_ERR_INVALID_ARG before touching the device.
* The product package never imports the oracle.
"""
import ast
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_02858_gb300 import build
    build.build()
    from paper_2106_02858_gb300 import cmcg
    return cmcg


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "cmcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function(lib):
    names = _declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lib.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(lib.EXPORTED) == set(names)


def _mesh(n=2):
    from paper_2106_02858_gb300 import inputs as I
    return I.kuhn_cube_mesh(n)


def test_validate_rejects_broken_meshes(lib):
    m = _mesh()
    eps, mu = np.ones(m.nt), np.ones(m.nt)
    opt = lib.cmcg_default_options(order=1)
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, mu, 2 * np.pi, opt)[0] == lib.CMCG_OK
    tags = m.tags.copy()
    tags[0, 1] = 1  # boundary tag on an interior face
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, tags), eps, mu, 2 * np.pi, opt)[0] == \
        lib.CMCG_ERR_NONCONFORMING_MESH
    tags = m.tags.copy()
    b = np.argwhere(tags > 0)[0]
    tags[b[0], b[1]] = 0  # unmatched face without tag
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, tags), eps, mu, 2 * np.pi, opt)[0] == \
        lib.CMCG_ERR_NONCONFORMING_MESH
    tets = np.concatenate([m.tets, m.tets[:1]])  # a duplicated tetrahedron: faces shared three times
    tg = np.concatenate([m.tags, m.tags[:1]])
    assert lib.cmcg_validate(lib.make_mesh(m.verts, tets, tg), np.ones(m.nt + 1), np.ones(m.nt + 1), 2 * np.pi,
                             opt)[0] == lib.CMCG_ERR_NONCONFORMING_MESH
    bad = m.tets.copy()
    bad[0, 1] = bad[0, 0]
    assert lib.cmcg_validate(lib.make_mesh(m.verts, bad, m.tags), eps, mu, 2 * np.pi, opt)[0] == lib.CMCG_ERR_INVALID_ARG
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), -eps, mu, 2 * np.pi, opt)[0] == \
        lib.CMCG_ERR_INVALID_ARG
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, mu, -1.0, opt)[0] == lib.CMCG_ERR_INVALID_ARG
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, mu, 1.0,
                             lib.cmcg_default_options(order=4))[0] == lib.CMCG_ERR_INVALID_ARG
    for bad_opt in (dict(stage_variant=-1), dict(stage_overlap=3), dict(stage_overlap=-1)):
        assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, mu, 1.0,
                                 lib.cmcg_default_options(order=1, **bad_opt))[0] == lib.CMCG_ERR_INVALID_ARG
    tags = m.tags.copy()
    tags[0, 0] = 7
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, tags), eps, mu, 1.0, opt)[0] == lib.CMCG_ERR_INVALID_ARG
    flat = m.verts.copy()
    flat[:, 2] = 0.0  # every tetrahedron degenerate
    assert lib.cmcg_validate(lib.make_mesh(flat, m.tets, m.tags), eps, mu, 1.0, opt)[0] == lib.CMCG_ERR_INVALID_ARG


@pytest.mark.parametrize("which", ["plain", "scatterer", "batched", "uneven"])
def test_steps_per_period_match_oracle(lib, which):
    from paper_2106_02858_gb300 import inputs as I
    from oracle.geometry import build_geometry
    from oracle.timestep import steps_per_period
    p = {"plain": I.plain_fp64_cube, "scatterer": I.scatterer_sphere, "batched": lambda: I.batched_rhs(nrhs=1),
         "uneven": lambda: I.uneven_batch(count=3)[2]}[which]()
    rc, M = lib.cmcg_validate(lib.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags), p.eps, p.mu, p.omega,
                              lib.cmcg_default_options(order=p.order))
    assert rc == lib.CMCG_OK
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)
    assert M == steps_per_period(g, p.omega)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_reference_matrices_match_oracle(lib, q):
    from oracle.refelem import ref_element
    M, Dr, Ds, Dt, L = lib.cmcg_reference_matrices(q)
    R = ref_element(q)
    # unit tet x = (r + 1) / 2: d/dx = 2 d/dr, dV_unit = dV_biunit / 8
    assert np.allclose(M, R.M / 8, atol=1e-14)
    assert np.allclose(Dr, 2 * R.Dr, atol=1e-11)
    assert np.allclose(Ds, 2 * R.Ds, atol=1e-11)
    assert np.allclose(Dt, 2 * R.Dt, atol=1e-11)
    # library face masses use the unit-tet face areas; the oracle's use area-2 reference triangles
    area = [np.sqrt(3) / 2, 0.5, 0.5, 0.5]
    nfp = R.Nfp
    for f in range(4):
        assert np.allclose(L[:, f * nfp:(f + 1) * nfp], 4 * area[f] * R.LIFT[:, f * nfp:(f + 1) * nfp], atol=1e-11)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = _mesh()
    with pytest.raises(lib.CMCGError) as ei:
        lib.cmcg_create(lib.make_mesh(m.verts, m.tets, m.tags), np.ones(m.nt), np.ones(m.nt), 1.0,
                        lib.cmcg_default_options())
    assert ei.value.code in (lib.CMCG_ERR_NO_DEVICE, lib.CMCG_ERR_CUDA)


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2106_02858_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                tree = ast.parse(open(os.path.join(dirpath, f)).read())
                for node in ast.walk(tree):
                    if isinstance(node, (ast.Import, ast.ImportFrom)):
                        mods = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
                        assert not any(m.split(".")[0] == "oracle" for m in mods), (f, mods)
    # and the oracle only takes the seeded input generators from the package
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            for mod in re.findall(r"from (paper_2106_02858_gb300[\w.]*) import", src):
                assert mod == "paper_2106_02858_gb300.inputs", (f, mod)


def test_every_handle_entry_rejects_a_null_handle(lib):
    """Each entry that takes a handle or a server returns CMCG_ERR_INVALID_ARG for NULL, without
    touching the device (the argument checks come before any CUDA call)."""
    L = lib._lib
    INV = lib.CMCG_ERR_INVALID_ARG
    d = np.zeros(8)
    p = d.ctypes.data_as(lib._dp)
    pp = (lib._dp * 1)(p)
    import ctypes as C
    info = lib.cmcg_info()
    calls = {
        "cmcg_set_stream": lambda: L.cmcg_set_stream(None, None),
        "cmcg_get_sizes": lambda: L.cmcg_get_sizes(None, None, None, None, None, None),
        "cmcg_get_tuning": lambda: L.cmcg_get_tuning(None, None, None),
        "cmcg_get_problem": lambda: L.cmcg_get_problem(None, 0, None, None, None),
        "dgtd_apply": lambda: L.dgtd_apply(None, 0.0, p, None, None, 0, p),
        "dgtd_period_forward": lambda: L.dgtd_period_forward(None, p, None, None, p, None, None),
        "dgtd_period_adjoint": lambda: L.dgtd_period_adjoint(None, p, p),
        "cmcg_solve": lambda: L.cmcg_solve(None, p, None, 1e-6, 10, p, p, p, p, C.byref(info)),
        "cmcg_solve_batch": lambda: L.cmcg_solve_batch(None, pp, None, 1e-6, 10, pp, pp, pp, pp, None),
        "cmcg_solve_batch_n": lambda: L.cmcg_solve_batch_n(None, 1, pp, None, 1e-6, 10, pp, pp, pp, pp, None),
        "cmcg_fw_solve": lambda: L.cmcg_fw_solve(None, p, None, 2, p, p, p, p),
        "cmcg_fw_solve_batch": lambda: L.cmcg_fw_solve_batch(None, 2, pp, None, pp, pp, pp, pp),
        "cmcg_set_boundary_data": lambda: L.cmcg_set_boundary_data(None, 0, p, None),
        "cmcg_set_conductivity": lambda: L.cmcg_set_conductivity(None, 0, p),
        "cmcg_slot_admit": lambda: L.cmcg_slot_admit(None, 0, p, None),
        "cmcg_slot_round": lambda: L.cmcg_slot_round(None, 1e-6, 10, None),
        "cmcg_slot_take": lambda: L.cmcg_slot_take(None, 0, p, p, p, p, None),
        "cmcg_slot_state": lambda: L.cmcg_slot_state(None, 0),
        "cmcg_slot_state_bytes": lambda: L.cmcg_slot_state_bytes(None, 0),
        "cmcg_slot_save": lambda: L.cmcg_slot_save(None, 0, p, 8),
        "cmcg_slot_restore": lambda: L.cmcg_slot_restore(None, 0, p, 8),
        "cmcg_solve_multifreq": lambda: L.cmcg_solve_multifreq(None, 1, (C.c_int * 1)(1), pp, None, 1e-6, 10, pp, pp,
                                                               pp, pp, None),
        "cmcg_measure_peaks": lambda: L.cmcg_measure_peaks(-1, None, None),
        "cmcg_inner": lambda: L.cmcg_inner(None, p, p, None),
        "cmcg_profile_enable": lambda: L.cmcg_profile_enable(None, 1),
        "cmcg_profile_read": lambda: L.cmcg_profile_read(None, None, None, None, None),
        "cmcg_server_add_model": lambda: L.cmcg_server_add_model(None, None, p, p, 1.0, 1, 0, None),
        "cmcg_server_submit": lambda: L.cmcg_server_submit(None, 0, p, None, None),
        "cmcg_server_poll": lambda: L.cmcg_server_poll(None, 1, 0, p, p, p, p, None, None),
        "cmcg_server_stats": lambda: L.cmcg_server_stats(None, None, None, None, None),
    }
    for name, call in calls.items():
        assert call() == INV, name
    assert L.cmcg_batch_size(None) <= 0
    assert L.cmcg_kernel_launches(None) == 0
    assert L.cmcg_device_bytes(None) == 0
    L.cmcg_destroy(None)
    L.cmcg_server_destroy(None)


def test_server_options_are_checked_before_the_device(lib):
    import torch
    for bad in (dict(max_batch=0), dict(workers=0), dict(workers=65), dict(max_wait_ms=-1.0), dict(tol=-1.0),
                dict(max_iter=-1)):
        with pytest.raises(lib.CMCGError) as ei:
            lib.cmcg_server_create(lib.cmcg_server_default_options(**bad))
        assert ei.value.code == lib.CMCG_ERR_INVALID_ARG, bad
    if not torch.cuda.is_available():
        with pytest.raises(lib.CMCGError) as ei:
            lib.cmcg_server_create(lib.cmcg_server_default_options())
        assert ei.value.code in (lib.CMCG_ERR_NO_DEVICE, lib.CMCG_ERR_CUDA)


def test_empty_and_undersized_inputs_are_rejected(lib):
    m = _mesh(1)
    eps, mu = np.ones(m.nt), np.ones(m.nt)
    opt = lib.cmcg_default_options(order=1)
    empty = lib.make_mesh(m.verts, m.tets[:0], m.tags[:0])
    assert lib.cmcg_validate(empty, eps[:0], mu[:0], 2 * np.pi, opt)[0] == lib.CMCG_ERR_INVALID_ARG
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, mu, 0.0, opt)[0] == lib.CMCG_ERR_INVALID_ARG
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, np.zeros(m.nt), 2 * np.pi, opt)[0] == \
        lib.CMCG_ERR_INVALID_ARG
    bad_opt = lib.cmcg_default_options(order=1, steps_per_period=-1)
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, mu, 2 * np.pi, bad_opt)[0] == \
        lib.CMCG_ERR_INVALID_ARG
    bad_opt = lib.cmcg_default_options(order=1, launch_graphs=3)
    assert lib.cmcg_validate(lib.make_mesh(m.verts, m.tets, m.tags), eps, mu, 2 * np.pi, bad_opt)[0] == \
        lib.CMCG_ERR_INVALID_ARG
