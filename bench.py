#!/usr/bin/env python
"""Benchmark of the CMCG hot path on one GB300 (or N replicas under torchrun).

Workload: the 24^3-cube Kuhn mesh minus a centred PEC cube of side 0.25
(81,648 tetrahedra), nodal P2 (4,898,880 dofs), eps = 4 in a seeded sphere of
radius 0.15, impedance outer boundary, omega = 4 pi (242 RK4 steps per period),
seeded Gaussian source.  A step is one complete CMCG solve (Algorithms init,
grad, cmcg and the final filter) with FP32 sweeps and FP64 CG scalars, to a
relative CG residual of 1e-5; its filtered result is compared with the FP64
solve of the same problem in the same run.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CMCG solves/s at 1e-4 rel. L2 vs FP64 plain; DG dof-updates/s; p50/p99 latency"
UNIT = "solves/s"
CG_TOL = 1e-5
MAX_ITER = 2000
WORKLOAD = ("scatterer 24^3 Kuhn cube minus centred PEC cube (81,648 tets), P2 / RK4, eps=4 sphere r=0.15, "
            "impedance outer boundary, omega=4pi, seeded Gaussian source, CG rel. residual 1e-5")
# CG iterations of this workload at CG_TOL, used only to extrapolate the oracle's
# per-step time of the reference arm to a whole solve (the main arm uses the live count).
CG_ITERS_FOR_REFERENCE = 35
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "dg_stage_scatterer24_P2_fp32.md")
STAGE_SRC = os.path.join(ROOT, "paper_2106_02858_gb300", "csrc", "dg_stage.cuh")
# FP32 stage-kernel forms, indexed by cmcg_options.stage_variant - 1.
STAGE_FORMS = ["dg_stage_kernel<float, 1>", "dg_stage_kernel<float, 3>", "dg_stage_kernel<float, 4>",
               "dg_stage_quad<float, 4>", "dg_stage_quad<float, 5>", "dg_stage_quad<float, 6>",
               "dg_stage_tc (tcgen05 3xTF32)"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------------
# Oracle timing (CPU baseline / reference arm): runs in a child process, one thread.
# ---------------------------------------------------------------------------------------------

def _oracle_child(steps: int, warmup: int) -> None:
    from paper_2106_02858_gb300 import inputs as I
    from oracle.geometry import build_geometry
    from oracle.timestep import Stepper, rk4_step
    p = I.scatterer_sphere()
    g = build_geometry(p.mesh.verts, p.mesh.tets, p.mesh.tags, p.eps, p.mu, p.order)
    st = Stepper(g, p.omega)
    import numpy as np
    U = I.random_field(np.random.default_rng(0), p.nt, p.order)
    phi = st.phi()  # source-free operator, as in the 2 n_iter + 1 source-free sweeps
    times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        U, _ = rk4_step(phi, k * st.dt, U, st.dt)
        t1 = time.perf_counter()
        if k >= warmup:
            times.append(t1 - t0)
    print(json.dumps({"step_s": times, "M": st.M, "ndof": p.ndof}))


def host_cpu():
    """(logical cores, model name) of this host, from os.cpu_count() and lscpu."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_sample(steps: int, warmup: int, nproc: int = 1):
    """Times RK4 steps of the oracle in ``nproc`` concurrent single-thread processes (replicas of
    the same program on the same input); returns per-step times of every replica and M, ndof."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, "-c", f"import bench; bench._oracle_child({steps}, {warmup})"]
    procs = [subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for _ in range(nproc)]
    outs = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    return {"step_s": [o["step_s"] for o in outs], "M": outs[0]["M"], "ndof": outs[0]["ndof"]}


def oracle_rate(r):
    """Steps per second of a replica sample: every replica's steps over the slowest replica's time."""
    per = [sum(ts) for ts in r["step_s"]]
    return len(per) * len(r["step_s"][0]) / max(per)


# ---------------------------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv", "-lms", "200",
                                          "-i", str(self.gpu), "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for row in csv.reader(fh):
                if not row or row[0].strip().startswith("index"):
                    continue
                rows.append([c.strip() for c in row])
        os.unlink(self.path)
        sm = [float(re.sub(r"[^0-9.]", "", r[1])) for r in rows if re.sub(r"[^0-9.]", "", r[1])]
        smax = [float(re.sub(r"[^0-9.]", "", r[2])) for r in rows if re.sub(r"[^0-9.]", "", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# Roofline model of the stage kernel.
# ---------------------------------------------------------------------------------------------

def stage_algorithmic_bytes(nt: int, ndof: int, b: int) -> float:
    """Algorithmic bytes of one source-free RK4 stage (nested form), averaged over a step.

    Per step and dof: 11 field-vector accesses (stage 1 reads U, writes v; stages 2-4
    read v and U and write v' or U); neighbour traces are re-reads of the same
    vector, counted once.  Per tetrahedron and stage: 9 affine factors, 1/eps, 1/mu,
    4 faces x (normal + 4 flux coefficients) in the sweep precision, and 4 int32
    neighbour codes."""
    field = 11.0 / 4.0 * b * ndof
    geometry = (9 + 2 + 4 * 7) * b + 4 * 4
    return field + geometry * nt


def stage_algorithmic_flops(nt: int, q: int) -> float:
    """Algorithmic FP32 flops of one source-free nested RK4 stage (fma = 2, mul/add = 1), per
    tetrahedron: reference derivatives of 6 components in 3 directions (18 Np^2 fma), chain rule
    and curl with the material factor (12 flops per output value, 6 Np values), per face node the
    6 jumps and two fluxes (64 flops, 4 Nfp nodes), the lift of 6 components (24 Np Nfp fma) and
    the stage update (6 Np fma)."""
    np_ = (q + 1) * (q + 2) * (q + 3) // 6
    nfp = (q + 1) * (q + 2) // 2
    per_tet = 36 * np_ * np_ + 72 * np_ + 256 * nfp + 48 * np_ * nfp + 12 * np_
    return float(per_tet) * nt


# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (maximum SM clock).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def recorded_traffic(stage_variant: int):
    """Per-launch DRAM bytes of the stage kernel from the committed ncu summary, if that
    summary was taken of the same kernel form with the kernel source unchanged since; else None."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    txt = open(PROFILE_SUMMARY).read()
    m_sha = re.search(r"stage kernel source sha256:\s*([0-9a-f]{64})", txt)
    m_var = re.search(r"stage variant:\s*(\d+)", txt)
    m_tr = re.search(r"dram bytes per launch \(read \+ write\):\s*([0-9.eE+]+)", txt)
    if not (m_sha and m_tr and m_var) or int(m_var.group(1)) != stage_variant:
        return None
    sha = hashlib.sha256(open(STAGE_SRC, "rb").read()).hexdigest()
    return float(m_tr.group(1)) if sha == m_sha.group(1) else None


# ---------------------------------------------------------------------------------------------
# Replicas (N > 1): every rank solves its own problem; no data-path collective.
# ---------------------------------------------------------------------------------------------

def replica_throughput(local_s: float, steps: int, world: int, device=None):
    """Whole-job time = the slowest rank's time (MAX all-reduce of one scalar after
    the timed region), and throughput = solves of all ranks / that time."""
    total_s = float(local_s)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return total_s, steps * world / total_s


# ---------------------------------------------------------------------------------------------
# Secondary workloads: batched right-hand sides and a served request stream.
# ---------------------------------------------------------------------------------------------

def measure_batched_rhs(cmcg, I, fp32_peak=None, tf32_peak=None, reps: int = 3):
    """32 Gaussian sources on the 384-tet cube at P3 (omega = 4 pi) in one batch handle, FP32
    sweeps (kernel form chosen by timing), CG to 1e-6 per source; timed through the host-buffer
    batch entry."""
    prob = I.batched_rhs(nrhs=32)
    mesh = cmcg.make_mesh(prob.mesh.verts, prob.mesh.tets, prob.mesh.tags)
    nrhs = prob.j_re.shape[0]
    opt = cmcg.cmcg_default_options(order=prob.order, precision=cmcg.CMCG_FP32)
    h = cmcg.cmcg_create_batch([(mesh, prob.eps, prob.mu, prob.omega)] * nrhs, opt)
    form, tune = cmcg.cmcg_get_tuning(h)
    jr, ji = list(prob.j_re), list(prob.j_im)
    cmcg.cmcg_solve_batch(h, jr, ji, prob.tol, MAX_ITER)  # warm-up (captures the sweep graphs)
    cmcg.cmcg_profile_enable(h, True)
    t0 = time.perf_counter()
    for _ in range(reps):
        _e, _h, infos = cmcg.cmcg_solve_batch(h, jr, ji, prob.tol, MAX_ITER)
    dt = (time.perf_counter() - t0) / reps
    free_ms, free_stages, _sm, _ss = cmcg.cmcg_profile_read(h)
    steps = cmcg.cmcg_get_problem(h, 0)[1]
    periods = sum(3 + 2 * i.iters for i in infos)
    h.close()
    us = 1e3 * free_ms / max(free_stages, 1)
    np_, nfp = prob.np_, (prob.order + 1) * (prob.order + 2) // 2
    # the two contractions per tetrahedron and stage: volume 3 (components) x 3 Np x Np and lift
    # 3 x Np x 4 Nfp multiply-adds per E / H half, each as three TF32 products on the tensor cores
    mma_flops = 2 * 2 * 3 * (3 * np_ * np_ + np_ * 4 * nfp) * prob.nt * nrhs
    out = {"workload": "384-tet cube, P3, omega = 4 pi, 32 Gaussian sources in one handle, FP32, CG 1e-6",
           "solves_per_s": nrhs / dt, "ms_per_batch": dt * 1e3,
           "dof_updates_per_s": prob.nt * 6 * prob.np_ * steps * periods / dt,
           "cg_iters": [i.iters for i in infos][:4] + ["..."],
           "stage_form": STAGE_FORMS[form], "tuning_us": tune,
           "us_per_stage_launch": us,
           "note": "working set L2-resident: HBM fraction not meaningful"}
    if tf32_peak:
        out["tensor"] = {"achieved_tflops_3xtf32": 3 * mma_flops / (us * 1e-6) / 1e12, "peak_tf32_tflops": tf32_peak,
                         "peak_source": "measured (tcgen05 kind::tf32 loop in this run)"}
        out["tensor"]["frac"] = out["tensor"]["achieved_tflops_3xtf32"] / tf32_peak
    return out


def measure_uneven_batch(cmcg, I, hbm_peak):
    """The 64 uneven problems (n ~ U{6..20}, q ~ U{1,2,3}, omega ~ U{2,4,8} pi, eps on seeded
    2x2x2 blocks), one batch handle per order (kernel form chosen by timing), FP32, CG to 1e-5.
    One warm-up solve capped at one CG iteration captures the sweep graphs; the timed solves run
    the three handles one after the other.  HBM fraction: the stages' algorithmic bytes of the
    work each problem does (nested-form bytes for every stage: a lower bound on source stages)
    over the summed sweep time."""
    import numpy as np
    probs = I.uneven_batch()
    total_s = 0.0
    dof_updates = 0.0
    alg_bytes = 0.0
    sweep_ms = 0.0
    forms = {}
    iters = []
    for q in (1, 2, 3):
        sub = [p for p in probs if p.order == q]
        meshes = [cmcg.make_mesh(p.mesh.verts, p.mesh.tets, p.mesh.tags) for p in sub]
        opt = cmcg.cmcg_default_options(order=q, precision=cmcg.CMCG_FP32)
        h = cmcg.cmcg_create_batch([(m, p.eps, p.mu, p.omega) for m, p in zip(meshes, sub)], opt)
        forms[f"P{q}"] = STAGE_FORMS[cmcg.cmcg_get_tuning(h)[0]]
        jr, ji = [p.j_re for p in sub], [p.j_im for p in sub]
        cmcg.cmcg_solve_batch(h, jr, ji, 1e-5, 1)
        cmcg.cmcg_profile_enable(h, True)
        t0 = time.perf_counter()
        _e, _h, infos = cmcg.cmcg_solve_batch(h, jr, ji, 1e-5, MAX_ITER)
        total_s += time.perf_counter() - t0
        fm, _fs, sm, _ss = cmcg.cmcg_profile_read(h)
        sweep_ms += fm + sm
        s = 2 if q == 1 else 4
        for p, i in zip(sub, infos):
            assert i.status == cmcg.CMCG_OK, (p.name, i.status)
            per = 3 + 2 * i.iters
            dof_updates += p.ndof * i.steps_per_period * per
            field = (5.0 / 2.0 if s == 2 else 11.0 / 4.0) * 4 * p.ndof
            alg_bytes += per * i.steps_per_period * s * (field + ((9 + 2 + 4 * 7) * 4 + 16) * p.nt)
            iters.append(i.iters)
        h.close()
    achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9
    return {"workload": "64 problems: n^3 Kuhn cubes n ~ U{6..20}, P1-P3, omega in {2,4,8} pi, eps on seeded 2x2x2 "
                        "blocks U[1,4], impedance boundary, one seeded Gaussian source each; FP32, CG 1e-5; "
                        "one handle per order",
            "problems": len(probs), "dofs": int(sum(p.ndof for p in probs)),
            "solves_per_s": len(probs) / total_s, "seconds": total_s,
            "dof_updates_per_s": dof_updates / total_s, "stage_forms": forms,
            "cg_iters_min_median_max": [int(min(iters)), float(np.median(iters)), int(max(iters))],
            "hbm": {"achieved_gbs": achieved, "peak_gbs": hbm_peak, "frac": achieved / hbm_peak,
                    "note": "algorithmic bytes of the work done / summed sweep time (includes launch gaps)"}}


def measure_large_request(cmcg, I, hbm_peak):
    """The large request of the served stream at its stated size: the 64^3-cube Kuhn mesh
    (1,572,864 tets), P2 (94.4 M dofs), omega = 4 pi (644 RK4 steps per period), impedance
    boundary, one Gaussian source, FP32 sweeps, CG to 1e-6, through the host-buffer entry point.
    Its stage working set (about 1.3 GB) is far beyond L2, so the stage is HBM-bound."""
    p = I.cube_problem(64, 2, 4 * math.pi, (0.45, 0.5, 0.55), (0.0, 1.0, 0.0), 0.1, tol=1e-6)
    h, _m = cmcg.create_for_problem(p, precision=cmcg.CMCG_FP32)
    form, tune = cmcg.cmcg_get_tuning(h)
    cmcg.cmcg_profile_enable(h, True)
    t0 = time.perf_counter()
    _e, _h, info = cmcg.cmcg_solve(h, p.j_re, p.j_im, p.tol, MAX_ITER)
    dt = time.perf_counter() - t0
    fm, fs, sm, ss = cmcg.cmcg_profile_read(h)
    h.close()
    stage_us = 1e3 * fm / max(fs, 1)
    alg = stage_algorithmic_bytes(p.nt, p.ndof, 4)
    achieved = alg / (stage_us * 1e-6) / 1e9
    periods = 3 + 2 * info.iters
    return {"workload": "64^3 Kuhn cube (1,572,864 tets), P2 (94,371,840 dofs), omega = 4 pi, impedance boundary, "
                        "one Gaussian source, FP32, CG 1e-6, solved alone",
            "status": info.status, "seconds": dt, "cg_iters": info.iters, "steps_per_period": info.steps_per_period,
            "dof_updates_per_s": p.ndof * info.steps_per_period * periods / dt,
            "stage_form": STAGE_FORMS[form], "tuning_us": tune,
            "stage_us": stage_us, "source_stage_us": 1e3 * sm / max(ss, 1),
            "hbm": {"achieved_gbs": achieved, "peak_gbs": hbm_peak, "frac": achieved / hbm_peak,
                    "algorithmic_bytes_per_launch": alg}}


def measure_serving(cmcg, I, rate_hz: float = 150.0, n_small: int = 150, n_large: int = 3, seed: int = 0,
                    workers: int = 4, max_batch: int = 32, max_wait_ms: float = 5.0):
    """A Poisson stream through the serving runtime (continuous batching: `workers` threads with
    their own streams, batches of up to `max_batch`): small requests are one P3 source on the
    384-tet cube (the batched-RHS shape), large ones a 12^3-cube P2 problem; latency = submit to
    result, as the server reports it."""
    import threading
    import numpy as np
    small = I.batched_rhs(nrhs=32)
    large = I.cube_problem(12, 2, 4 * math.pi, (0.4, 0.5, 0.6), (0.0, 1.0, 0.0), 0.1, tol=1e-6)
    opt = cmcg.cmcg_server_default_options(precision=cmcg.CMCG_FP32, max_batch=max_batch, workers=workers,
                                           max_wait_ms=max_wait_ms, tol=1e-6, max_iter=MAX_ITER)
    srv = cmcg.cmcg_server_create(opt)
    ms = cmcg.make_mesh(small.mesh.verts, small.mesh.tets, small.mesh.tags)
    ml = cmcg.make_mesh(large.mesh.verts, large.mesh.tets, large.mesh.tags)
    m_small = cmcg.cmcg_server_add_model(srv, ms, small.eps, small.mu, small.omega, small.order)
    m_large = cmcg.cmcg_server_add_model(srv, ml, large.eps, large.mu, large.omega, large.order, max_batch=2)
    # warm-up: one batch of each model (graphs captured, handles pooled)
    for t in [cmcg.cmcg_server_submit(srv, m_small, small.j_re[k]) for k in range(8)]:
        cmcg.cmcg_server_poll(srv, t, m_small, wait=True)
    cmcg.cmcg_server_poll(srv, cmcg.cmcg_server_submit(srv, m_large, large.j_re), m_large, wait=True)
    rng = np.random.default_rng(seed)
    n = n_small + n_large
    kinds = np.array([0] * n_small + [1] * n_large)
    rng.shuffle(kinds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    tickets = [None] * n

    def submitter():
        t0 = time.perf_counter()
        for k in range(n):
            wait = arrivals[k] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            if kinds[k] == 0:
                tickets[k] = cmcg.cmcg_server_submit(srv, m_small, small.j_re[k % 32])
            else:
                tickets[k] = cmcg.cmcg_server_submit(srv, m_large, large.j_re)

    t_start = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat = {0: [], 1: []}
    for k in range(n):
        r = cmcg.cmcg_server_poll(srv, tickets[k], m_small if kinds[k] == 0 else m_large, wait=True)
        lat[int(kinds[k])].append(r[4])
    wall = time.perf_counter() - t_start
    stats = cmcg.cmcg_server_stats(srv)
    srv.close()
    # the same small request as a serial FP64 plain solve, for comparison
    h64, _m = cmcg.create_for_problem(small, precision=cmcg.CMCG_FP64)
    cmcg.cmcg_solve(h64, small.j_re[0], None, 1e-6, MAX_ITER)
    t0 = time.perf_counter()
    cmcg.cmcg_solve(h64, small.j_re[1], None, 1e-6, MAX_ITER)
    fp64_s = time.perf_counter() - t0
    h64.close()
    alls = lat[0] + lat[1]
    pct = lambda xs, q: float(np.percentile(xs, q)) if xs else None
    return {"workload": f"Poisson {rate_hz:g}/s: {n_small} small (384-tet cube P3, one source) + {n_large} "
                        f"large (10,368-tet cube P2) requests, FP32, CG 1e-6, {workers} workers, "
                        f"batches <= {max_batch}, window {max_wait_ms:g} ms",
            "offered_per_s": rate_hz,
            "solves_per_s": n / wall, "p50_ms": pct(alls, 50), "p99_ms": pct(alls, 99),
            "small_p50_ms": pct(lat[0], 50), "small_p99_ms": pct(lat[0], 99),
            "large_p50_ms": pct(lat[1], 50), "serial_fp64_plain_small_solves_per_s": 1.0 / fp64_s,
            "handles": stats["handles"],
            "device_bytes": stats["bytes_in_use"]}


# ---------------------------------------------------------------------------------------------
# Arms.
# ---------------------------------------------------------------------------------------------

def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    cores, model = host_cpu()
    r = oracle_sample(args.steps, args.warmup, nproc=cores)
    steps_per_s = oracle_rate(r)
    steps_per_solve = r["M"] * (3 + 2 * CG_ITERS_FOR_REFERENCE)
    value = steps_per_s / steps_per_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * max(sum(ts) for ts in r["step_s"]) / args.steps,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": f"host CPU, {cores} single-thread oracle processes"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
                         "sample": f"each step = one RK4 step (4 operator applications) of the FP64 numpy oracle on "
                                   f"the full 81,648-tet P2 mesh in each of {cores} concurrent single-thread "
                                   f"processes; solves/s = replicas x steps / slowest replica's time / (M x "
                                   f"(3 + 2 x {CG_ITERS_FOR_REFERENCE})) with M = {r['M']}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "dof_updates_per_s": r["ndof"] * steps_per_s,
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02858_gb300 import cmcg, inputs as I

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = I.scatterer_sphere(seed=args.seed + rank)
    h32, _m32 = cmcg.create_for_problem(prob, precision=cmcg.CMCG_FP32, device=local_rank,
                                        stage_variant=args.stage_variant)
    stream = torch.cuda.current_stream(dev)
    cmcg.cmcg_set_stream(h32, stream)
    jr = torch.from_numpy(prob.j_re).to(dev)
    ji = torch.from_numpy(prob.j_im).to(dev)
    outs = [torch.empty(prob.nt, 3, prob.np_, dtype=torch.float64, device=dev) for _ in range(4)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def solve():
        return cmcg.cmcg_solve_device(h32, jr, ji, CG_TOL, MAX_ITER, *outs)

    for _ in range(args.warmup):
        info = solve()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local_rank)
    sampler.start()
    cmcg.cmcg_profile_enable(h32, True)
    launches0 = cmcg.cmcg_kernel_launches(h32)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    infos = []
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        infos.append(solve())
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    launches = cmcg.cmcg_kernel_launches(h32) - launches0
    free_ms, free_stages, src_ms, src_stages = cmcg.cmcg_profile_read(h32)
    cmcg.cmcg_profile_enable(h32, False)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s, value = replica_throughput(sum(step_ms) / 1e3, args.steps, world, dev)
    iters = infos[-1].iters
    periods = 3 + 2 * iters
    dof_updates = prob.ndof * h32.steps * periods
    e32 = [o.cpu().numpy() for o in outs]

    # e2e: the host-buffer entry point, pinned inputs copied in and results read back every step.
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    jr_h, ji_h = pin(prob.j_re), pin(prob.j_im)
    e2e_ms = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        cmcg.cmcg_solve(h32, jr_h, ji_h, CG_TOL, MAX_ITER)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total, e2e_value = replica_throughput(sum(e2e_ms) / 1e3, len(e2e_ms), world, dev)
    nj = prob.nt * 3 * prob.np_ * 8
    h2d, d2h = 2 * nj, 4 * nj

    # The paper's comparison method at equal cost: the limiting-amplitude iteration (FW) run for
    # as many periods as one CMCG solve simulates, and its distance from the CMCG result.
    fw = None
    if not args.skip_fw:
        fw_periods = 3 + 2 * infos[-1].iters - 1  # FW simulates periods + 1
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        efw, hfw = cmcg.cmcg_fw_solve(h32, jr_h, ji_h, fw_periods)
        fw_s = time.perf_counter() - t0
        ecg, hcg = e32[0] + 1j * e32[1], e32[2] + 1j * e32[3]
        fwf = np.concatenate([efw, hfw], axis=1)
        cgf = np.concatenate([ecg, hcg], axis=1)
        d = fwf - cgf
        num = cmcg.cmcg_inner(h32, d.real, d.real) + cmcg.cmcg_inner(h32, d.imag, d.imag)
        den = cmcg.cmcg_inner(h32, cgf.real, cgf.real) + cmcg.cmcg_inner(h32, cgf.imag, cgf.imag)
        fw = {"periods": fw_periods + 1, "seconds": fw_s, "rel_l2_vs_cmcg": math.sqrt(num / den)}

    # FP64 plain solve of the same problem: accuracy of the FP32 result and the FP64 rate.
    fp64 = None
    if not args.skip_fp64:
        h64, _m64 = cmcg.create_for_problem(prob, precision=cmcg.CMCG_FP64, device=local_rank)
        cmcg.cmcg_set_stream(h64, stream)
        outs64 = [torch.empty_like(o) for o in outs]
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info64 = cmcg.cmcg_solve_device(h64, jr, ji, CG_TOL, MAX_ITER, *outs64)
        b.record(stream)
        torch.cuda.synchronize(dev)
        e64 = [o.cpu().numpy() for o in outs64]
        # (e, h) -> full (nt, 6, Np) real and imaginary parts
        re32, im32 = np.concatenate([e32[0], e32[2]], axis=1), np.concatenate([e32[1], e32[3]], axis=1)
        re64, im64 = np.concatenate([e64[0], e64[2]], axis=1), np.concatenate([e64[1], e64[3]], axis=1)
        dr, di = re32 - re64, im32 - im64
        num = cmcg.cmcg_inner(h64, dr, dr) + cmcg.cmcg_inner(h64, di, di)
        den = cmcg.cmcg_inner(h64, re64, re64) + cmcg.cmcg_inner(h64, im64, im64)
        fp64 = {"rel_l2": math.sqrt(num / den), "ms": a.elapsed_time(b), "iters": info64.iters}
        h64.close()

    # Roofline of the stage kernel over the timed region (source-free sweeps).
    peak, peak_kind = peaks()
    fp32_peak, tf32_peak = cmcg.cmcg_measure_peaks(local_rank)
    stage_us = free_ms * 1e3 / max(free_stages, 1)
    alg = stage_algorithmic_bytes(prob.nt, prob.ndof, 4)
    achieved = alg / (stage_us * 1e-6) / 1e9
    form, form_us = cmcg.cmcg_get_tuning(h32)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(form + 1), "kernel": f"{STAGE_FORMS[form]} (P2, nested RK4 stage)",
                "stage_variant": form + 1, "tuning_us": form_us,
                "alu": {"achieved": stage_algorithmic_flops(prob.nt, prob.order) / (stage_us * 1e-6) / 1e12,
                        "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": stage_algorithmic_flops(prob.nt, prob.order) / (stage_us * 1e-6) / 1e12
                        / fp32_peak, "peak_source": "measured (FP32 FMA loop in this run)",
                        "tf32_tensor_peak_tflops": tf32_peak,
                        "nominal_fp32_tflops": FP32_PEAK_TFLOPS},
                "algorithmic_bytes_per_launch": alg, "avg_launch_us": stage_us, "peak_source": peak_kind,
                "source_stage_us": src_ms * 1e3 / max(src_stages, 1)}

    batched = serving = uneven = large = None
    if rank == 0 and not args.skip_extra:
        batched = measure_batched_rhs(cmcg, I, fp32_peak, tf32_peak)
        uneven = measure_uneven_batch(cmcg, I, peak)
        serving = [measure_serving(cmcg, I, rate_hz=r, n_small=n - n // 20, n_large=n // 20, seed=k)
                   for k, (r, n) in enumerate(((20.0, 200), (40.0, 300), (80.0, 400), (160.0, 600)))]
        if not args.skip_large:
            large = measure_large_request(cmcg, I, peak)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cores, model = host_cpu()
        one = oracle_sample(2, 0, nproc=1)
        rate1 = oracle_rate(one)
        allc = oracle_sample(1, 0, nproc=cores)
        rate_all = oracle_rate(allc)
        steps_per_solve = h32.steps * periods
        cpu = {"value": rate_all / steps_per_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
               "cpu_model": model,
               "sample": f"RK4 steps (4 operator applications each) of the FP64 numpy oracle on the full mesh in "
                         f"{cores} concurrent single-thread processes (one step each); solves/s = steps per "
                         f"second / ({h32.steps} steps x {periods} periods, {iters} CG iterations)",
               "dof_updates_per_s": one["ndof"] * rate_all,
               "single_thread": {"value": rate1 / steps_per_solve, "unit": UNIT, "cores": 1,
                                 "sample": "2 RK4 steps in one single-thread process",
                                 "dof_updates_per_s": one["ndof"] * rate1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tets": prob.nt, "order": prob.order, "dofs": prob.ndof,
                       "steps_per_period": h32.steps, "cg_tol": CG_TOL, "sweep_precision": "fp32",
                       "cg_scalars": "fp64", "l2": "256 MiB buffer written between timed solves",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "cg_iters": iters, "periods_per_solve": periods,
            "dof_updates_per_s": dof_updates * args.steps * world / total_s,
            "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
            "rel_l2_vs_fp64": fp64["rel_l2"] if fp64 else None,
            "fp64_plain_solves_per_s": 1e3 / fp64["ms"] if fp64 else None,
            "fp64_plain_iters": fp64["iters"] if fp64 else None,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "clocks": clocks,
            "fw_at_equal_periods": fw,
            "batched_rhs": batched,
            "uneven_batch": uneven,
            "serving": serving,
            "serving_large_request": large,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h32.close()


def profile_sweep(args):
    """One source-free FP32 period sweep of the benchmark workload (968 stage launches);
    the command profiled by ncu for the stage kernel."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02858_gb300 import cmcg, inputs as I
    prob = I.scatterer_sphere(seed=args.seed)
    h, _m = cmcg.create_for_problem(prob, precision=cmcg.CMCG_FP32, stage_variant=args.stage_variant)
    dev = torch.device("cuda:0")
    u0 = torch.from_numpy(I.random_field(np.random.default_rng(0), prob.nt, prob.order)).to(dev)
    uT = torch.empty_like(u0)
    cmcg.dgtd_period_forward_device(h, u0, None, None, uT)
    torch.cuda.synchronize()
    print(json.dumps({"profile_sweep": "done", "launches": cmcg.cmcg_kernel_launches(h),
                      "tuning": cmcg.cmcg_get_tuning(h)}))
    h.close()


def profile_batched(args):
    """The 32-source P3 batch on the 384-tet cube (12,288 tetrahedra per stage launch) with a
    forced stage form: one solve capped at one CG iteration (4 sweeps: source, adjoint, and the
    iteration's two, plus the filtered sweep); the command profiled by ncu for the tensor-core form."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02858_gb300 import cmcg, inputs as I
    prob = I.batched_rhs(nrhs=32)
    mesh = cmcg.make_mesh(prob.mesh.verts, prob.mesh.tets, prob.mesh.tags)
    opt = cmcg.cmcg_default_options(order=prob.order, precision=cmcg.CMCG_FP32, stage_variant=args.stage_variant)
    h = cmcg.cmcg_create_batch([(mesh, prob.eps, prob.mu, prob.omega)] * 32, opt)
    cmcg.cmcg_solve_batch(h, list(prob.j_re), list(prob.j_im), prob.tol, 1)
    print(json.dumps({"profile_batched": "done", "launches": cmcg.cmcg_kernel_launches(h),
                      "tuning": cmcg.cmcg_get_tuning(h)}))
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fw", action="store_true")
    ap.add_argument("--skip-extra", action="store_true", help="skip the batched-RHS, uneven-batch and serving measurements")
    ap.add_argument("--skip-large", action="store_true", help="skip the 64^3-cube P2 request")
    ap.add_argument("--profile-sweep", action="store_true", help="run one period sweep only (for ncu)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="one capped solve of the 32-source P3 batch only (for ncu)")
    ap.add_argument("--stage-variant", type=int, default=0, help="force a stage-kernel form (see cmcg_options)")
    args = ap.parse_args()
    if args.profile_sweep:
        profile_sweep(args)
        return
    if args.profile_batched:
        profile_batched(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
