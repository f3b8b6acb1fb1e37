"""Host-side checks of bench.py's bookkeeping (no GPU).

* Algorithmic bytes of a nested RK4 stage: 11/4 field-vector accesses per dof (stage 1 reads U,
  writes v; stages 2-4 read v and U and write), plus the per-tetrahedron geometry, counted by
  hand for P2 FP32: 2.75 * 4 * 60 = 660 B of fields and (9 + 2 + 28) * 4 + 16 = 172 B of
  geometry per tetrahedron.
* Algorithmic flops of a stage, counted term by term for P1 and P2 from the operator's parts.
* The roofline's traffic is read from the committed ncu summary only when the summary names the
  same kernel form and the same kernel source; otherwise it is null.
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_stage_bytes_by_hand():
    nt = 1000
    ndof = nt * 60
    assert bench.stage_algorithmic_bytes(nt, ndof, 4) == nt * (660 + 172)
    assert bench.stage_algorithmic_bytes(81648, 81648 * 60, 4) == 81648 * 832


def test_stage_flops_by_hand():
    def by_hand(np_, nfp):
        volume = 6 * 3 * np_ * np_ * 2          # reference derivatives, fma = 2
        curl = 6 * np_ * (2 * 5 + 1 + 1)        # two 3-term physical derivatives, difference, 1/eps
        faces = 4 * nfp * 2 * (3 + 29)          # per face node and half: 3 jumps, two fluxes' 29 flops
        lift = 6 * np_ * 4 * nfp * 2
        update = 6 * np_ * 2
        return volume + curl + faces + lift + update
    assert bench.stage_algorithmic_flops(1, 1) == by_hand(4, 3) == 2256
    assert bench.stage_algorithmic_flops(1, 2) == by_hand(10, 6) == 8856
    assert bench.stage_algorithmic_flops(81648, 2) == 81648 * 8856


def test_recorded_traffic_needs_the_same_form_and_source(tmp_path, monkeypatch):
    src = open(bench.STAGE_SRC, "rb").read()
    sha = hashlib.sha256(src).hexdigest()
    summary = tmp_path / "p.md"
    summary.write_text(f"stage kernel source sha256: {sha}\nstage variant: 2\n"
                       "dram bytes per launch (read + write): 4.9e7\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    assert bench.recorded_traffic(2) == 4.9e7
    assert bench.recorded_traffic(3) is None
    summary.write_text("stage kernel source sha256: " + "0" * 64 + "\nstage variant: 2\n"
                       "dram bytes per launch (read + write): 4.9e7\n")
    assert bench.recorded_traffic(2) is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.recorded_traffic(2) is None
