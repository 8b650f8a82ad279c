"""Host logic of the bench that feeds its roofline object: the committed DRAM
traffic record is used only while the quadrature kernel sources are the ones
it was captured on, and the peak falls back when the measured file lacks it."""
import json
import os
import shutil
import time

import pytest

import bench

SOURCES = ("nl_quad.cuh", "nl_assemble.cuh", "nl_assemble32.cu")


@pytest.fixture()
def fake_root(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2302_07499_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2302_07499_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _write_record(root, sha, value=1.5e9):
    rec = {"source_sha": sha, "dram_bytes_per_step": value}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))


def test_traffic_record_used_while_sources_match(fake_root):
    _write_record(fake_root, bench._kernel_source_sha())
    assert bench._traffic_record() == 1.5e9


def test_traffic_record_dropped_once_a_source_changes(fake_root):
    _write_record(fake_root, bench._kernel_source_sha())
    for f in SOURCES:
        p = fake_root / "paper_2302_07499_gb300" / "csrc" / f
        orig = p.read_bytes()
        p.write_bytes(orig + b"\n")
        assert bench._traffic_record() is None, f
        p.write_bytes(orig)
    assert bench._traffic_record() == 1.5e9


def test_traffic_record_missing_or_malformed(fake_root):
    assert bench._traffic_record() is None
    (fake_root / "profiles" / "traffic.json").write_text("{not json")
    assert bench._traffic_record() is None


def test_committed_traffic_record_is_consistent():
    """The committed record scales the captured launch's bytes by the ratio of
    cut events it states, so its per-step figure follows from its own fields,
    and it was taken on the current kernel sources."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    cap = rec["dram_read_bytes_captured"] + rec["dram_write_bytes_captured"]
    want = cap * rec["cut_points_per_step"] / rec["cut_points_captured"]
    assert abs(rec["dram_bytes_per_step"] - want) <= 1e-9 * want
    assert rec["source_sha"] == bench._kernel_source_sha()
    assert len(rec["source_sha"]) == 16


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._measured_peak("hbm_gbs", 6800.0) == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    assert bench._measured_peak("hbm_gbs", 6800.0) == (7000.5, "measured")
    assert bench._measured_peak("bf16_tflops", 1900.0) == (1900.0, "fallback")


def test_quadrature_ops_counts_each_unit_once():
    """Each counted unit adds its own per-unit operation figure: pairs carry
    four outer points each, and the cut-point work adds linearly."""
    zero = dict(pairs=0, cut_points=0, mc_samples=0, mc_accepted=0)
    assert bench._quadrature_ops(zero) == 0
    for key, per in (("cut_points", bench.OPS_PER_CUT), ("mc_samples", bench.OPS_PER_SAMPLE),
                     ("mc_accepted", bench.OPS_PER_ACCEPTED), ("pairs", 4 * bench.OPS_PER_PAIR_POINT)):
        st = dict(zero, **{key: 1000})
        assert bench._quadrature_ops(st) == 1000 * per, key
    st = dict(pairs=3, cut_points=5, mc_samples=7, mc_accepted=2)
    parts = sum(bench._quadrature_ops(dict(zero, **{k: v})) for k, v in st.items())
    assert bench._quadrature_ops(st) == parts


def _fake_smi(dirpath, rows):
    script = dirpath / "nvidia-smi"
    body = "\n".join("echo '%s'; sleep 0.02" % r for r in rows)
    script.write_text("#!/bin/sh\n%s\nexec sleep 30\n" % body)
    script.chmod(0o755)


def test_clock_sampler_parses_rows_and_reasons(tmp_path, monkeypatch):
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage"]
    _fake_smi(tmp_path, rows)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    c = s.stop()
    assert c["samples"] == 3                    # malformed rows are skipped
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_entry_errors_metric():
    """The bench's per-entry error: relative to the entry, with the floors
    for near-zero entries (1e-3 of the diagonals' geometric mean, 1e-7 of the
    largest diagonal)."""
    import numpy as np
    rp = np.array([0, 2, 4])
    ci = np.array([0, 1, 0, 1])
    ref = np.array([4.0, 1e-9, 1e-9, 1.0])
    got = ref * np.array([1 + 1e-6, 1.0, 1.0, 1.0]) + np.array([0.0, 2e-6, 0.0, 0.0])
    e = bench.entry_errors((rp, ci, got), (rp, ci, ref))
    assert abs(e[0] - 1e-6) < 1e-15
    assert abs(e[1] - 2e-6 / (1e-3 * 2.0)) < 1e-12          # floor: 1e-3 sqrt(4 * 1)
    assert e[2] == 0.0 and e[3] == 0.0


def test_l2_error_of_the_interpolant_of_the_quadratic():
    """For u = |x|^2 the P1 interpolant's error on an element is
    sum_{i<j} lambda_i lambda_j |v_i - v_j|^2; its square integrates exactly
    from the monomial integrals of the barycentrics, which the bench's
    degree-5 rule must reproduce."""
    import math
    import numpy as np
    import nl_inputs as I
    mesh = I.kuhn_box(-0.25, 1.25, 6, jitter_frac=0.2, seed=5)
    u = (mesh.verts ** 2).sum(axis=1)
    got = bench.l2_error_quadratic(mesh, u)

    def mono(alpha, vol):
        return vol * 6.0 * math.prod(math.factorial(a) for a in alpha) / math.factorial(sum(alpha) + 3)
    pairs = [(i, j) for i in range(4) for j in range(i + 1, 4)]
    want = 0.0
    for t in np.nonzero(mesh.tet_in_omega)[0]:
        v = mesh.verts[mesh.tets[t]]
        vol = abs(np.linalg.det(v[1:] - v[0])) / 6
        c = {p: float(np.sum((v[p[0]] - v[p[1]]) ** 2)) for p in pairs}
        for p in pairs:
            for r in pairs:
                alpha = [0, 0, 0, 0]
                for k in p + r:
                    alpha[k] += 1
                want += c[p] * c[r] * mono(alpha, vol)
    assert abs(got - math.sqrt(want)) <= 1e-12 * math.sqrt(want)
