"""Host-side logic of bench.py that needs no GPU: the reference arm (the
oracle timed on the host cores) and its JSON line, the DRAM-traffic lookup in
the committed ncu summary (returned only while the kernel's sources are the
ones that were profiled), the measured HBM peak, and the oracle integrator
baseline of the block-step workload.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synth import plummer  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--n", "4096", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, check=True, timeout=600).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_traffic_is_reported_only_for_the_profiled_sources(monkeypatch):
    full = bench.force_traffic_per_launch(1 << 20)
    if full is None:
        pytest.skip("the force kernel changed since its ncu summary was taken")
    # O(N) traffic scales linearly with the launch size
    assert bench.force_traffic_per_launch(1 << 19) == pytest.approx(full / 2)
    monkeypatch.setattr(bench, "force_sources_sha256", lambda sources=None: "0" * 64)
    assert bench.force_traffic_per_launch(1 << 20) is None


def test_traffic_lookup_prefers_an_exact_capture(tmp_path):
    # A summary may carry captures at several N: the launch size's own capture
    # is taken as it is (the whole/sliced plan's partials do not scale with
    # N); any other N scales the largest capture linearly.
    h = bench.force_sources_sha256()
    prof = tmp_path / "k.md"
    prof.write_text("force sources sha256 (k_force.cu, ...): %s\n"
                    "dram bytes per launch at N=262144: 7.8e7\n"
                    "dram bytes per launch at N=1048576: 2.4e8\n" % h)
    assert bench.force_traffic_per_launch(1 << 20, str(prof)) == 2.4e8
    assert bench.force_traffic_per_launch(1 << 18, str(prof)) == 7.8e7
    assert bench.force_traffic_per_launch(1 << 21, str(prof)) == pytest.approx(4.8e8)
    assert bench.force_traffic_per_launch(1 << 19, str(prof)) == pytest.approx(1.2e8)
    prof.write_text("force sources sha256: %s\n" % ("f" * 64) +
                    "dram bytes per launch at N=1048576: 2.4e8\n")
    assert bench.force_traffic_per_launch(1 << 20, str(prof)) is None
    prof.write_text("force sources sha256: %s\n" % h)       # no capture at all
    assert bench.force_traffic_per_launch(1 << 20, str(prof)) is None


def test_measured_hbm_peak(tmp_path, monkeypatch):
    peak = bench.hbm_peak_gbs()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert peak == pytest.approx(float(json.load(f)["hbm_gbs"]))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))      # no measured file there
    assert bench.hbm_peak_gbs() == bench.HBM_GBS_FALLBACK


def test_oracle_blockstep_baseline_whole_run_and_projection():
    m, x, v = plummer(128, 2)
    gpu = {"interactions": 10 ** 9, "steps": 100, "interactions_per_s": 1e11}
    whole = bench.oracle_blockstep_rate(m, x, v, 1.0 / 256, 3, 0.125, gpu, 30.0)
    assert whole["whole_run"] and whole["steps"] > 0 and whole["value"] > 0
    assert whole["kind"] == "oracle" and "projected_whole_run_s" not in whole
    # a budget far below the run: at least one step, then the projection
    part = bench.oracle_blockstep_rate(m, x, v, 1.0 / 256, 3, 0.125, gpu, 1e-4)
    assert not part["whole_run"] and 1 <= part["steps"] < whole["steps"]
    assert part["projected_whole_run_s"] == pytest.approx(gpu["interactions"] / part["value"])
    # a system whose integrator start-up alone exceeds the budget: the
    # oracle's force on a sample instead
    m2, x2, v2 = plummer(2048, 3)
    samp = bench.oracle_blockstep_rate(m2, x2, v2, 1.0 / 256, 3, 0.125, gpu, 1e-3)
    assert not samp["whole_run"] and "steps" not in samp and samp["value"] > 0


def test_bench_error_metric_matches_the_parity_tests():
    # The benchmark's accuracy figures use the per-particle metric of the
    # parity tests: the same pair-magnitude sums, and err = |d| / max(|ref|, S/10)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from nbtest import force_errors, pair_magnitudes
    import numpy as np
    m, x, v = plummer(300, 41)
    idx = np.array([0, 7, 150, 299], dtype=np.int32)
    eps = 1.0 / 256
    sa, sk = bench.pair_magnitude_sums(m, x, v, eps, idx, chunk=3)
    ta, tk = pair_magnitudes(m, x, v, eps, idx)
    assert np.allclose(sa, ta, rtol=1e-12) and np.allclose(sk, tk, rtol=1e-12)
    r = np.random.default_rng(3)
    ref = (r.normal(size=(4, 3)), r.normal(size=(4, 3)), -np.abs(r.normal(size=4)) - 1.0)
    got = tuple(q * (1 + 1e-7 * r.normal(size=q.shape)) for q in ref)
    e = bench.force_error_stats(got, ref, sa, sk)
    ea, ek, ep = force_errors(got, ref, (sa, sk))
    assert np.isclose(e[0], ea.max()) and np.isclose(e[1], ek.max()) and np.isclose(e[2], ep.max())
