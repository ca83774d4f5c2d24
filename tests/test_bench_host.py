"""Host-side parts of bench.py (no GPU): the CPU-baseline extrapolation, the
reference arm's JSON line, the flop counts behind the rooflines, the DRAM
traffic record and its source hashes, the time-to-solution list, the clock
sampler's parsing and the peak-file fallback."""
import argparse
import json
import time

import pytest

import bench


class _FakeProblem:
    """Stands in for the oracle's operator: one application costs
    a + b x (rings in the subset) seconds."""

    def __init__(self, nsub, a, b):
        self.cost = a + b * nsub

    def matvec(self, x):
        time.sleep(self.cost)


def test_oracle_fit_separates_ring_independent_work(monkeypatch):
    a, b, nring = 0.05, 4e-4, 4095

    def fake_problem(stride):
        nsub = len(range(0, nring, stride))
        return _FakeProblem(nsub, a, b), None, nring, nsub

    monkeypatch.setattr(bench, "_oracle_problem", fake_problem)
    r = bench.oracle_sample(strides=(32, 8))
    expect = 1.0 / ((a + b * nring) * bench.NB)
    # sleep() overshoots by up to a few ms per sample
    assert r["value"] == pytest.approx(expect, rel=0.15)
    assert r["kind"] == "oracle" and r["unit"] == bench.UNIT and r["cores"] >= 1
    assert "fitted a + b x rings" in r["sample"]
    # scaling the whole denser sample by the ring ratio would count a about 8 times
    naive = 1.0 / ((a + b * 512) * (nring / 512) * bench.NB)
    assert r["value"] > 1.15 * naive


def test_oracle_fit_falls_back_on_noisy_samples(monkeypatch):
    # the sparser subset measured slower than the denser one: no negative slope
    costs = {128: 0.03, 512: 0.02}

    class P:
        def __init__(self, n):
            self.n = n

        def matvec(self, x):
            time.sleep(costs[self.n])

    def fake_problem(stride):
        nsub = 128 if stride == 32 else 512
        return P(nsub), None, 4095, nsub

    monkeypatch.setattr(bench, "_oracle_problem", fake_problem)
    r = bench.oracle_sample(strides=(32, 8))
    assert r["value"] > 0.0
    assert r["value"] == pytest.approx(1.0 / (0.02 * 4095 / 512 * bench.NB), rel=0.3)


def _fake_sample(**kw):
    time.sleep(0.01)
    return {"value": 2.5e-3, "unit": bench.UNIT, "cores": 16, "kind": "oracle", "sample": "fake",
            "per_realization_s": 1.0 / (2.5e-3 * bench.NB)}


def test_reference_line_contract(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample", _fake_sample)
    monkeypatch.setattr(bench, "oracle_full_grid", lambda: 55.0)
    monkeypatch.setattr(bench, "oracle_extras", lambda: {"cores": 16})
    monkeypatch.delenv("RANK", raising=False)
    args = argparse.Namespace(steps=2, warmup=3, gpus=1)
    assert bench.run_reference(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] == pytest.approx(2.5e-3)
    # ms_per_step is the wall time of one bounded sample step, not 1 / value
    assert 5.0 <= d["ms_per_step"] < 1000.0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["steps"] == 2 and d["warmup"] == 3
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == 16
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    fc = d["fit_check"]
    assert fc["full_grid_operator_s"] == 55.0
    assert fc["fit_predicted_s"] == pytest.approx(50.0)
    assert fc["rel_err"] == pytest.approx(-5.0 / 55.0)


def test_reference_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample", _fake_sample)
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=2, warmup=3, gpus=2)) == 0
    assert capsys.readouterr().out.strip() == ""


def test_flop_counts():
    # per (l, m, ring pair): 4 flops per temperature map, 16 per (Q, U) pair
    assert bench.contraction_flops(10, 3, 2, 1) == 10 * 3 * (4 * 2 + 16 * 1)
    # plus the recurrence: 3 shared (spin 0) and 8 shared (spin 2)
    assert bench.legendre_flops(10, 3, 2, 1) == 10 * 3 * ((3 + 4 * 2) + (8 + 16 * 1))
    assert bench.legendre_flops(10, 3, 2, 0) == 10 * 3 * (3 + 4 * 2)


def test_ring_fft_flops_counts_one_dft_per_ring_pair():
    import math
    # N_side 1: no polar pairs, two equatorial pairs of n = 4 (one is the equator alone)
    assert bench.ring_fft_flops(1) == 2 * 5 * 4 * 2
    # N_side 2: polar pair n = 4, three equatorial pairs of n = 8
    assert bench.ring_fft_flops(2) == 5 * 4 * 2 + 3 * 5 * 8 * 3
    # the pairs cover every ring: 2 sum(n) - n_equator = 12 N^2 pixels
    n = 64
    pix = 2 * sum(4 * i for i in range(1, n)) + (n + 1) * 2 * 4 * n - 4 * n
    assert pix == 12 * n * n
    assert bench.ring_fft_flops(n) > 5 * 4 * n * math.log2(4 * n) * (n + 1)


def test_traffic_record_needs_unchanged_sources(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2306_15511_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "ringfft.cu").write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.sources_hash(["ringfft.cu"])
    (tmp_path / "profiles" / "traffic.json").write_text(
        json.dumps({"ring_fft_fp32": {"dram_bytes_per_unit": 20.0, "sources_sha": sha}}))
    assert bench.traffic_record("ring_fft_fp32", 1000) == 20000.0
    assert bench.traffic_record("leg_synth_fp32", 1000) is None
    (csrc / "ringfft.cu").write_text("kernel v2")
    assert bench.traffic_record("ring_fft_fp32", 1000) is None


def test_clock_sampler_parses_nvidia_smi_rows(tmp_path):
    """The clocks record of the JSON line: median SM clock under load, the
    maximum, and every throttle reason seen Active in any sample."""
    rows = [
        "0, 2070, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1310.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1290.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    ck = bench.Clocks(0)
    ck.proc, ck.path = _Done(), str(path)
    r = ck.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3
    assert not path.exists()


def test_clock_sampler_without_nvidia_smi():
    ck = bench.Clocks(0)
    r = ck.stop()       # never started
    assert r["sm_mhz"] is None and r["reasons"]


def test_measured_peaks_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6682.5, "bf16_tflops": 1900.3}')
    peaks, src = bench.measured_peaks()
    assert src == "measured" and peaks["hbm_gbs"] == 6682.5


def test_committed_traffic_record_matches_the_current_sources():
    """profiles/traffic.json holds the tensor-core classes' DRAM bytes per
    Fourier coefficient with the sources' hash at the capture; the bench
    reports them only while the sources are unchanged, so a record that no
    longer matches would silently drop roofline.traffic."""
    path = bench.os.path.join(bench.ROOT, "profiles", "traffic.json")
    rec = json.load(open(path))
    for cls in ("leg_synth_fp32", "leg_analysis_fp32"):
        assert rec[cls]["sources_sha"] == bench.sources_hash(bench.CLASS_SOURCES[cls]), cls
        assert bench.traffic_record(cls, 1.0) == rec[cls]["dram_bytes_per_unit"]


def test_time_to_solution_lists_every_full_solve_fastest_first():
    ex = {"mixed_full_solve": {"precond": "diag", "time_to_1e-6_s": 35.0, "iterations": 1736, "converged": True,
                               "rel_residual": 9e-7},
          "mixed_full_solve_azim": {"precond": "azim (l_b 1024)", "time_to_1e-6_s": 12.7, "iterations": 200,
                                    "converged": True, "rel_residual": 2e-7},
          "mixed_full_solve_azim_lb512": {"precond": "azim (l_b 512)", "time_to_1e-6_s": 11.3, "iterations": 440,
                                          "converged": True, "rel_residual": 9e-7},
          "sht_pairs_per_s": {}}
    out = bench._time_to_solution(ex)
    assert [o["precond"] for o in out] == ["azim (l_b 512)", "azim (l_b 1024)", "diag"]
    assert out[0]["fp32_iterations"] == 440
    assert bench._time_to_solution({}) is None
