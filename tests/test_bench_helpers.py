"""Host logic of the benchmark on CPU: the roofline arithmetic (the method's
per-unit figures times the device counters, over the derived FP32 peak),
the ncu traffic marker that is only trusted while the kernel sources it was
captured from are unchanged, the clock record that decides whether a run is
kept, and the oracle sample's windows."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

COUNTERS = dict(pairs_sum=7_680_000, eval_fwd=500_000_000, composited_fwd=400_000_000,
                eval_rewalk=794_000_000, eval_back=791_000_000, composited_rewalk=631_000_000,
                hits_back=631_000_000)


def test_fp32_peak_is_the_unit_count_product():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12, rel=1e-6)


def test_compositing_flops_take_the_per_pair_figures():
    c = COUNTERS
    assert bench.phase_algorithmic("render", c, 0, 0, 1) == ("flop", 15.0 * c["eval_fwd"])
    assert bench.phase_algorithmic("render_bwd", c, 0, 0, 1) == ("flop", 45.0 * c["eval_back"])
    kind, f = bench.phase_algorithmic("train", c, 0, 0, 1)
    assert kind == "flop" and f == 15.0 * c["eval_rewalk"] + 45.0 * c["eval_back"]
    # the stricter count grows with every counter it names and with the pixels (loss)
    _, base = bench.phase_algorithmic("train", c, 0, 3 * 1000, 1, fine=True)
    for key in ("eval_rewalk", "eval_back", "composited_rewalk", "hits_back"):
        _, more = bench.phase_algorithmic("train", dict(c, **{key: c[key] + 1000}), 0, 3 * 1000, 1, fine=True)
        assert more > base, key
    _, more = bench.phase_algorithmic("train", c, 0, 3 * 2000, 1, fine=True)
    assert more > base


def test_binning_phases_are_byte_bound_per_unit():
    c = dict(COUNTERS, pair_sort_passes=1)
    assert bench.phase_algorithmic("tile_sort", c, 1_000_000, 0, 1) == ("byte", 20.0 * c["pairs_sum"])
    assert bench.phase_algorithmic("depth_sort", c, 1_000_000, 0, 1) == ("byte", 68.0 * 1_000_000)
    assert bench.phase_algorithmic("emit", c, 1_000_000, 0, 1) == ("byte", 8.0 * c["pairs_sum"] + 52.0e6)


def test_train_roofline_divides_the_flops_by_the_event_time():
    c = COUNTERS
    prof = {"train": (2 * 1.8, 2, 2)}  # two launches, 3.6 ms in total
    r = bench.train_roofline(c, prof, 0, 2)
    flops = 15.0 * c["eval_rewalk"] + 45.0 * c["eval_back"]
    assert r["achieved"] == pytest.approx(flops / 3.6e-3 / 1e12, abs=0.01)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP32_PEAK_TFLOPS, abs=1e-3)
    assert r["ms_per_step"] == pytest.approx(1.8)
    assert bench.train_roofline(c, {}, 0, 2) is None   # no time measured: no roofline


def _tree(tmp_path, raster=b"kernel v1", internal=b"header v1", traffic=149123840):
    csrc = tmp_path / "paper_2507_19718_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "raster.cu").write_bytes(raster)
    (csrc / "gsc_internal.cuh").write_bytes(internal)
    prof = tmp_path / "profiles"
    prof.mkdir()
    marker = (f"<!-- ncu kernel=train traffic_bytes_per_launch={traffic} "
              f"raster_sha256={hashlib.sha256(raster).hexdigest()} "
              f"internal_sha256_16={hashlib.sha256(internal).hexdigest()[:16]} -->")
    (prof / "train_1080p_1M.md").write_text("# summary\n\n" + marker + "\n")
    return csrc


def test_traffic_marker_holds_only_for_the_captured_sources(tmp_path):
    csrc = _tree(tmp_path)
    assert bench.ncu_traffic("train", str(tmp_path)) == 149123840
    assert bench.ncu_traffic("render", str(tmp_path)) is None          # no summary for that kernel
    (csrc / "raster.cu").write_bytes(b"kernel v2")                     # the kernel changed since
    assert bench.ncu_traffic("train", str(tmp_path)) is None
    (csrc / "raster.cu").write_bytes(b"kernel v1")
    (csrc / "gsc_internal.cuh").write_bytes(b"header v2")              # so did a header it includes
    assert bench.ncu_traffic("train", str(tmp_path)) is None


def _clock_summary(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.path = str(p)
    return s.summary()


def test_clock_record_reports_median_max_and_throttle_reasons(tmp_path):
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1200.0, 0x40, Not Active, Active, Not Active, Not Active"
    s = _clock_summary(tmp_path, [ok, ok, cap])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s = _clock_summary(tmp_path, [ok, hot, hot, "garbage line"])
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_thermal_slowdown"] and s["samples"] == 3
    s = _clock_summary(tmp_path, [])
    assert s["reasons"] == ["unsampled"] and s["samples"] == 0


def test_oracle_sample_windows_cover_the_frame_in_three_steps():
    cells = set()
    for step in range(3):
        for x, y, w, h in bench.sample_windows(step):
            assert 0 <= x and x + w <= bench.WIDTH and 0 <= y and y + h <= bench.HEIGHT
            cells.add((3 * x // bench.WIDTH, 3 * y // bench.HEIGHT))
    assert cells == {(i, j) for i in range(3) for j in range(3)}
    assert bench.sample_windows(4) == bench.sample_windows(4)   # seeded
