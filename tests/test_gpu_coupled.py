"""Cache-coupled tracing (Algorithm 1, Eq. 2) trades bias for variance and
runtime with C (Sec. 4.3 "bias-variance trade-off", Sec. 4.4): terminating
into the cache more often (small C) shortens the paths, so the tracer runs
faster, and leans on the cache, so the image's bias grows and its variance
falls; a large C approaches the uncached tracer.  That is the shape under
Algorithm 1 read per call, as it is printed (each call divides the albedo
product by its own Tr + eps).  Read cumulatively, as Russian roulette
(survivors keep every earlier 1/(Tr + eps)), the bias and runtime move the
same way but a small C raises the variance instead (256 frames per C at the
benchmark's 480x270 view: 43 at C = 0.1 against 0.003 at C = 4): the
survivors of small-Tr decisions carry large weights."""
import pytest

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu


def _sweep(mode):
    from paper_2507_19718_gb300 import coupled
    sc = synth.scene_frame(96, seed=synth.BASE_SEED + 1)
    rows = coupled.sweep(sc, synth.level_sizes(60_000, 3), width=320, height=192, Cs=(0.1, 4.0),
                         train_frames=24, eval_frames=48, ref_spp=256, max_bounces=8, tr_out=mode)
    return {row["C"]: row for row in rows}


def test_per_call_reading_trades_bias_for_variance_and_runtime(gpu):
    r = _sweep(gpu.TR_OUT_PER_CALL)
    assert r[0.1]["bias2"] > r[4.0]["bias2"] > r["off"]["bias2"]
    assert r[0.1]["variance"] < r[4.0]["variance"]
    assert r[0.1]["variance"] < r["off"]["variance"]
    assert r[0.1]["trace_ms"] < r[4.0]["trace_ms"] < r["off"]["trace_ms"]


def test_cumulative_reading_moves_bias_and_runtime(gpu):
    # its variance is heavy-tailed (rare survivors of small-Tr decisions carry
    # weights up to 1/eps), so a few dozen frames do not order it reliably
    r = _sweep(gpu.TR_OUT_CUMULATIVE)
    assert r[0.1]["bias2"] > r[4.0]["bias2"]
    assert r[0.1]["trace_ms"] < r["off"]["trace_ms"]
