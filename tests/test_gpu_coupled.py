"""Cache-coupled tracing (Algorithm 1, Eq. 2) trades bias for runtime with C
(Sec. 4.3, 4.4): terminating into the cache more often (small C) shortens
the paths, so the tracer runs faster, and leans on the cache, so the image's
bias grows; a large C approaches the uncached tracer.  (Under the cumulative
Russian-roulette reading of Tr_out, survivors of small-C decisions carry
weights 1/Tr, so the per-frame variance is reported but not ordered.)"""
import pytest

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu


def test_c_moves_along_the_bias_and_runtime_scale(gpu):
    from paper_2507_19718_gb300 import coupled
    sc = synth.scene_frame(96, seed=synth.BASE_SEED + 1)
    rows = coupled.sweep(sc, synth.level_sizes(60_000, 3), width=320, height=192, Cs=(0.1, 4.0),
                         train_frames=24, eval_frames=16, ref_spp=256, max_bounces=8)
    r = {row["C"]: row for row in rows}
    assert r[0.1]["bias2"] > r[4.0]["bias2"]
    assert r[0.1]["bias2"] > r["off"]["bias2"]
    assert r[0.1]["trace_ms"] < r["off"]["trace_ms"]
    for row in rows:
        assert row["trace_ms"] > 0 and row["variance"] > 0
