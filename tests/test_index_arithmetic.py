"""Index arithmetic of the kernels, checked on the CPU.

The pair emission finds the row of pair k in a Gaussian's bin rectangle,
wj bins wide, as trunc((float(k) + 0.5) * rcp_rn(wj)) in FP32 instead of an
integer division.  The ABI bounds make wj <= 2048 and k < 2^22 (images up
to 65535 px wide and high, bins of at least 32 px).  Both FP32 steps round
to nearest and are monotone in k, so the row is right for every k once it
is right for the first and the last pair of every row; numpy's float32
arithmetic rounds as the device does (IEEE round to nearest even, the
reciprocal correctly rounded like __frcp_rn)."""
import numpy as np

MAX_BINS = 65535 // 32 + 1      # bins along one image axis at the smallest bin
MAX_K = MAX_BINS * MAX_BINS     # pairs in the largest bin rectangle


def _row(k, rcp):
    return ((k.astype(np.float32) + np.float32(0.5)) * rcp).astype(np.int64)


def test_emission_row_from_the_fp32_reciprocal_is_the_integer_quotient():
    assert MAX_BINS == 2048 and MAX_K == 1 << 22
    for wj in range(1, MAX_BINS + 1):
        rcp = np.float32(1.0) / np.float32(wj)
        m = np.arange(1, (MAX_K - 1) // wj + 1, dtype=np.int64)   # rows that start below MAX_K
        first = m * wj                                            # first pair of row m
        assert (_row(first, rcp) == m).all(), wj
        assert (_row(first - 1, rcp) == m - 1).all(), wj            # last pair of row m - 1
        last = np.array([MAX_K - 1], dtype=np.int64)
        assert _row(last, rcp)[0] == (MAX_K - 1) // wj, wj
    assert _row(np.array([0]), np.float32(1.0))[0] == 0


def test_a_plain_fp32_quotient_would_not_do():
    # without the half-pair offset the product can round up onto the next
    # integer just below a row start (the offset keeps it 1/(2 wj) away)
    bad = 0
    for wj in (3, 5, 7, 11, 13, 49, 97, 769, 2047):
        rcp = np.float32(1.0) / np.float32(wj)
        m = np.arange(1, (MAX_K - 1) // wj + 1, dtype=np.int64)
        k = m * wj - 1
        bad += int((((k.astype(np.float32)) * rcp).astype(np.int64) != m - 1).sum())
        bad += int((((m * wj).astype(np.float32) * rcp).astype(np.int64) != m).sum())
    assert bad > 0
