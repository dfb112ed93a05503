"""Error model of the FP16 split used by the tensor-core tree level (CPU, no GPU).

The level product W_m P (P: 64-amplitude parent rows in real form, 128 floats) runs on
FP16 tensor cores as W_hi P_hi + W_hi P_lo + W_lo P_hi.  Each row is scaled by a power
of two s so that its largest |component| lies in [2^14, 2^15); hi is x s rounded to a
multiple of 16 in FP32 (adding and removing 1.5 2^27), lo = fp16(x s - hi).  These
tests restate that arithmetic in numpy and check the claims the kernel relies on:

* hi is exactly representable in FP16 and x s - hi is exact in FP32 (|x s - hi| <= 8);
* hi + lo reproduces x s within 2^-9, i.e. the split is within 2^-23 of the row's
  largest component whatever the spread of magnitudes across rows;
* the three-product sum is within a few 2^-22 of the exact product, relative to
  |W| |P| row by row.
"""
import numpy as np
import pytest

ROUND = np.float32(1.5 * 2.0 ** 27)


def row_scale(rows):
    """Power of two per row: largest |component| in [2^14, 2^15) (1 for zero rows)."""
    mx = np.max(np.abs(rows), axis=1)
    e = np.zeros(len(rows), dtype=np.int64)
    nz = mx > 0
    e[nz] = 14 - np.floor(np.log2(mx[nz])).astype(np.int64)
    return np.ldexp(np.ones(len(rows)), e).astype(np.float32)


def split(rows32):
    s = row_scale(rows32)
    xs = rows32 * s[:, None]                                   # exact (power of two)
    hi = (xs + ROUND).astype(np.float32) - ROUND               # FP32 rounding to 16
    hi = hi.astype(np.float32)
    lo = (xs - hi).astype(np.float32)
    return s, xs, hi, lo


def wide_rows(rng, nrows=256, k=128):
    """Rows whose magnitudes span 2^-60 .. 2^0 across rows, Gaussian within a row."""
    scale = np.ldexp(1.0, -rng.integers(0, 60, size=nrows))
    return (rng.standard_normal((nrows, k)) * scale[:, None]).astype(np.float32)


def test_hi_exact_in_fp16_and_rest_exact():
    rng = np.random.default_rng(1)
    rows = wide_rows(rng)
    s, xs, hi, lo = split(rows)
    assert np.all(np.abs(hi) <= 2.0 ** 15)
    assert np.array_equal(hi.astype(np.float16).astype(np.float32), hi)
    assert np.all(np.mod(hi, 16.0) == 0)
    # xs - hi computed in FP32 equals the exact difference (checked in FP64)
    assert np.array_equal(lo.astype(np.float64), xs.astype(np.float64) - hi.astype(np.float64))
    assert np.all(np.abs(lo) <= 8.0)


def test_split_within_2_pow_minus_23_of_row_max():
    rng = np.random.default_rng(2)
    rows = wide_rows(rng)
    s, xs, hi, lo = split(rows)
    lo16 = lo.astype(np.float16).astype(np.float64)
    recon = (hi.astype(np.float64) + lo16) / s[:, None].astype(np.float64)
    rowmax = np.max(np.abs(rows.astype(np.float64)), axis=1)
    err = np.max(np.abs(recon - rows.astype(np.float64)), axis=1)
    assert np.all(err <= 2.0 ** -23 * rowmax), np.max(err / rowmax)


def test_three_product_sum_close_to_exact_product():
    rng = np.random.default_rng(3)
    P = wide_rows(rng, nrows=128)                              # parent rows (N x K)
    W = (rng.standard_normal((128, 128)) / 11.3).astype(np.float32)
    sp, _, ph, pl = split(P)
    sw, _, wh, wl = split(W.reshape(1, -1))
    wh = wh.reshape(128, 128).astype(np.float16).astype(np.float64)
    wl = wl.reshape(128, 128).astype(np.float16).astype(np.float64)
    ph = ph.astype(np.float16).astype(np.float64)
    pl = pl.astype(np.float16).astype(np.float64)
    approx = (ph @ wh.T + pl @ wh.T + ph @ wl.T) / (sp[:, None].astype(np.float64) * float(sw[0]))
    exact = P.astype(np.float64) @ W.astype(np.float64).T
    bound = np.abs(P.astype(np.float64)) @ np.abs(W.astype(np.float64)).T
    assert np.all(np.abs(approx - exact) <= 4 * 2.0 ** -22 * bound)


@pytest.mark.parametrize("drop", ["lo_p", "lo_w"])
def test_dropping_a_cross_term_breaks_the_bound(drop):
    """The check above is sharp enough to see a missing product."""
    rng = np.random.default_rng(4)
    P = wide_rows(rng, nrows=64)
    W = (rng.standard_normal((128, 128)) / 11.3).astype(np.float32)
    sp, _, ph, pl = split(P)
    sw, _, wh, wl = split(W.reshape(1, -1))
    wh = wh.reshape(128, 128).astype(np.float16).astype(np.float64)
    wl = wl.reshape(128, 128).astype(np.float16).astype(np.float64)
    ph = ph.astype(np.float16).astype(np.float64)
    pl = pl.astype(np.float16).astype(np.float64)
    terms = ph @ wh.T + (0 if drop == "lo_p" else pl @ wh.T) + (0 if drop == "lo_w" else ph @ wl.T)
    approx = terms / (sp[:, None].astype(np.float64) * float(sw[0]))
    exact = P.astype(np.float64) @ W.astype(np.float64).T
    bound = np.abs(P.astype(np.float64)) @ np.abs(W.astype(np.float64)).T
    assert np.any(np.abs(approx - exact) > 4 * 2.0 ** -22 * bound)
