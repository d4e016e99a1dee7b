"""The tiled nodal kernels split a flat thread index t into (t mod w, t div w) with one
float multiplication by 1/w instead of an integer division by a run-time w.  Exact for
every t < 2^16 and every w the kernels use (checked here with the same binary32
arithmetic: round-to-nearest product, truncating conversion)."""
import numpy as np


def test_float_quotient_truncation_is_exact():
    t = np.arange(0, 1 << 16, dtype=np.int64)
    tf = t.astype(np.float32) + np.float32(0.5)
    for w in range(1, 257):
        inv = np.float32(1.0) / np.float32(w)
        v = (tf * inv).astype(np.int64)
        assert np.array_equal(v, t // w), w
        assert np.array_equal(t - v * w, t % w), w
