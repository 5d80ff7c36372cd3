"""Host-side merge of exact node records (pdd_records_merge): every 128-bit
sum adds with its carry, counts add; checked against Python integers."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def pdd():
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    return pdd


def _to_ints(rec):
    out = []
    for w in range(0, 14, 2):
        out.append((int(rec[w + 1]) << 64) | int(rec[w]))
    return out + [int(rec[14]), int(rec[15])]


def test_merge_matches_big_integers(pdd):
    rng = np.random.default_rng(1)
    n = 50
    a = rng.integers(0, 2**64, size=(n, 16), dtype=np.uint64)
    b = rng.integers(0, 2**64, size=(n, 16), dtype=np.uint64)
    a[:, 14:] %= 2**40  # counts: no wrap in 64 bits
    b[:, 14:] %= 2**40
    a[0, 0] = b[0, 0] = 2**64 - 1  # forces a carry
    want = []
    for i in range(n):
        x, y = _to_ints(a[i]), _to_ints(b[i])
        z = [(p + q) % 2**128 for p, q in zip(x[:7], y[:7])] + [x[7] + y[7], x[8] + y[8]]
        want.append(z)
    dst = a.copy()
    pdd.pdd_records_merge(dst.ctypes.data, b.ctypes.data, n)
    for i in range(n):
        assert _to_ints(dst[i]) == want[i]
    pdd.pdd_records_merge(None, None, 0)
    with pytest.raises(pdd.PddError):
        pdd.pdd_records_merge(None, b.ctypes.data, 3)
