"""The PNG build divides node IDs by the partition size q with a multiply-high
instead of a division: key = floor(v * m / 2^64) with m = ceil(2^64 / q)
(q = 1: key = v). This checks that identity over every q the library accepts
(1..32768) at the numerators where it is tightest: just below and at every
multiple of q near the top of the 32-bit range, and random v."""
import numpy as np

MAX_Q = 32768


def mulhi_div(v: int, q: int) -> int:
    if q == 1:
        return v
    m = (2**64 - 1) // q + 1  # ceil(2^64 / q), as computed on the host
    return (v * m) >> 64


def test_identity_for_every_partition_size():
    rng = np.random.default_rng(1709)
    top = 2**32 - 1
    for q in range(1, MAX_Q + 1):
        k_hi = top // q
        cands = {0, 1, q - 1, q, top, top - 1}
        for kk in (k_hi, k_hi - 1, 1, 2):
            for dv in (-1, 0, 1, q - 1):
                v = kk * q + dv
                if 0 <= v <= top:
                    cands.add(v)
        for v in cands:
            assert mulhi_div(v, q) == v // q, (v, q)
    for q in rng.integers(1, MAX_Q + 1, size=2000):
        for v in rng.integers(0, 2**32, size=64, dtype=np.uint64):
            assert mulhi_div(int(v), int(q)) == int(v) // int(q)


def test_error_bound_argument():
    # v*m/2^64 - v/q = v*(m - 2^64/q)/2^64 < 2^32/2^64, while the fraction of
    # v/q is at most 1 - 1/q: the floor is exact while 2^-32 < 1/q.
    for q in (2, 3, 7, 1000, 32767, 32768):
        m = (2**64 - 1) // q + 1
        assert 0 <= m * q - 2**64 < q
        assert 2**32 * (m * q - 2**64) < 2**64 // q * q
