"""Exactness of the integer detail path of the FP16-storage form.

The details of a sibling group decide the mesh, so every form computes them
with the rounding of the FP64 canonical prediction (Def. Details, s = 1
prediction of Table 1).  For FP16 storage the library evaluates them with
64-bit integers in units of 2^-30 instead: a finite half is an integer
multiple of 2^-24 below 2^16, so the canonical FP64 operations (sums of at
most four stored values, products with c1 = -1/8 and c1^2 = 1/64, the
difference with the child) never round.  This test checks that claim on the
operations themselves: for random finite halves (normal, subnormal, zero,
the largest exponents) the canonical FP64 sequence, evaluated with IEEE
round-to-nearest doubles, gives bit for bit the value the integer sequence
gives, for both signs of the cross term and in 1D and 2D.
"""
import numpy as np

C1 = -0.125


def _halves(rng, n):
    """Random finite FP16 values, weighted towards the extremes."""
    bits = rng.integers(0, 1 << 16, size=n, dtype=np.uint32)
    e = (bits >> 10) & 31
    bits = np.where(e == 31, bits & ~np.uint32(1 << 10), bits)  # no Inf / NaN
    h = bits.astype(np.uint16).view(np.float16)
    k = rng.integers(0, 8, size=n)
    h = np.where(k == 0, np.float16(0.0), h)  # zeros
    h = np.where(k == 1, (rng.integers(0, 1024, size=n).astype(np.uint16)).view(np.float16), h)  # subnormals
    return h


def _fp64_canonical(v, c, cross, d):
    """Largest |child - prediction| with the FP64 operations in the library's
    canonical order (each numpy float64 operation rounds to nearest)."""
    v = v.astype(np.float64)
    c = c.astype(np.float64)
    if d == 1:
        q = C1 * (v[2] - v[0])
        pr = [v[1] + q, v[1] - q]
    else:
        qx = C1 * (v[5] - v[3])
        qy = C1 * (v[7] - v[1])
        q2 = (C1 * C1) * (((v[8] - v[6]) - v[2]) + v[0])
        a, b = v[4] + qx, v[4] - qx
        t0, t1, t2, t3 = a + qy, b + qy, a - qy, b - qy
        if cross > 0:
            pr = [t0 + q2, t1 - q2, t2 - q2, t3 + q2]
        else:
            pr = [t0 - q2, t1 + q2, t2 + q2, t3 - q2]
    return np.max(np.abs(np.stack([c[i] - pr[i] for i in range(len(pr))])), axis=0)


def _units30(h):
    """A finite half as an integer in units of 2^-30, from its bits."""
    b = h.view(np.uint16).astype(np.int64)
    e = (b >> 10) & 31
    m = b & 1023
    a = np.where(e > 0, (1024 | m) << np.maximum(e - 1, 0), m)
    return np.where(b & 0x8000, -64 * a, 64 * a)


def _integer(v, c, cross, d):
    w = _units30(v)
    cc = _units30(c)
    if d == 1:
        q = -((w[2] - w[0]) >> 3)
        pr = [w[1] + q, w[1] - q]
    else:
        qx = -((w[5] - w[3]) >> 3)
        qy = -((w[7] - w[1]) >> 3)
        q2 = (((w[8] - w[6]) - w[2]) + w[0]) >> 6
        a, b = w[4] + qx, w[4] - qx
        s = q2 if cross > 0 else -q2
        pr = [a + qy + s, b + qy - s, a - qy - s, b - qy + s]
    m = np.max(np.abs(np.stack([cc[i] - pr[i] for i in range(len(pr))])), axis=0)
    assert m.max() < 2 ** 50
    return m.astype(np.float64) * 2.0 ** -30  # exact: below 2^53, power-of-two scale


def test_units_are_the_half_values():
    rng = np.random.Generator(np.random.PCG64(0))
    h = _halves(rng, 200000)
    assert np.array_equal(_units30(h).astype(np.float64) * 2.0 ** -30, h.astype(np.float64))


def test_integer_details_equal_fp64_canonical():
    rng = np.random.Generator(np.random.PCG64(1))
    n = 100000
    for d, ns in ((1, 3), (2, 9)):
        for cross in (1, -1):
            v = np.stack([_halves(rng, n) for _ in range(ns)])
            c = np.stack([_halves(rng, n) for _ in range(1 << d)])
            want = _fp64_canonical(v, c, cross, d)
            got = _integer(v, c, cross, d)
            assert np.array_equal(want.view(np.int64), got.view(np.int64)), (d, cross)


def test_integer_details_on_smooth_fields():
    """Near-cancelling details (smooth data), where rounding would show."""
    rng = np.random.Generator(np.random.PCG64(2))
    n = 100000
    base = rng.uniform(-3, 3, size=n)
    slope = rng.uniform(-1, 1, size=(2, n)) * 1e-2
    for cross in (1, -1):
        xs = np.array([-1, 0, 1])
        v = np.stack([(base + slope[0] * xs[k % 3] + slope[1] * xs[k // 3]).astype(np.float16) for k in range(9)])
        c = np.stack([(base + 0.25 * (slope[0] * (1 - 2 * (k & 1)) + slope[1] * (1 - 2 * (k >> 1)))).astype(np.float16)
                      for k in range(4)])
        want = _fp64_canonical(v, c, cross, 2)
        got = _integer(v, c, cross, 2)
        assert np.array_equal(want.view(np.int64), got.view(np.int64))
