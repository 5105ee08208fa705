"""The band walk's dedupe, checked against the arithmetic it rests on (CPU).

The oracle skips a sample whose voxel equals ANY earlier voxel of the same
point (Section 2.2, each voxel once per point). The GPU walks compare a
sample with the previous sample's voxel only. The two are the same test
because every voxel coordinate is a monotone function of the sample index k:
t_k = (k - M) v, the correctly rounded fused multiply-add t_k d + p, the
product by 1/v and floor are each monotone, and so is the range test on the
floored coordinate, so in-range samples are consecutive and a repeat of an
earlier voxel repeats the previous one too.

Here the exact single-precision sequence (fused multiply-add emulated exactly,
see brute_dense.fma32) is evaluated on random rays, rays along and near the
axes, rays through voxel boundaries and rays crossing the key's coordinate
limit, and both dedupe rules are compared sample by sample.
"""
import numpy as np

from brute_dense import F32, fma32

LIMIT = F32(8 * (1 << 20))      # voxel coordinate range of the 21-bit block key


def walk(P, D, v, M):
    """(voxels (K, 3) int64, in-range mask (K,)) of one point's band."""
    v = F32(v)
    inv_v = F32(1.0) / v
    K = 2 * M + 1
    g = np.zeros((K, 3), dtype=np.int64)
    ok = np.ones(K, dtype=bool)
    for k in range(K):
        tk = F32(k - M) * v
        for i in range(3):
            q = np.floor(fma32(tk, D[i], P[i]) * inv_v)
            ok[k] &= bool(-LIMIT <= q < LIMIT)
            g[k, i] = int(q)
    return g, ok


def fresh_any(g, ok):
    out = []
    for k in range(len(g)):
        out.append(bool(ok[k]) and not any(ok[j] and (g[j] == g[k]).all() for j in range(k)))
    return out


def fresh_prev(g, ok):
    return [bool(ok[k]) and not (k > 0 and ok[k - 1] and (g[k - 1] == g[k]).all())
            for k in range(len(g))]


def rays(rng, n):
    out = []
    for _ in range(n):
        kind = rng.integers(5)
        d = rng.normal(size=3)
        if kind == 1:                       # along an axis, either sign
            d = np.zeros(3)
            d[rng.integers(3)] = rng.choice([-1.0, 1.0])
        elif kind == 2:                     # near an axis
            d = np.zeros(3)
            d[rng.integers(3)] = 1.0
            d += rng.normal(scale=1e-6, size=3)
        d = (d / np.linalg.norm(d)).astype(F32)
        v = F32(rng.choice([0.005, 0.01, 0.02, 0.05, 0.0137]))
        p = rng.uniform(-3, 3, size=3)
        if kind == 3:                       # through voxel boundaries
            p = (np.round(p / v) * v).astype(F32)
        if kind == 4:                       # across the coordinate limit
            p[rng.integers(3)] = float(LIMIT) * float(v) * rng.choice([-1.0, 1.0])
        out.append((p.astype(F32), d, v, int(rng.choice([2, 4, 8]))))
    return out


def test_voxel_coordinates_are_monotone_along_the_band():
    rng = np.random.default_rng(20261203)
    for P, D, v, M in rays(rng, 400):
        g, ok = walk(P, D, v, M)
        idx = np.nonzero(ok)[0]
        if len(idx):
            assert (np.diff(idx) == 1).all()            # in-range samples are consecutive
        for i in range(3):
            d = np.diff(g[ok, i])
            assert (d >= 0).all() or (d <= 0).all(), (P, D, v, M, i)


def test_previous_sample_dedupe_equals_any_earlier_dedupe():
    rng = np.random.default_rng(7)
    repeats = 0
    for P, D, v, M in rays(rng, 400):
        g, ok = walk(P, D, v, M)
        a, b = fresh_any(g, ok), fresh_prev(g, ok)
        assert a == b, (P, D, v, M)
        repeats += sum(ok) - sum(a)
    assert repeats > 50         # the rule was exercised: samples do repeat a voxel
