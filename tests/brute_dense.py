"""Second, independent statement of one fused frame, for pinning the oracle.

A vectorised numpy formulation over a DENSE voxel grid (no blocks, no map, no
hash): every sample of every point is computed at once, duplicates within a
point are masked, and contributions are scattered with ``np.add.at`` into a
dense array spanning the bounding box of the accepted voxels. It follows the
same definition as the oracle (paper Section 2 plus readings R1-R6 in the
oracle's header) but shares none of its code, data structures or loop order.

Single-precision rounding is reproduced per operation: numpy float32 arrays
round every +, -, *, /, sqrt to nearest-even; fused multiply-add is emulated
exactly with the round-to-odd method of Boldo and Melquiond ("Emulation of FMA
and correctly rounded sums: proved algorithms using rounding to odd", IEEE
Trans. Computers 57(4), 2008): the float64 sum of the exact float64 product and
the addend is rounded to odd, then to float32.

Intended for tiny frames only (a few thousand points).
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def fma32(a, b, c):
    """Correctly rounded float32 fused multiply-add a*b + c (element-wise)."""
    a = np.asarray(a, dtype=F32).astype(np.float64)
    b = np.asarray(b, dtype=F32).astype(np.float64)
    c = np.asarray(c, dtype=F32).astype(np.float64)
    p = a * b                      # exact: 24 + 24 significant bits <= 53
    s = p + c                      # rounded to nearest float64
    # TwoSum: exact error e with p + c = s + e
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    # round to odd: if inexact and the last significand bit is even, step toward e
    bits = s.view(np.uint64)
    even = (bits & np.uint64(1)) == 0
    fix = (e != 0) & even & np.isfinite(s)
    toward = np.where(e > 0, np.inf, -np.inf)
    s = np.where(fix, np.nextafter(s, toward), s)
    return s.astype(F32)


def fuse_dense(depth, intr, pose, voxel, trunc, rgb=None):
    """Return {(gx, gy, gz): (weight, tsdf_mean, r, g, b)} for one frame into an empty volume."""
    depth = np.asarray(depth, dtype=F32)
    H, W = depth.shape
    fx, fy, cx, cy = (F32(x) for x in np.asarray(intr, dtype=F32))
    P = np.asarray(pose, dtype=F32).reshape(4, 4)
    R = P[:3, :3]
    t = P[:3, 3]
    v = F32(voxel)
    tau = F32(trunc)
    inv_v = F32(1.0) / v
    M = int(np.rint(np.float32(tau / v)))   # round half to even, like lrintf

    vv, uu = np.nonzero(np.isfinite(depth) & (depth > 0))
    d = depth[vv, uu]
    u = uu.astype(F32)
    w = vv.astype(F32)
    rx = (u - cx) / fx
    ry = (w - cy) / fy
    pc = [rx * d, ry * d, d]
    n = np.sqrt(fma32(rx, rx, fma32(ry, ry, F32(1.0))))
    dr = [rx / n, ry / n, F32(1.0) / n]
    # the ray in the world frame: start P = R p + t, direction D = R d
    Pw = [fma32(R[i, 2], pc[2], fma32(R[i, 1], pc[1], fma32(R[i, 0], pc[0], t[i])))
          for i in range(3)]
    Dw = [fma32(R[i, 2], dr[2], fma32(R[i, 1], dr[1], R[i, 0] * dr[0])) for i in range(3)]

    K = 2 * M + 1
    npts = d.shape[0]
    G = np.zeros((K, npts, 3), dtype=np.int64)
    ok = np.ones((K, npts), dtype=bool)
    for k in range(K):
        tk = F32(k - M) * v
        for i in range(3):
            sw = fma32(tk, Dw[i], Pw[i])
            fg = np.floor(sw * inv_v)
            ok[k] &= (fg >= F32(-8388608.0)) & (fg < F32(8388608.0))
            G[k, :, i] = np.where(np.isfinite(fg), fg, 0).astype(np.int64)
    # each distinct voxel once per point: drop sample k if an earlier sample hit it
    first = np.ones((K, npts), dtype=bool)
    for k in range(K):
        for j in range(k):
            first[k] &= ~np.all(G[k] == G[j], axis=1)
    keep = ok & first

    # voxel centre in the camera frame, c = A g + b: A = v R^T, b = R^T (v/2 - t)
    gf = G.astype(F32)
    h = [fma32(F32(0.5), v, -t[i]) for i in range(3)]
    A = [[v * R[i, j] for i in range(3)] for j in range(3)]
    b = [fma32(R[2, j], h[2], fma32(R[1, j], h[1], R[0, j] * h[0])) for j in range(3)]
    cc = [fma32(A[j][2], gf[:, :, 2], fma32(A[j][1], gf[:, :, 1], fma32(A[j][0], gf[:, :, 0], b[j])))
          for j in range(3)]
    zc = cc[2]
    front = zc > F32(0.0)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        iz = F32(1.0) / np.where(front, zc, F32(1.0))
        qu = np.floor(fma32(fx, cc[0] * iz, cx) + F32(0.5))
        qv = np.floor(fma32(fy, cc[1] * iz, cy) + F32(0.5))
    inside = front & (qu >= 0) & (qu < F32(W)) & (qv >= 0) & (qv < F32(H))
    qi = np.where(inside, qu, 0).astype(np.int64)
    qj = np.where(inside, qv, 0).astype(np.int64)
    d2 = depth[qj, qi]
    with np.errstate(invalid="ignore"):
        seen = inside & np.isfinite(d2) & (d2 > 0) & ((d2 - zc) >= -tau)
    acc = keep & seen
    sdf = d[None, :] - zc
    tsdf = np.minimum(F32(1.0), np.maximum(F32(-1.0), sdf / tau))

    if not acc.any():
        return {}
    ks, ps = np.nonzero(acc)
    g = G[ks, ps]
    lo = g.min(axis=0)
    ext = g.max(axis=0) - lo + 1
    flat = np.ravel_multi_index((g - lo).T, ext)
    size = int(np.prod(ext))
    wsum = np.zeros(size, dtype=np.int64)
    tsum = np.zeros(size, dtype=np.float64)
    np.add.at(wsum, flat, 1)
    np.add.at(tsum, flat, tsdf[ks, ps].astype(np.float64))
    csum = np.zeros((3, size), dtype=np.float64)
    if rgb is not None:
        col = np.asarray(rgb, dtype=np.uint8)[vv, uu].astype(np.float64) / 255.0
        for c in range(3):
            np.add.at(csum[c], flat, col[ps, c])
    out = {}
    for f in np.nonzero(wsum)[0]:
        gi = tuple(int(x) for x in (np.array(np.unravel_index(f, ext)) + lo))
        wv = wsum[f]
        out[gi] = (int(wv), tsum[f] / wv, csum[0, f] / wv, csum[1, f] / wv, csum[2, f] / wv)
    return out
