"""Test helpers: convert per-block exports to global-voxel dictionaries.

An export is (coords (n,3) int32, vox (n,5,512)) with channel order
(tsdf mean, weight, red, green, blue) and local voxel index
l = lx + 8*ly + 64*lz inside an 8^3 block (the library's documented layout).
"""
import numpy as np

_L = np.arange(512)
_LOCAL = np.stack([_L % 8, (_L // 8) % 8, _L // 64], axis=1)


def voxel_arrays(coords, vox):
    """(global voxel coords (m,3) int64, values (m,5)) of voxels with weight > 0, sorted."""
    coords = np.asarray(coords, dtype=np.int64)
    vox = np.asarray(vox)
    bi, li = np.nonzero(vox[:, 1, :] > 0)
    g = coords[bi] * 8 + _LOCAL[li]
    vals = vox[bi, :, li]
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0]))
    return g[order], vals[order]


def voxel_dict(coords, vox):
    g, vals = voxel_arrays(coords, vox)
    return {tuple(int(x) for x in gi): tuple(float(y) for y in vi) for gi, vi in zip(g, vals)}


def sort_blocks(coords, vox):
    coords = np.asarray(coords)
    order = np.lexsort((coords[:, 2], coords[:, 1], coords[:, 0]))
    return coords[order], np.asarray(vox)[order]
