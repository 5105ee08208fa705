"""CPU oracle for hash-blocked TSDF fusion -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product (the CUDA library and its
Python binding) never imports, links or executes anything here, and this
package imports nothing from the product.

``tsdf_oracle.cpp`` is a plain single-threaded C++ implementation of the
*definition* of a fused frame (paper Section 2; readings R1-R6 are stated in
its header comment). This module compiles it with g++ (contraction off) and
wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsdf_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtsdf_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 3: "POOL_FULL", 4: "TABLE_FULL", 7: "POISONED"}
STAT_FIELDS = ("points", "samples", "contributions", "unique_voxels", "unique_blocks",
               "new_blocks", "range_rejects", "over_pool")
CHANNELS = ("tsdf", "weight", "r", "g", "b")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_create.restype = ctypes.c_void_p
            L.oracle_create.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_uint32,
                                        ctypes.c_uint32]
            L.oracle_destroy.argtypes = [ctypes.c_void_p]
            L.oracle_reset.argtypes = [ctypes.c_void_p]
            L.oracle_block_count.restype = ctypes.c_uint32
            L.oracle_block_count.argtypes = [ctypes.c_void_p]
            L.oracle_fuse.restype = ctypes.c_int
            L.oracle_fuse.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
            L.oracle_export_some.restype = None
            L.oracle_export_some.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                             ctypes.c_void_p, ctypes.c_void_p]
            L.oracle_extract.restype = ctypes.c_uint32
            L.oracle_extract.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_uint32]
            L.oracle_set_voxel.restype = ctypes.c_int
            L.oracle_set_voxel.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_double, ctypes.c_uint32]
            L.oracle_export.restype = ctypes.c_uint32
            L.oracle_export.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_uint32]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleVolume:
    """A fused volume computed by the CPU oracle."""

    def __init__(self, voxel_size, truncation, table_slots, pool_blocks):
        self._L = lib()
        self._h = self._L.oracle_create(voxel_size, truncation, table_slots, pool_blocks)
        if not self._h:
            raise ValueError("oracle_create rejected the volume parameters")
        self.voxel_size = float(voxel_size)
        self.truncation = float(truncation)
        self.last_stats = None

    def close(self):
        if self._h:
            self._L.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        self._L.oracle_reset(self._h)

    def fuse(self, depth, intr, pose, rgb=None) -> str:
        depth = np.ascontiguousarray(depth, dtype=np.float32)
        H, W = depth.shape
        intr = np.ascontiguousarray(intr, dtype=np.float32).reshape(4)
        pose = np.ascontiguousarray(pose, dtype=np.float32).reshape(16)
        if rgb is not None:
            rgb = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(H, W, 3)
        st = np.zeros(8, dtype=np.uint64)
        code = self._L.oracle_fuse(self._h, _ptr(depth), W, H, _ptr(intr), _ptr(pose),
                                   _ptr(rgb), _ptr(st))
        self.last_stats = dict(zip(STAT_FIELDS, (int(x) for x in st)))
        return STATUS_NAMES.get(code, f"UNKNOWN({code})")

    def fuse_frame(self, frame, with_rgb=True) -> str:
        return self.fuse(frame.depth, frame.intr, frame.pose, frame.rgb if with_rgb else None)

    def block_count(self) -> int:
        return int(self._L.oracle_block_count(self._h))

    def export(self, double=False):
        """(coords int32 (n,3), voxels (n,5,512)) ordered by block coordinate."""
        n = int(self._L.oracle_export(self._h, None, None, None, 0))
        coords = np.zeros((n, 3), dtype=np.int32)
        vox = np.zeros((n, 5, 512), dtype=np.float64 if double else np.float32)
        if n:
            self._L.oracle_export(self._h, _ptr(coords), None if double else _ptr(vox),
                                  _ptr(vox) if double else None, n)
        return coords, vox

    def export_coords(self):
        """Block coordinates only, (n, 3) int32, ordered by coordinate."""
        n = int(self._L.oracle_export(self._h, None, None, None, 0))
        coords = np.zeros((n, 3), dtype=np.int32)
        if n:
            self._L.oracle_export(self._h, _ptr(coords), None, None, n)
        return coords

    def extract(self):
        """Marching tetrahedra (readings E1-E4 in tsdf_oracle.cpp):
        (triangles (n,3,3) float64, cells (n,4) int32 {gx, gy, gz, 2*tet+sub})."""
        n = int(self._L.oracle_extract(self._h, None, None, 0))
        tris = np.zeros((n, 3, 3), dtype=np.float64)
        cells = np.zeros((n, 4), dtype=np.int32)
        if n:
            self._L.oracle_extract(self._h, _ptr(tris), _ptr(cells), n)
        return tris, cells

    def set_voxel(self, gx, gy, gz, tsdf_sum, weight=1):
        """Write one voxel's tsdf sum and weight directly (hand-built grids)."""
        if self._L.oracle_set_voxel(self._h, int(gx), int(gy), int(gz), float(tsdf_sum),
                                    int(weight)):
            raise ValueError("pool exhausted")

    def export_some(self, coords):
        """(found (n,) bool, voxels (n,5,512) float64) for the given block coordinates."""
        coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 3)
        n = len(coords)
        vox = np.zeros((n, 5, 512), dtype=np.float64)
        found = np.zeros(n, dtype=np.uint8)
        if n:
            self._L.oracle_export_some(self._h, _ptr(coords), n, _ptr(vox), _ptr(found))
        return found.astype(bool), vox
