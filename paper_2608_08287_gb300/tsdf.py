"""Python binding of libtsdf (include/tsdf.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
computation of its own. Device buffers may be given as torch CUDA tensors or
as raw device addresses (int); streams as torch streams, raw cudaStream_t
handles (int) or None (the legacy default stream, which is PyTorch's default
stream).

The CUDA library must be built (``paper_2608_08287_gb300.build``); if it is
missing, importing a function fails loudly -- there is no CPU fallback. With
the environment variable TSDF_CHECKED=1 the checked build is loaded instead
(every pool, table, coordinate and image index range-checked on the device).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, LIB_CHECKED

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "POOL_FULL", 4: "TABLE_FULL",
          5: "PUBLISH_TIMEOUT", 6: "BOUNDS", 7: "POISONED", 8: "CUDA"}
OPTIONS = {"probe_load": 0, "publish_timeout_ns": 1, "integrate_mode": 2, "threads": 3,
           "allocate_mode": 4, "fuse_mode": 5, "ctas_per_sm": 6, "use_graph": 7,
           "slot_index": 8, "probe_bound": 9, "threads_per_point": 10,
           "batch_stages": 11, "batch_streams": 12}
ERRBITS = {"POOL_FULL": 1, "TABLE_FULL": 2, "PUBLISH_TIMEOUT": 4, "BOUNDS": 8}
EMPTY_KEY = 0xFFFFFFFFFFFFFFFF
NOALLOC_MAX_PIXELS = 1 << 20
CHANNELS = ("tsdf", "weight", "r", "g", "b")

EXPORTED = ("tsdf_volume_bytes", "tsdf_volume_create", "tsdf_volume_create_in",
            "tsdf_volume_reset", "tsdf_volume_destroy", "tsdf_volume_set_option",
            "tsdf_volume_layout", "tsdf_fuse_frame", "tsdf_fuse_frame_async",
            "tsdf_fuse_frame_host", "tsdf_fuse_frame_host_noalloc", "tsdf_fuse_frames_host",
            "tsdf_allocate_async",
            "tsdf_integrate_async",
            "tsdf_volume_status", "tsdf_volume_block_count", "tsdf_export_blocks",
            "tsdf_block_key", "tsdf_block_slot", "tsdf_status_string", "tsdf_version",
            "tsdf_launch_count", "tsdf_batch_create", "tsdf_batch_destroy",
            "tsdf_batch_set_option", "tsdf_fuse_batch_async", "tsdf_batch_status",
            "tsdf_server_create", "tsdf_server_destroy", "tsdf_server_clock",
            "tsdf_server_submit", "tsdf_server_poll", "tsdf_server_pending",
            "tsdf_server_replay", "tsdf_volume_table_stats", "tsdf_volume_copy",
            "tsdf_autotune_frame", "tsdf_batch_autotune", "tsdf_extract_mesh_async",
            "tsdf_extract_mesh", "tsdf_volume_checkpoint_bytes", "tsdf_volume_save",
            "tsdf_volume_load", "tsdf_set_l2_fetch_bytes")


class tsdf_intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float)]


class tsdf_pose(ctypes.Structure):
    _fields_ = [("m", ctypes.c_float * 16)]


class tsdf_layout(ctypes.Structure):
    _fields_ = [("base", ctypes.c_void_p), ("bytes", ctypes.c_size_t),
                ("block_count", ctypes.c_void_p), ("error_word", ctypes.c_void_p),
                ("table", ctypes.c_void_p), ("block_coords", ctypes.c_void_p),
                ("voxel_sums", ctypes.c_void_p), ("blue_sums", ctypes.c_void_p),
                ("table_slots", ctypes.c_uint32), ("pool_blocks", ctypes.c_uint32),
                ("table_offset", ctypes.c_size_t), ("coords_offset", ctypes.c_size_t),
                ("voxel_sums_offset", ctypes.c_size_t), ("blue_sums_offset", ctypes.c_size_t)]


class tsdf_table_stats(ctypes.Structure):
    _fields_ = [("occupied_slots", ctypes.c_uint64), ("probe_sum", ctypes.c_uint64),
                ("probe_max", ctypes.c_uint32), ("blocks", ctypes.c_uint32),
                ("weight_sum", ctypes.c_uint64)]


class tsdf_tuning(ctypes.Structure):
    _fields_ = [("allocate_mode", ctypes.c_int), ("integrate_mode", ctypes.c_int),
                ("fuse_mode", ctypes.c_int), ("probe_load", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("candidates", ctypes.c_int), ("best_ms", ctypes.c_float),
                ("default_ms", ctypes.c_float), ("threads_per_point", ctypes.c_int),
                ("batch_streams", ctypes.c_int)]


class tsdf_extract_timing(ctypes.Structure):
    _fields_ = [("compute_ms", ctypes.c_float), ("d2h_ms", ctypes.c_float),
                ("d2h_bytes", ctypes.c_uint64)]


class tsdf_frame(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("intr", tsdf_intrinsics), ("pose", tsdf_pose)]


class tsdf_request(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("intr", tsdf_intrinsics), ("pose", tsdf_pose),
                ("arrival_s", ctypes.c_double), ("tag", ctypes.c_uint64),
                ("reset_volume", ctypes.c_int)]


class tsdf_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("arrival_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("status", ctypes.c_int)]


class TsdfError(RuntimeError):
    def __init__(self, status: str, where: str = ""):
        super().__init__(f"{where}: TSDF_ERR_{status}" if where else f"TSDF_ERR_{status}")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """The loaded libtsdf.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = LIB_CHECKED if os.environ.get("TSDF_CHECKED") == "1" else LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"libtsdf.so is not built ({path}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(path)
        st = ctypes.c_int
        sig = {
            "tsdf_volume_bytes": (ctypes.c_size_t, [ctypes.c_uint32, ctypes.c_uint32]),
            "tsdf_volume_create": (st, [ctypes.c_float, ctypes.c_float, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.POINTER(_P)]),
            "tsdf_volume_create_in": (st, [_P, ctypes.c_size_t, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_uint32, ctypes.c_uint32, _P,
                                           ctypes.POINTER(_P)]),
            "tsdf_volume_reset": (st, [_P, _P]),
            "tsdf_volume_destroy": (None, [_P]),
            "tsdf_volume_set_option": (st, [_P, ctypes.c_int, ctypes.c_int64]),
            "tsdf_volume_layout": (st, [_P, ctypes.POINTER(tsdf_layout)]),
            "tsdf_fuse_frame": (st, [_P, _P, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(tsdf_intrinsics), ctypes.POINTER(tsdf_pose),
                                     _P, _P]),
            "tsdf_fuse_frame_async": (st, [_P, _P, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(tsdf_intrinsics),
                                           ctypes.POINTER(tsdf_pose), _P, _P]),
            "tsdf_fuse_frame_host": (st, [_P, _P, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(tsdf_intrinsics),
                                          ctypes.POINTER(tsdf_pose), _P, _P]),
            "tsdf_fuse_frame_host_noalloc": (st, [_P, _P, ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(tsdf_intrinsics),
                                                  ctypes.POINTER(tsdf_pose), _P, _P]),
            "tsdf_fuse_frames_host": (st, [ctypes.POINTER(tsdf_frame), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), _P]),
            "tsdf_allocate_async": (st, [_P, _P, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(tsdf_intrinsics),
                                         ctypes.POINTER(tsdf_pose), _P]),
            "tsdf_integrate_async": (st, [_P, _P, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(tsdf_intrinsics),
                                          ctypes.POINTER(tsdf_pose), _P, _P]),
            "tsdf_volume_status": (st, [_P, _P]),
            "tsdf_volume_block_count": (st, [_P, _P, ctypes.POINTER(ctypes.c_uint32)]),
            "tsdf_export_blocks": (st, [_P, _P, _P, ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_uint32), _P]),
            "tsdf_block_key": (ctypes.c_uint64, [ctypes.c_int32] * 3),
            "tsdf_block_slot": (ctypes.c_uint32, [ctypes.c_int32] * 3 + [ctypes.c_uint32]),
            "tsdf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "tsdf_version": (ctypes.c_char_p, []),
            "tsdf_launch_count": (ctypes.c_uint64, []),
            "tsdf_set_l2_fetch_bytes": (st, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
            "tsdf_batch_create": (st, [ctypes.c_int, ctypes.POINTER(_P)]),
            "tsdf_batch_destroy": (None, [_P]),
            "tsdf_batch_set_option": (st, [_P, ctypes.c_int, ctypes.c_int64]),
            "tsdf_fuse_batch_async": (st, [_P, ctypes.POINTER(tsdf_frame), ctypes.c_int, _P]),
            "tsdf_batch_status": (st, [_P, _P, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
            "tsdf_server_create": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P)]),
            "tsdf_server_destroy": (None, [_P]),
            "tsdf_server_clock": (ctypes.c_double, [_P]),
            "tsdf_server_submit": (st, [_P, ctypes.POINTER(tsdf_request)]),
            "tsdf_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(tsdf_completion),
                                                ctypes.c_int]),
            "tsdf_server_pending": (ctypes.c_int, [_P]),
            "tsdf_server_replay": (st, [_P, ctypes.POINTER(tsdf_request), ctypes.c_int,
                                        ctypes.POINTER(tsdf_completion)]),
            "tsdf_volume_table_stats": (st, [_P, _P, ctypes.POINTER(tsdf_table_stats)]),
            "tsdf_volume_copy": (st, [_P, _P, _P]),
            "tsdf_volume_checkpoint_bytes": (ctypes.c_size_t, [_P]),
            "tsdf_volume_save": (st, [_P, _P, ctypes.c_size_t, _P]),
            "tsdf_volume_load": (st, [_P, _P, ctypes.c_size_t, _P]),
            "tsdf_extract_mesh_async": (st, [_P, _P, _P, ctypes.c_uint32, _P, _P]),
            "tsdf_extract_mesh": (st, [_P, _P, _P, ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(tsdf_extract_timing), _P]),
            "tsdf_autotune_frame": (st, [_P, _P, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(tsdf_intrinsics),
                                         ctypes.POINTER(tsdf_pose), _P, ctypes.c_int, _P,
                                         ctypes.POINTER(tsdf_tuning)]),
            "tsdf_batch_autotune": (st, [_P, ctypes.POINTER(tsdf_frame), ctypes.c_int,
                                         ctypes.c_int, _P, ctypes.POINTER(tsdf_tuning)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------
def _dptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_cuda") and not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device address of {type(x)}")


def _hptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("expected a C-contiguous array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if getattr(x, "is_cuda", False):
            raise ValueError("expected a host tensor")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot take a host address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s or None
    return getattr(s, "cuda_stream", 0) or None


def intrinsics(intr) -> tsdf_intrinsics:
    """A tsdf_intrinsics struct from (fx, fy, cx, cy) (or the struct itself)."""
    if isinstance(intr, tsdf_intrinsics):
        return intr
    return tsdf_intrinsics(*[float(x) for x in np.asarray(intr, dtype=np.float32).reshape(4)])


def pose_struct(pose) -> tsdf_pose:
    """A tsdf_pose struct from a 4x4 row-major matrix (or the struct itself)."""
    if isinstance(pose, tsdf_pose):
        return pose
    p = tsdf_pose()
    ctypes.memmove(p.m, np.ascontiguousarray(pose, dtype=np.float32).reshape(16).ctypes.data,
                   64)
    return p


def _intr(intr):
    return ctypes.byref(intrinsics(intr))


def _pose(pose):
    return ctypes.byref(pose_struct(pose))


def _st(code: int) -> str:
    return STATUS.get(int(code), f"UNKNOWN({code})")


# ----------------------------------------------------------------------------
# the C entry points
# ----------------------------------------------------------------------------
def tsdf_volume_bytes(table_slots: int, pool_blocks: int) -> int:
    return int(lib().tsdf_volume_bytes(table_slots, pool_blocks))


def tsdf_volume_create(voxel_size, truncation, table_slots, pool_blocks):
    h = _P()
    st = _st(lib().tsdf_volume_create(voxel_size, truncation, table_slots, pool_blocks,
                                      ctypes.byref(h)))
    if st != "OK":
        raise TsdfError(st, "tsdf_volume_create")
    return h


def tsdf_volume_create_in(dev_mem, nbytes, voxel_size, truncation, table_slots, pool_blocks,
                          stream=None):
    h = _P()
    st = _st(lib().tsdf_volume_create_in(_dptr(dev_mem), nbytes, voxel_size, truncation,
                                         table_slots, pool_blocks, _stream(stream),
                                         ctypes.byref(h)))
    if st != "OK":
        raise TsdfError(st, "tsdf_volume_create_in")
    return h


def tsdf_volume_reset(vol, stream=None) -> str:
    return _st(lib().tsdf_volume_reset(vol, _stream(stream)))


def tsdf_volume_destroy(vol) -> None:
    lib().tsdf_volume_destroy(vol)


def tsdf_volume_set_option(vol, option, value) -> str:
    opt = OPTIONS[option] if isinstance(option, str) else int(option)
    return _st(lib().tsdf_volume_set_option(vol, opt, int(value)))


def tsdf_volume_layout(vol) -> tsdf_layout:
    out = tsdf_layout()
    st = _st(lib().tsdf_volume_layout(vol, ctypes.byref(out)))
    if st != "OK":
        raise TsdfError(st, "tsdf_volume_layout")
    return out


def tsdf_fuse_frame(vol, depth, width, height, intr, pose, rgb=None, stream=None) -> str:
    return _st(lib().tsdf_fuse_frame(vol, _dptr(depth), width, height, _intr(intr), _pose(pose),
                                     _dptr(rgb), _stream(stream)))


def tsdf_fuse_frame_async(vol, depth, width, height, intr, pose, rgb=None, stream=None) -> str:
    return _st(lib().tsdf_fuse_frame_async(vol, _dptr(depth), width, height, _intr(intr),
                                           _pose(pose), _dptr(rgb), _stream(stream)))


def tsdf_fuse_frame_host(vol, depth, width, height, intr, pose, rgb=None, stream=None) -> str:
    return _st(lib().tsdf_fuse_frame_host(vol, _hptr(depth), width, height, _intr(intr),
                                          _pose(pose), _hptr(rgb), _stream(stream)))


def tsdf_fuse_frame_host_noalloc(vol, depth, width, height, intr, pose, rgb=None,
                                 stream=None) -> str:
    """Host-input fusion that allocates nothing: the frame is staged in a fixed
    array inside the library (at most NOALLOC_MAX_PIXELS pixels), for callers
    that cannot let the library call cudaMalloc."""
    return _st(lib().tsdf_fuse_frame_host_noalloc(vol, _hptr(depth), width, height, _intr(intr),
                                                  _pose(pose), _hptr(rgb), _stream(stream)))


def tsdf_allocate_async(vol, depth, width, height, intr, pose, stream=None) -> str:
    return _st(lib().tsdf_allocate_async(vol, _dptr(depth), width, height, _intr(intr),
                                         _pose(pose), _stream(stream)))


def tsdf_integrate_async(vol, depth, width, height, intr, pose, rgb=None, stream=None) -> str:
    return _st(lib().tsdf_integrate_async(vol, _dptr(depth), width, height, _intr(intr),
                                          _pose(pose), _dptr(rgb), _stream(stream)))


def tsdf_volume_status(vol, stream=None) -> str:
    return _st(lib().tsdf_volume_status(vol, _stream(stream)))


def tsdf_volume_block_count(vol, stream=None) -> int:
    n = ctypes.c_uint32()
    st = _st(lib().tsdf_volume_block_count(vol, _stream(stream), ctypes.byref(n)))
    if st != "OK":
        raise TsdfError(st, "tsdf_volume_block_count")
    return int(n.value)


def tsdf_export_blocks(vol, stream=None, voxels=True):
    """(coords int32 (n,3), voxels float32 (n,5,512) or None) in pool order."""
    n = ctypes.c_uint32()
    st = _st(lib().tsdf_export_blocks(vol, None, None, 0, ctypes.byref(n), _stream(stream)))
    if st != "OK":
        raise TsdfError(st, "tsdf_export_blocks")
    coords = np.zeros((n.value, 3), dtype=np.int32)
    vox = np.zeros((n.value, 5, 512), dtype=np.float32) if voxels else None
    if n.value:
        m = ctypes.c_uint32()
        st = _st(lib().tsdf_export_blocks(vol, coords.ctypes.data,
                                          vox.ctypes.data if voxels else None, n.value,
                                          ctypes.byref(m), _stream(stream)))
        if st != "OK":
            raise TsdfError(st, "tsdf_export_blocks")
    return coords, vox


def tsdf_volume_table_stats(vol, stream=None) -> dict:
    out = tsdf_table_stats()
    st = _st(lib().tsdf_volume_table_stats(vol, _stream(stream), ctypes.byref(out)))
    if st != "OK":
        raise TsdfError(st, "tsdf_volume_table_stats")
    return {k: int(getattr(out, k)) for k, _ in tsdf_table_stats._fields_}


def tsdf_volume_copy(dst, src, stream=None) -> str:
    return _st(lib().tsdf_volume_copy(dst, src, _stream(stream)))


def tsdf_volume_checkpoint_bytes(vol) -> int:
    return int(lib().tsdf_volume_checkpoint_bytes(vol))


def tsdf_volume_save(vol, stream=None):
    """(status, the checkpoint as a uint8 numpy array, or None)."""
    n = tsdf_volume_checkpoint_bytes(vol)
    buf = np.empty(max(n, 1), dtype=np.uint8)
    st = _st(lib().tsdf_volume_save(vol, buf.ctypes.data if n else None, n, _stream(stream)))
    return st, (buf if st == "OK" else None)


def tsdf_volume_load(vol, checkpoint, stream=None) -> str:
    """checkpoint: a uint8 numpy array (or bytes) written by tsdf_volume_save."""
    buf = np.ascontiguousarray(np.frombuffer(checkpoint, dtype=np.uint8)
                               if isinstance(checkpoint, (bytes, bytearray)) else checkpoint,
                               dtype=np.uint8)
    return _st(lib().tsdf_volume_load(vol, buf.ctypes.data if buf.size else None, buf.size,
                                      _stream(stream)))


def tsdf_extract_mesh_async(vol, triangles, cells, capacity, count, stream=None) -> str:
    """Device buffers (torch tensors or addresses): triangles (cap, 9) float32,
    cells (cap, 4) int32, count a uint32/int32 device scalar."""
    return _st(lib().tsdf_extract_mesh_async(vol, _dptr(triangles), _dptr(cells), int(capacity),
                                             _dptr(count), _stream(stream)))


def tsdf_extract_mesh(vol, stream=None, cells=True):
    """(triangles float32 (n,3,3), cells int32 (n,4) or None, timing dict)."""
    n = ctypes.c_uint32()
    st = _st(lib().tsdf_extract_mesh(vol, None, None, 0, ctypes.byref(n), None,
                                     _stream(stream)))
    if st != "OK":
        raise TsdfError(st, "tsdf_extract_mesh")
    tris = np.zeros((n.value, 3, 3), dtype=np.float32)
    cel = np.zeros((n.value, 4), dtype=np.int32) if cells else None
    t = tsdf_extract_timing()
    if n.value:
        m = ctypes.c_uint32()
        st = _st(lib().tsdf_extract_mesh(vol, tris.ctypes.data, cel.ctypes.data if cells else None,
                                         n.value, ctypes.byref(m), ctypes.byref(t),
                                         _stream(stream)))
        if st != "OK":
            raise TsdfError(st, "tsdf_extract_mesh")
    return tris, cel, {"compute_ms": float(t.compute_ms), "d2h_ms": float(t.d2h_ms),
                       "d2h_bytes": int(t.d2h_bytes)}


def _tuning(t):
    return {k: (float(getattr(t, k)) if k.endswith("_ms") else int(getattr(t, k)))
            for k, _ in tsdf_tuning._fields_}


def tsdf_autotune_frame(vol, depth, width, height, intr, pose, rgb=None, reps=5,
                        stream=None):
    """(status, tuning dict or None)."""
    out = tsdf_tuning()
    st = _st(lib().tsdf_autotune_frame(vol, _dptr(depth), int(width), int(height), _intr(intr),
                                       _pose(pose), _dptr(rgb), int(reps), _stream(stream),
                                       ctypes.byref(out)))
    return st, (_tuning(out) if st == "OK" else None)


def tsdf_batch_autotune(batch, frames, n=None, reps=5, stream=None):
    """(status, tuning dict or None) for a ctypes array of tsdf_frame."""
    n = len(frames) if n is None else n
    out = tsdf_tuning()
    st = _st(lib().tsdf_batch_autotune(batch, frames, int(n), int(reps), _stream(stream),
                                       ctypes.byref(out)))
    return st, (_tuning(out) if st == "OK" else None)


def tsdf_block_key(bx, by, bz) -> int:
    return int(lib().tsdf_block_key(bx, by, bz))


def tsdf_block_slot(bx, by, bz, table_slots) -> int:
    return int(lib().tsdf_block_slot(bx, by, bz, table_slots))


def tsdf_status_string(code: int) -> str:
    return lib().tsdf_status_string(code).decode()


def tsdf_version() -> str:
    return lib().tsdf_version().decode()


def tsdf_set_l2_fetch_bytes(nbytes):
    """(status, the previous value) of the context-wide L2 fetch granularity."""
    prev = ctypes.c_int(0)
    st = _st(lib().tsdf_set_l2_fetch_bytes(int(nbytes), ctypes.byref(prev)))
    return st, prev.value


def tsdf_launch_count() -> int:
    return int(lib().tsdf_launch_count())


def tsdf_batch_create(max_frames):
    h = _P()
    st = _st(lib().tsdf_batch_create(max_frames, ctypes.byref(h)))
    if st != "OK":
        raise TsdfError(st, "tsdf_batch_create")
    return h


def tsdf_batch_destroy(batch) -> None:
    lib().tsdf_batch_destroy(batch)


def tsdf_batch_set_option(batch, option, value) -> str:
    opt = OPTIONS[option] if isinstance(option, str) else int(option)
    return _st(lib().tsdf_batch_set_option(batch, opt, int(value)))


def make_frames(items):
    """ctypes array of tsdf_frame from (volume handle, depth, rgb, intr, pose) tuples;
    depth is a CUDA tensor (H, W) or (address, width, height)."""
    arr = (tsdf_frame * len(items))()
    for i, (vol, depth, rgb, intr, pose) in enumerate(items):
        if isinstance(depth, tuple):
            addr, w, h = depth
        else:
            addr, h, w = _dptr(depth), depth.shape[-2], depth.shape[-1]
        arr[i].volume = vol.value if isinstance(vol, ctypes.c_void_p) else vol
        arr[i].depth = addr
        arr[i].rgb = _dptr(rgb)
        arr[i].width = int(w)
        arr[i].height = int(h)
        arr[i].intr = intrinsics(intr)
        arr[i].pose = pose_struct(pose)
    return arr


def make_host_frames(items):
    """ctypes array of tsdf_frame with HOST buffers, from (volume handle, depth,
    rgb, intr, pose) tuples; depth and rgb are numpy arrays or CPU tensors
    (rgb may be None)."""
    arr = (tsdf_frame * len(items))()
    for i, (vol, depth, rgb, intr, pose) in enumerate(items):
        arr[i].volume = vol.value if isinstance(vol, ctypes.c_void_p) else vol
        arr[i].depth = _hptr(depth)
        arr[i].rgb = _hptr(rgb)
        arr[i].height, arr[i].width = int(depth.shape[-2]), int(depth.shape[-1])
        arr[i].intr = intrinsics(intr)
        arr[i].pose = pose_struct(pose)
    return arr


def tsdf_fuse_frames_host(frames, n=None, stream=None):
    """(status, [per-frame status]) for a ctypes array of tsdf_frame with host
    buffers (make_host_frames)."""
    n = len(frames) if n is None else n
    out = (ctypes.c_int * max(1, n))()
    st = _st(lib().tsdf_fuse_frames_host(frames, n, out, _stream(stream)))
    return st, [_st(out[i]) for i in range(n)]


def tsdf_fuse_batch_async(batch, frames, n=None, stream=None) -> str:
    n = len(frames) if n is None else n
    return _st(lib().tsdf_fuse_batch_async(batch, frames, n, _stream(stream)))


def tsdf_batch_status(batch, n, stream=None):
    """(overall status, [status per frame of the last batch])."""
    out = (ctypes.c_int * max(1, n))()
    st = _st(lib().tsdf_batch_status(batch, _stream(stream), out, n))
    return st, [_st(out[i]) for i in range(n)]


def tsdf_server_create(mode, max_batch, max_inflight, max_frame_pixels, staging_frames,
                       use_graph=1, stream=None):
    h = _P()
    st = _st(lib().tsdf_server_create(mode, max_batch, max_inflight, max_frame_pixels,
                                      staging_frames, int(use_graph), _stream(stream),
                                      ctypes.byref(h)))
    if st != "OK":
        raise TsdfError(st, "tsdf_server_create")
    return h


def tsdf_server_destroy(server) -> None:
    lib().tsdf_server_destroy(server)


def tsdf_server_clock(server) -> float:
    return float(lib().tsdf_server_clock(server))


def tsdf_server_submit(server, request) -> str:
    return _st(lib().tsdf_server_submit(server, ctypes.byref(request)))


def tsdf_server_poll(server, out, capacity=None) -> int:
    return int(lib().tsdf_server_poll(server, out, len(out) if capacity is None else capacity))


def tsdf_server_pending(server) -> int:
    return int(lib().tsdf_server_pending(server))


def tsdf_server_replay(server, requests, n=None):
    """(status, completions array) for a ctypes array of tsdf_request."""
    n = len(requests) if n is None else n
    out = (tsdf_completion * max(1, n))()
    st = _st(lib().tsdf_server_replay(server, requests, n, out))
    return st, out


class Batch:
    """Owning wrapper around a tsdf_batch*."""

    def __init__(self, max_frames, **options):
        self.handle = tsdf_batch_create(max_frames)
        self.max_frames = max_frames
        for k, x in options.items():
            if tsdf_batch_set_option(self.handle, k, x) != "OK":
                raise ValueError(f"bad batch option {k}={x}")

    def close(self):
        if getattr(self, "handle", None):
            tsdf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value) -> str:
        return tsdf_batch_set_option(self.handle, option, value)

    def fuse_async(self, items, stream=None) -> str:
        """items: (Volume, depth tensor, rgb tensor or None, intr, pose) per frame."""
        frames = make_frames([(v.handle, d, c, i, p) for v, d, c, i, p in items])
        self._keep = (frames, items)   # buffers stay referenced until the next call
        return tsdf_fuse_batch_async(self.handle, frames, len(items), stream)

    def status(self, n, stream=None):
        return tsdf_batch_status(self.handle, n, stream)

    def autotune(self, items, reps=5, stream=None):
        """items as for fuse_async; their volumes must be empty and are left empty."""
        frames = make_frames([(v.handle, d, c, i, p) for v, d, c, i, p in items])
        self._keep = (frames, items)
        return tsdf_batch_autotune(self.handle, frames, len(items), reps, stream)


# ----------------------------------------------------------------------------
# convenience: an owning handle
# ----------------------------------------------------------------------------
class Volume:
    """Owning wrapper around a tsdf_volume*; every method is one C call."""

    def __init__(self, voxel_size, truncation, table_slots, pool_blocks, memory=None,
                 stream=None):
        self.voxel_size = float(voxel_size)
        self.truncation = float(truncation)
        self.table_slots = int(table_slots)
        self.pool_blocks = int(pool_blocks)
        self._memory = memory
        if memory is None:
            self.handle = tsdf_volume_create(voxel_size, truncation, table_slots, pool_blocks)
        else:
            nbytes = memory.numel() * memory.element_size()
            self.handle = tsdf_volume_create_in(memory, nbytes, voxel_size, truncation,
                                                table_slots, pool_blocks, stream)

    def close(self):
        if getattr(self, "handle", None):
            tsdf_volume_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fuse(self, depth, intr, pose, rgb=None, stream=None, sync=True) -> str:
        h, w = depth.shape[-2], depth.shape[-1]
        fn = tsdf_fuse_frame if sync else tsdf_fuse_frame_async
        return fn(self.handle, depth, w, h, intr, pose, rgb, stream)

    def fuse_host(self, depth, intr, pose, rgb=None, stream=None) -> str:
        h, w = depth.shape[-2], depth.shape[-1]
        return tsdf_fuse_frame_host(self.handle, depth, w, h, intr, pose, rgb, stream)

    def status(self, stream=None) -> str:
        return tsdf_volume_status(self.handle, stream)

    def reset(self, stream=None) -> str:
        return tsdf_volume_reset(self.handle, stream)

    def block_count(self, stream=None) -> int:
        return tsdf_volume_block_count(self.handle, stream)

    def export(self, stream=None, voxels=True):
        return tsdf_export_blocks(self.handle, stream, voxels)

    def set_option(self, option, value) -> str:
        return tsdf_volume_set_option(self.handle, option, value)

    def layout(self) -> tsdf_layout:
        return tsdf_volume_layout(self.handle)

    def autotune(self, depth, intr, pose, rgb=None, reps=5, stream=None):
        h, w = depth.shape[-2], depth.shape[-1]
        return tsdf_autotune_frame(self.handle, depth, w, h, intr, pose, rgb, reps, stream)

    def extract_mesh(self, stream=None, cells=True):
        return tsdf_extract_mesh(self.handle, stream, cells)

    def table_stats(self, stream=None) -> dict:
        return tsdf_volume_table_stats(self.handle, stream)

    def copy_from(self, other, stream=None) -> str:
        return tsdf_volume_copy(self.handle, other.handle, stream)

    def save(self, stream=None):
        return tsdf_volume_save(self.handle, stream)

    def load(self, checkpoint, stream=None) -> str:
        return tsdf_volume_load(self.handle, checkpoint, stream)
