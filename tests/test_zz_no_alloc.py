"""tsdf_fuse_frame_host_noalloc: the host-buffer fuse call that allocates
nothing.

Some callers cannot let the library call cudaMalloc: a real-time capture loop
must not stall on an allocation (cudaMalloc can block and synchronise the
device), a process whose device memory is budgeted by its own allocator cannot
have a library take more behind its back, and a plugin host may forbid plugins
to own device memory. For them this entry point stages the host frame in one
fixed array compiled into the library instead of staging the volume allocates.

Checked here: two calls in a row give the oracle's volume (block-key set and
weights exact, means within the parity tolerance) and the same volume as
tsdf_fuse_frame_host; a frame without colour; that repeated calls take no
device memory; that frames above the limit are refused. This file is
collected last, so that a run stopping at the first failure has run every
other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2608_08287_gb300 import synth, tsdf
from voxels import sort_blocks

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the mean tolerance of the GPU parity tests
SPEC = synth.VolumeSpec(0.005, 0.02, 1 << 18, 1 << 16)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    oracle.build()
    torch.cuda.set_device(0)


def _volume(spec=SPEC):
    return tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)


def _oracle(spec=SPEC):
    return oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                               spec.pool_blocks)


def _same_as_oracle(gv, ov):
    gc, gx = sort_blocks(*gv.export())
    oc, ox = ov.export(double=True)
    assert np.array_equal(gc, oc), "block-key sets differ"
    assert np.array_equal(gx[:, 1], ox[:, 1].astype(np.float32)), "weights differ"
    if len(gc):
        assert float(np.max(np.abs(gx[:, [0, 2, 3, 4]] - ox[:, [0, 2, 3, 4]]))) <= TOL
    return len(gc)


def _same(a, b):
    ac, ax = sort_blocks(*a.export())
    bc, bx = sort_blocks(*b.export())
    assert np.array_equal(ac, bc), "block-key sets differ"
    assert np.array_equal(ax[:, 1], bx[:, 1]), "weights differ"
    if len(ac):
        assert float(np.max(np.abs(ax[:, [0, 2, 3, 4]] - bx[:, [0, 2, 3, 4]]))) <= TOL


def _host(f, colour=True):
    d = torch.from_numpy(f.depth).pin_memory()
    c = torch.from_numpy(f.rgb).pin_memory() if colour else None
    return d, c


def test_noalloc_matches_oracle_and_host_entry_point_on_two_calls():
    frames = [synth.room_frame(0), synth.room_frame(9)]
    a, b, ov = _volume(), _volume(), _oracle()
    blocks = []
    for f in frames:   # two calls in a row: the shared staging is reused
        d, c = _host(f)
        assert tsdf.tsdf_fuse_frame_host_noalloc(a.handle, d, f.width, f.height, f.intr,
                                                 f.pose, c) == "OK"
        assert tsdf.tsdf_fuse_frame_host(b.handle, d, f.width, f.height, f.intr, f.pose,
                                         c) == "OK"
        assert ov.fuse_frame(f) == "OK"
        blocks.append(_same_as_oracle(a, ov))
        _same(a, b)
    assert blocks[0] > 5000 and blocks[1] > blocks[0]


def test_noalloc_without_colour():
    frames = [synth.room_frame(3), synth.room_frame(12)]
    a, ov = _volume(), _oracle()
    for f in frames:
        d, _ = _host(f, colour=False)
        assert tsdf.tsdf_fuse_frame_host_noalloc(a.handle, d, f.width, f.height, f.intr,
                                                 f.pose, None) == "OK"
        assert ov.fuse_frame(f, with_rgb=False) == "OK"
        assert _same_as_oracle(a, ov) > 5000
    _, gx = a.export()
    assert not np.any(gx[:, 2:5]), "no colour was given, so every colour mean is zero"


def test_noalloc_takes_no_device_memory():
    f = synth.room_frame(5)
    d, c = _host(f)
    v = _volume()
    # the first call on the device looks up the staging array's address (and
    # may load the library's code); device memory is measured after it
    assert tsdf.tsdf_fuse_frame_host_noalloc(v.handle, d, f.width, f.height, f.intr, f.pose,
                                             c) == "OK"
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(10):
        assert tsdf.tsdf_fuse_frame_host_noalloc(v.handle, d, f.width, f.height, f.intr,
                                                 f.pose, c) == "OK"
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "the no-allocation call took device memory"
    # the measurement sees an allocation of this size: the volume-staged host
    # call on a fresh volume allocates its staging (2.15 MB for this frame)
    w = _volume()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert tsdf.tsdf_fuse_frame_host(w.handle, d, f.width, f.height, f.intr, f.pose,
                                     c) == "OK"
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1


def test_noalloc_rejects_frames_above_its_limit():
    spec = synth.VolumeSpec(0.01, 0.04, 1 << 10, 1 << 8)
    v = _volume(spec)
    w = 1025
    h = tsdf.NOALLOC_MAX_PIXELS // w + 1
    assert w * h > tsdf.NOALLOC_MAX_PIXELS
    depth = np.zeros((h, w), np.float32)
    st = tsdf.tsdf_fuse_frame_host_noalloc(v.handle, depth, w, h, (100, 100, 512, 512),
                                           np.eye(4, dtype=np.float32))
    assert st == "INVALID_ARG"
    assert v.block_count() == 0


def test_noalloc_refuses_bad_frames_before_copying():
    v = _volume()
    f = synth.room_frame(0)
    d, c = _host(f)
    bad = np.array(f.intr, dtype=np.float32).copy()
    bad[0] = 0.0   # fx = 0: refused by the frame check, nothing is enqueued
    assert tsdf.tsdf_fuse_frame_host_noalloc(v.handle, d, f.width, f.height, bad, f.pose,
                                             c) == "INVALID_ARG"
    assert v.block_count() == 0
    # the array is still usable afterwards
    assert tsdf.tsdf_fuse_frame_host_noalloc(v.handle, d, f.width, f.height, f.intr, f.pose,
                                             c) == "OK"
    assert v.block_count() > 5000
