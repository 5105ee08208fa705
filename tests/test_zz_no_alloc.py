"""tsdf_fuse_frame_host_noalloc against tsdf_fuse_frame_host.

The no-allocation entry point is for callers that cannot let the library call
cudaMalloc (a real-time loop that must not stall on an allocation, a process
whose device memory is fully budgeted by its own allocator, a plugin host that
forbids plugins to own device memory). It stages host frames in one fixed
array compiled into the library instead of volume-owned staging. This file is
collected last so that a run stopping at the first failure has run every other
test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2608_08287_gb300 import synth, tsdf
from voxels import sort_blocks

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the mean tolerance of the GPU parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    torch.cuda.set_device(0)


def _same(a, b):
    ac, ax = sort_blocks(*a.export())
    bc, bx = sort_blocks(*b.export())
    assert np.array_equal(ac, bc), "block-key sets differ"
    assert np.array_equal(ax[:, 1], bx[:, 1]), "weights differ"
    if len(ac):
        assert float(np.max(np.abs(ax[:, [0, 2, 3, 4]] - bx[:, [0, 2, 3, 4]]))) <= TOL
    return len(ac)


def test_noalloc_matches_host_entry_point_on_two_calls():
    spec = synth.VolumeSpec(0.005, 0.02, 1 << 18, 1 << 16)
    frames = [synth.room_frame(0), synth.room_frame(9)]
    a = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    b = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    blocks = []
    for f in frames:   # two calls in a row: the shared staging is reused
        d = torch.from_numpy(f.depth).pin_memory()
        c = torch.from_numpy(f.rgb).pin_memory()
        assert tsdf.tsdf_fuse_frame_host_noalloc(a.handle, d, f.width, f.height, f.intr,
                                                 f.pose, c) == "OK"
        assert tsdf.tsdf_fuse_frame_host(b.handle, d, f.width, f.height, f.intr, f.pose,
                                         c) == "OK"
        blocks.append(_same(a, b))
    assert blocks[0] > 5000 and blocks[1] > blocks[0]


def test_noalloc_rejects_frames_above_its_limit():
    spec = synth.VolumeSpec(0.01, 0.04, 1 << 10, 1 << 8)
    v = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    w = 1025
    h = tsdf.NOALLOC_MAX_PIXELS // w + 1
    assert w * h > tsdf.NOALLOC_MAX_PIXELS
    depth = np.zeros((h, w), np.float32)
    st = tsdf.tsdf_fuse_frame_host_noalloc(v.handle, depth, w, h, (100, 100, 512, 512),
                                           np.eye(4, dtype=np.float32))
    assert st == "INVALID_ARG"
    assert v.block_count() == 0
