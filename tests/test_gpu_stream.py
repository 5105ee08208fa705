"""tsdf_fuse_frames_host: frames in host memory fused in order, each frame's
copy overlapping the fusion of the one before it. Every result is compared
with the oracle fed the same frames: block-key set and weights exact, means
within 1e-5 (the sums of Section 2.2 accumulate in a different order).
Statuses follow the single-frame calls: an overflow reports its error and
poisons the volume, later frames of that volume report POISONED."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2608_08287_gb300 import synth, tsdf
from voxels import sort_blocks

pytestmark = pytest.mark.gpu
TOL = 1e-5
SPEC = synth.VolumeSpec(0.01, 0.04, 1 << 18, 1 << 16)   # the 320x240 session class


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    oracle.build()
    torch.cuda.set_device(0)


def _vol(spec=SPEC):
    return tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)


def _oracle(spec=SPEC):
    return oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                               spec.pool_blocks)


def _frames(ids, w=320, h=240):
    return [synth.room_frame(i, width=w, height=h) for i in ids]


def _pinned(f, colour=True):
    d = torch.from_numpy(f.depth).pin_memory()
    c = torch.from_numpy(f.rgb).pin_memory() if colour else None
    return d, c


def _same_as_oracle(gv, ov):
    gc, gx = sort_blocks(*gv.export())
    oc, ox = ov.export(double=True)
    assert np.array_equal(gc, oc), "block-key sets differ"
    assert np.array_equal(gx[:, 1], ox[:, 1].astype(np.float32)), "weights differ"
    if len(gc):
        assert float(np.max(np.abs(gx[:, [0, 2, 3, 4]] - ox[:, [0, 2, 3, 4]]))) <= TOL
    return len(gc)


def test_stream_into_one_volume_equals_oracle():
    frames = _frames(range(0, 60, 10))
    v, ov = _vol(), _oracle()
    bufs = [_pinned(f) for f in frames]
    arr = tsdf.make_host_frames([(v.handle, d, c, f.intr, f.pose)
                                 for f, (d, c) in zip(frames, bufs)])
    st, per = tsdf.tsdf_fuse_frames_host(arr)
    assert st == "OK" and per == ["OK"] * len(frames)
    for f in frames:
        assert ov.fuse_frame(f) == "OK"
    assert _same_as_oracle(v, ov) > 1000


def test_stream_each_frame_into_its_own_volume_and_repeat_calls():
    frames = _frames([3, 17, 31, 45])
    vols = [_vol() for _ in frames]
    bufs = [_pinned(f, colour=(i != 2)) for i, f in enumerate(frames)]
    items = [(v.handle, d, c, f.intr, f.pose) for v, f, (d, c) in zip(vols, frames, bufs)]
    for rep in range(2):      # the second call reuses the staging and streams
        st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(items))
        assert st == "OK" and per == ["OK"] * 4
    for i, (v, f) in enumerate(zip(vols, frames)):
        ov = _oracle()
        for _ in range(2):
            assert ov.fuse_frame(f, with_rgb=(i != 2)) == "OK"
        assert _same_as_oracle(v, ov) > 500


def test_stream_grows_its_staging_and_takes_pageable_buffers():
    small = _frames([5], 160, 120)[0]
    big = synth.room_frame(7)                         # 640x480 after 160x120
    spec_small = synth.VolumeSpec(0.02, 0.08, 1 << 16, 1 << 14)
    a, b = _vol(spec_small), _vol(synth.VolumeSpec(0.005, 0.02, 1 << 20, 1 << 18))
    st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(
        [(a.handle, small.depth, small.rgb, small.intr, small.pose)]))
    assert st == "OK"
    # the owner of the staging is frames[0].volume: a takes the larger frame too
    st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(
        [(a.handle, small.depth, small.rgb, small.intr, small.pose),
         (b.handle, big.depth, big.rgb, big.intr, big.pose)]))
    assert st == "OK" and per == ["OK", "OK"]
    oa, ob = _oracle(spec_small), _oracle(synth.VolumeSpec(0.005, 0.02, 1 << 20, 1 << 18))
    assert oa.fuse_frame(small) == "OK" and oa.fuse_frame(small) == "OK"
    assert ob.fuse_frame(big) == "OK"
    assert _same_as_oracle(a, oa) > 100
    assert _same_as_oracle(b, ob) > 5000


def test_stream_overflow_poisons_only_its_volume():
    frames = _frames([0, 20, 40])
    tiny = synth.VolumeSpec(0.01, 0.04, 1 << 12, 600)      # fewer blocks than one frame has
    bad, good = _vol(tiny), _vol()
    bufs = [_pinned(f) for f in frames]
    items = []
    for f, (d, c) in zip(frames, bufs):
        items.append((bad.handle, d, c, f.intr, f.pose))
        items.append((good.handle, d, c, f.intr, f.pose))
    st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(items))
    assert st == "POOL_FULL"
    assert per[0] == "POOL_FULL" and per[2] == per[4] == "POISONED"
    assert per[1] == per[3] == per[5] == "OK"
    assert bad.block_count() == tiny.pool_blocks          # min(claimed, pool)
    ov = _oracle()
    for f in frames:
        assert ov.fuse_frame(f) == "OK"
    assert _same_as_oracle(good, ov) > 1000
    # the poisoned volume refuses further frames until reset
    st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames([items[0]]))
    assert st == "POISONED" and per == ["POISONED"]
    assert bad.reset() == "OK"
    st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames([items[0]]))
    assert st == "POOL_FULL"


def test_stream_refuses_an_invalid_frame_before_enqueueing():
    frames = _frames([0, 10, 20])
    v = _vol()
    bufs = [_pinned(f) for f in frames]
    items = [(v.handle, d, c, f.intr, f.pose) for f, (d, c) in zip(frames, bufs)]
    bad_intr = np.array(frames[1].intr, dtype=np.float32).copy()
    bad_intr[1] = np.nan
    items[1] = (v.handle, bufs[1][0], bufs[1][1], bad_intr, frames[1].pose)
    st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(items))
    assert st == "INVALID_ARG"
    assert v.block_count() == 0                            # nothing was fused
    assert tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(items[:1]))[0] == "OK"
    assert v.block_count() > 1000


def test_l2_fetch_granularity_changes_no_result():
    """tsdf_set_l2_fetch_bytes (a context-wide cache hint): the volume with a
    32-byte fetch equals the oracle, the previous value comes back, and values
    other than 0, 32, 64, 128 are refused."""
    f = _frames([7])[0]
    st, before = tsdf.tsdf_set_l2_fetch_bytes(32)
    assert st == "OK"
    try:
        v, ov = _vol(), _oracle()
        d, c = _pinned(f)
        st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(
            [(v.handle, d, c, f.intr, f.pose)]))
        assert st == "OK"
        assert ov.fuse_frame(f) == "OK"
        assert _same_as_oracle(v, ov) > 500
        assert tsdf.tsdf_set_l2_fetch_bytes(48)[0] == "INVALID_ARG"
    finally:
        st, cur = tsdf.tsdf_set_l2_fetch_bytes(before)
    assert st == "OK" and cur == 32


def test_stream_over_many_volumes_reads_every_status():
    """More distinct volumes than one gather of status words holds (256): the
    error words of the last frame of every volume are gathered in chunks. One
    volume overflows; every other frame reports OK and equals the oracle."""
    f = _frames([11], 160, 120)[0]
    spec = synth.VolumeSpec(0.02, 0.08, 1 << 12, 1 << 11)
    tiny = synth.VolumeSpec(0.02, 0.08, 1 << 12, 8)
    n = 300
    vols = [_vol(tiny if i == 271 else spec) for i in range(n)]
    d, c = _pinned(f)
    items = [(v.handle, d, c, f.intr, f.pose) for v in vols]
    st, per = tsdf.tsdf_fuse_frames_host(tsdf.make_host_frames(items))
    assert st == "POOL_FULL"
    assert per[271] == "POOL_FULL"
    assert all(p == "OK" for i, p in enumerate(per) if i != 271)
    ov = _oracle(spec)
    assert ov.fuse_frame(f) == "OK"
    nb = ov.block_count()
    assert all(v.block_count() == nb for i, v in enumerate(vols) if i != 271)
    assert _same_as_oracle(vols[299], ov) == nb
    assert vols[271].block_count() == tiny.pool_blocks
