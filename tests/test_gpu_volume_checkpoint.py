"""Checkpoint and resume (tsdf_volume_save / tsdf_volume_load) on the GPU.

A checkpoint holds the volume's whole device state, so a volume restored from
it and fed the next frame must equal the oracle fed every frame; the
checkpoint must refuse a volume of other sizes or settings, a short buffer and
a buffer that is not a checkpoint, and carry the poisoned state along.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2608_08287_gb300 import synth, tsdf
from test_gpu_parity import assert_same_volume, to_dev

pytestmark = pytest.mark.gpu

SPEC = synth.VolumeSpec(0.01, 0.04, 1 << 14, 1 << 14)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    oracle.build()
    torch.cuda.set_device(0)


def volume(spec=SPEC, **opts):
    v = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    for k, x in opts.items():
        assert v.set_option(k, x) == "OK"
    return v


def fuse(v, f):
    d, c = to_dev(f)
    return v.fuse(d, f.intr, f.pose, c)


FRAMES = [synth.room_frame(9 * k, width=160, height=120) for k in range(4)]


@pytest.mark.parametrize("slot_index", [0, 1])
def test_resume_equals_uninterrupted_fusion(slot_index):
    ov = oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SPEC.table_slots,
                             SPEC.pool_blocks)
    a = volume(slot_index=slot_index)
    for f in FRAMES[:2]:
        assert fuse(a, f) == ov.fuse_frame(f) == "OK"
    st, ck = a.save()
    assert st == "OK" and len(ck) == tsdf.tsdf_volume_checkpoint_bytes(a.handle)
    assert len(ck) == 64 + tsdf.tsdf_volume_bytes(SPEC.table_slots, SPEC.pool_blocks)
    b = volume(slot_index=slot_index)
    assert fuse(b, FRAMES[3]) == "OK"          # some other state, replaced by the load
    assert b.load(ck) == "OK"
    assert b.block_count() == a.block_count()
    assert_same_volume(b, ov)
    for f in FRAMES[2:]:
        assert ov.fuse_frame(f) == fuse(a, f) == fuse(b, f) == "OK"
    assert_same_volume(a, ov)
    assert_same_volume(b, ov)
    # the checkpoint is a copy: a later one of the moved-on source differs
    st2, ck2 = a.save()
    assert st2 == "OK" and not np.array_equal(ck, ck2)
    # a checkpoint of an empty volume empties a used one
    st, empty = volume(slot_index=slot_index).save()
    assert st == "OK" and b.load(empty) == "OK" and b.block_count() == 0
    ov2 = oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SPEC.table_slots,
                              SPEC.pool_blocks)
    assert fuse(b, FRAMES[1]) == ov2.fuse_frame(FRAMES[1]) == "OK"
    assert_same_volume(b, ov2)


def test_load_refuses_other_volumes_and_bad_buffers():
    a = volume()
    assert fuse(a, FRAMES[0]) == "OK"
    st, ck = a.save()
    assert st == "OK"
    n0 = a.block_count()
    others = [volume(synth.VolumeSpec(0.02, 0.04, SPEC.table_slots, SPEC.pool_blocks)),
              volume(synth.VolumeSpec(0.01, 0.05, SPEC.table_slots, SPEC.pool_blocks)),
              volume(synth.VolumeSpec(0.01, 0.04, SPEC.table_slots, SPEC.pool_blocks // 2)),
              volume(synth.VolumeSpec(0.01, 0.04, SPEC.table_slots * 2, SPEC.pool_blocks)),
              volume(slot_index=1)]
    for v in others:
        assert v.load(ck) == "INVALID_ARG"
        assert v.block_count() == 0                  # unchanged
    b = volume()
    assert b.load(ck[:-1]) == "INVALID_ARG"          # short
    assert b.load(ck[:63]) == "INVALID_ARG"          # not even a header
    bad = ck.copy()
    bad[0] ^= 0xFF                                   # not a checkpoint
    assert b.load(bad) == "INVALID_ARG"
    assert b.block_count() == 0
    assert b.load(ck) == "OK" and b.block_count() == n0
    # a save into too small a buffer is refused
    small = np.empty(16, np.uint8)
    assert tsdf._st(tsdf.lib().tsdf_volume_save(a.handle, small.ctypes.data, small.size,
                                                None)) == "INVALID_ARG"


def test_poisoned_state_travels_with_the_checkpoint():
    small = synth.VolumeSpec(0.01, 0.04, 1 << 12, 64)
    a = volume(small)
    assert fuse(a, FRAMES[0]) == "POOL_FULL"
    st, ck = a.save()
    assert st == "OK"
    b = volume(small)
    assert b.load(ck) == "OK"
    assert fuse(b, FRAMES[1]) == "POISONED"
    assert b.reset() == "OK"
    assert fuse(b, FRAMES[1]) in ("OK", "POOL_FULL")
