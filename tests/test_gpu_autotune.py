"""The autotuners (tsdf_autotune_frame, tsdf_batch_autotune) on the GPU.

A tuner may pick any configuration -- every strategy computes the same
volume -- so the checks are that it leaves the data alone (a volume tuned on
a scratch copy keeps its bytes; a batch's volumes are left empty), that the
configuration it reports is a valid one and is applied, and that fusing with
it still matches the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2608_08287_gb300 import synth, tsdf
from test_gpu_parity import assert_same_volume, to_dev

pytestmark = pytest.mark.gpu

SPEC = synth.VolumeSpec(0.01, 0.04, 1 << 16, 1 << 15)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    oracle.build()
    torch.cuda.set_device(0)


def frame(k, w=160, h=120):
    return synth.room_frame(6 * k, width=w, height=h)


def check_tuning(t, batch):
    assert t["allocate_mode"] in ((1, 2) if batch else (0, 1, 2))
    assert t["integrate_mode"] in ((0, 1) if batch else (0, 1, 2)) and t["fuse_mode"] in (0, 1, 2)
    assert t["probe_load"] in (0, 1, 2)
    if batch:
        assert 0 <= t["ctas_per_sm"] <= 4 and t["use_graph"] in (0, 1)
        assert t["threads_per_point"] == 1
        assert t["batch_streams"] in (0, 4, 8, 16)
    else:
        assert t["threads_per_point"] in (0, 1, 2, 4, 8)
        assert t["threads_per_point"] <= 1 or (t["fuse_mode"] == 2 and t["probe_load"] == 0)
    assert 0 < t["best_ms"] <= t["default_ms"]
    assert t["candidates"] >= (10 if batch else 17)


def test_autotune_frame_keeps_the_volume_and_applies_the_choice():
    gv = tsdf.Volume(SPEC.voxel_size, SPEC.truncation, SPEC.table_slots, SPEC.pool_blocks)
    ov = oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SPEC.table_slots,
                             SPEC.pool_blocks)
    f0, f1 = frame(0), frame(1)
    d0, c0 = to_dev(f0)
    assert gv.fuse(d0, f0.intr, f0.pose, c0) == ov.fuse_frame(f0) == "OK"
    before = gv.export()
    d1, c1 = to_dev(f1)
    st, t = gv.autotune(d1, f1.intr, f1.pose, c1, reps=3)
    assert st == "OK", st
    check_tuning(t, batch=False)
    after = gv.export()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert gv.fuse(d1, f1.intr, f1.pose, c1) == ov.fuse_frame(f1) == "OK"
    assert_same_volume(gv, ov)


def test_autotune_frame_reports_overflow_and_leaves_volume_usable():
    tiny = synth.VolumeSpec(0.01, 0.04, 1 << 12, 64)
    gv = tsdf.Volume(tiny.voxel_size, tiny.truncation, tiny.table_slots, tiny.pool_blocks)
    f = frame(0)
    d, c = to_dev(f)
    st, t = gv.autotune(d, f.intr, f.pose, c, reps=1)
    assert st == "POOL_FULL" and t is None
    assert gv.status() == "OK" and gv.block_count() == 0   # only the scratch overflowed


def _sessions(n):
    res = [(160, 120), (320, 240), (160, 120), (320, 240), (640, 480), (160, 120)][:n]
    vols, ovs, items = [], [], []
    for i, (w, h) in enumerate(res):
        spec = synth.VolumeSpec(0.01, 0.04, 1 << 17, 1 << 16)
        vols.append(tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots,
                                spec.pool_blocks))
        ovs.append(oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                                       spec.pool_blocks))
        f = frame(3 * i, w, h)
        d, c = to_dev(f)
        items.append((vols[-1], d, c, f.intr, f.pose, f))
    return vols, ovs, items


def test_batch_autotune_leaves_volumes_empty_and_result_matches_oracle():
    vols, ovs, items = _sessions(6)
    batch = tsdf.Batch(8, use_graph=1)
    st, t = batch.autotune([x[:5] for x in items], reps=2)
    assert st == "OK", st
    check_tuning(t, batch=True)
    assert all(v.block_count() == 0 for v in vols)
    assert batch.fuse_async([x[:5] for x in items]) == "OK"
    assert batch.status(len(items))[0] == "OK"
    for (v, _, _, _, _, f), ov in zip(items, ovs):
        assert ov.fuse_frame(f) == "OK"
        assert_same_volume(v, ov)


def test_batch_autotune_needs_empty_volumes():
    vols, ovs, items = _sessions(2)
    v, d, c, intr, pose, _ = items[0]
    assert v.fuse(d, intr, pose, c) == "OK"
    batch = tsdf.Batch(4)
    st, t = batch.autotune([x[:5] for x in items], reps=1)
    assert st == "INVALID_ARG" and t is None
    assert v.reset() == "OK"
    st, t = batch.autotune([x[:5] for x in items], reps=1)
    assert st == "OK"
