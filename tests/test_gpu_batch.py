"""Batched fusion (many sessions, one frame each per call) against the
single-frame path and the CPU oracle: each session's result must be the same
alone and in the mix (block-key set and weights exact, means within 1e-5).
Both launch forms are covered: one launch per frame over the batch's streams
(TSDF_OPT_BATCH_STREAMS k > 0, the default) and one persistent launch for the
whole batch (0), with and without graphs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2608_08287_gb300 import synth, tsdf
from voxels import sort_blocks

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    oracle.build()
    torch.cuda.set_device(0)


def sessions(n, seed=7):
    """Mixed resolutions (160x120 / 320x240 / 640x480 scaled cameras), each a
    different view of the room, each with its own volume size."""
    out = []
    res = [(160, 120, 1 << 16), (320, 240, 1 << 17), (640, 480, 1 << 18)]
    u = synth.uniform(seed, 3, n)
    for i in range(n):
        w, h, slots = res[int(u[i] * 3) % 3]
        out.append(dict(w=w, h=h, spec=synth.VolumeSpec(0.005, 0.02, slots, slots // 2),
                        frame0=(i * 23) % 300))
    return out


def frame_of(s, k):
    return synth.room_frame((s["frame0"] + 5 * k) % 300, width=s["w"], height=s["h"])


def new_volume(spec):
    return tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)


def dev(frame):
    return (torch.from_numpy(frame.depth).cuda(), torch.from_numpy(frame.rgb).cuda())


def same(a, b):
    ac, ax = sort_blocks(*a.export())
    bc, bx = sort_blocks(*b.export())
    assert np.array_equal(ac, bc), "block-key sets differ"
    assert np.array_equal(ax[:, 1], bx[:, 1]), "weights differ"
    if len(ac):
        assert float(np.max(np.abs(ax[:, [0, 2, 3, 4]] - bx[:, [0, 2, 3, 4]]))) <= TOL
    return len(ac)


def run_batched(ss, rounds, **opts):
    vols = [new_volume(s["spec"]) for s in ss]
    batch = tsdf.Batch(len(ss), **opts)
    for k in range(rounds):
        items = []
        for s, v in zip(ss, vols):
            f = frame_of(s, k)
            d, c = dev(f)
            items.append((v, d, c, f.intr, f.pose))
        assert batch.fuse_async(items) == "OK"
        st, per = batch.status(len(ss))
        assert st == "OK" and all(p == "OK" for p in per)
    return vols


def run_single(ss, rounds):
    vols = [new_volume(s["spec"]) for s in ss]
    for k in range(rounds):
        for s, v in zip(ss, vols):
            f = frame_of(s, k)
            d, c = dev(f)
            assert v.fuse(d, f.intr, f.pose, c) == "OK"
    return vols


PERSISTENT = dict(batch_streams=0)


@pytest.mark.parametrize("opts", [
    # one persistent launch for the whole batch
    dict(PERSISTENT), dict(PERSISTENT, fuse_mode=0), dict(PERSISTENT, fuse_mode=0, allocate_mode=2),
    dict(PERSISTENT, fuse_mode=0, integrate_mode=1), dict(PERSISTENT, fuse_mode=1),
    dict(PERSISTENT, use_graph=1), dict(PERSISTENT, use_graph=1, fuse_mode=0),
    dict(PERSISTENT, use_graph=1, fuse_mode=1, ctas_per_sm=2),
    # one launch per frame over the batch's streams
    dict(), dict(batch_streams=1), dict(batch_streams=3, fuse_mode=0),
    dict(batch_streams=16, fuse_mode=1),
    dict(batch_streams=5, fuse_mode=0, allocate_mode=2, integrate_mode=1),
    dict(batch_streams=2, probe_load=1)])
def test_batch_equals_single_frame_path(opts):
    ss = sessions(9)
    b = run_batched(ss, 2, **opts)
    a = run_single(ss, 2)
    total = sum(same(x, y) for x, y in zip(a, b))
    assert total > 1000


@pytest.mark.parametrize("streams", [0, 8])
def test_batch_equals_oracle(streams):
    ss = sessions(5, seed=11)
    vols = run_batched(ss, 2, use_graph=1, batch_streams=streams)
    for s, v in zip(ss, vols):
        ov = oracle.OracleVolume(s["spec"].voxel_size, s["spec"].truncation,
                                 s["spec"].table_slots, s["spec"].pool_blocks)
        for k in range(2):
            assert ov.fuse_frame(frame_of(s, k)) == "OK"
        gc, gx = sort_blocks(*v.export())
        oc, ox = ov.export(double=True)
        assert np.array_equal(gc, oc)
        assert np.array_equal(gx[:, 1], ox[:, 1].astype(np.float32))
        assert float(np.max(np.abs(gx[:, [0, 2, 3, 4]] - ox[:, [0, 2, 3, 4]]))) <= TOL


@pytest.mark.parametrize("streams", [0, 4])
def test_batches_of_changing_composition(streams):
    """Graph replays (persistent launch) or lanes (per-frame launches) over
    batches whose frames, sizes and count change from call to call."""
    ss = sessions(12, seed=5)
    vols = [new_volume(s["spec"]) for s in ss]
    ref = [new_volume(s["spec"]) for s in ss]
    batch = tsdf.Batch(12, use_graph=1, batch_streams=streams)
    rng = np.random.default_rng(3)
    rounds = [0] * len(ss)
    for _ in range(5):
        pick = sorted(rng.choice(len(ss), size=int(rng.integers(1, len(ss) + 1)), replace=False))
        items = []
        for i in pick:
            f = frame_of(ss[i], rounds[i])
            d, c = dev(f)
            items.append((vols[i], d, c, f.intr, f.pose))
            assert ref[i].fuse(d, f.intr, f.pose, c) == "OK"
            rounds[i] += 1
        assert batch.fuse_async(items) == "OK"
        assert batch.status(len(pick))[0] == "OK"
    for a, b in zip(ref, vols):
        same(a, b)


@pytest.mark.parametrize("streams", [0, 8])
def test_batch_reports_overflow_per_frame(streams):
    ss = sessions(4, seed=9)
    vols = [new_volume(s["spec"]) for s in ss]
    tiny = tsdf.Volume(0.005, 0.02, 1 << 10, 8)
    vols[2] = tiny
    batch = tsdf.Batch(4, batch_streams=streams)
    items = []
    for s, v in zip(ss, vols):
        f = frame_of(s, 0)
        d, c = dev(f)
        items.append((v, d, c, f.intr, f.pose))
    assert batch.fuse_async(items) == "OK"
    st, per = batch.status(4)
    assert st == "POOL_FULL"
    assert per[2] == "POOL_FULL" and per[0] == per[1] == per[3] == "OK"
    assert batch.fuse_async(items) == "POISONED"     # the poisoned volume rejects the call
    assert tiny.reset() == "OK"


def test_batch_rejects_bad_arguments():
    s = sessions(1)[0]
    v = new_volume(s["spec"])
    f = frame_of(s, 0)
    d, c = dev(f)
    batch = tsdf.Batch(2)
    assert batch.fuse_async([(v, d, c, f.intr, f.pose), (v, d, c, f.intr, f.pose)]) == \
        "INVALID_ARG"                                 # one frame per volume
    frames = tsdf.make_frames([(v.handle, d, c, f.intr, f.pose)] * 3)
    assert tsdf.tsdf_fuse_batch_async(batch.handle, frames, 3) == "INVALID_ARG"   # > max
    assert batch.set_option("allocate_mode", 0) == "INVALID_ARG"
    assert batch.set_option("batch_streams", -1) == "INVALID_ARG"
    assert batch.set_option("batch_streams", 17) == "INVALID_ARG"
    assert batch.set_option("batch_streams", 16) == "OK"


@pytest.mark.parametrize("use_graph,streams", [(0, 0), (1, 0), (0, 8)])
def test_batch_stages_one_at_a_time_equal_both(use_graph, streams):
    """TSDF_OPT_BATCH_STAGES: stage A of every frame in one call, then stage B
    of the same frames in another, equals the oracle (as both stages in one
    call do)."""
    ss = sessions(6, seed=13)
    vols = [new_volume(s["spec"]) for s in ss]
    ba = tsdf.Batch(len(ss), fuse_mode=0, batch_stages=1, use_graph=use_graph,
                    batch_streams=streams)
    bb = tsdf.Batch(len(ss), fuse_mode=0, batch_stages=2, use_graph=use_graph,
                    batch_streams=streams)
    for k in range(2):
        items = []
        for s, v in zip(ss, vols):
            f = frame_of(s, k)
            d, c = dev(f)
            items.append((v, d, c, f.intr, f.pose))
        assert ba.fuse_async(items) == "OK"
        assert bb.fuse_async(items) == "OK"
        st, per = bb.status(len(ss))
        assert st == "OK" and all(p == "OK" for p in per)
    for s, v in zip(ss, vols):
        ov = oracle.OracleVolume(s["spec"].voxel_size, s["spec"].truncation,
                                 s["spec"].table_slots, s["spec"].pool_blocks)
        for k in range(2):
            assert ov.fuse_frame(frame_of(s, k)) == "OK"
        gc, gx = sort_blocks(*v.export())
        oc, ox = ov.export(double=True)
        assert np.array_equal(gc, oc)
        assert np.array_equal(gx[:, 1], ox[:, 1].astype(np.float32))
        assert float(np.max(np.abs(gx[:, [0, 2, 3, 4]] - ox[:, [0, 2, 3, 4]]))) <= TOL
    assert ba.set_option("batch_stages", 0) == "INVALID_ARG"
    assert ba.set_option("batch_stages", 4) == "INVALID_ARG"
