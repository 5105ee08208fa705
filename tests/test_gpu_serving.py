"""The serving loop: every session's volume, fused through continuous batching
(frames of many sessions mixed in each launch), equals fusing that session's
frames alone, in order, through the single-frame path (block-key set and
weights exact, means within 1e-5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2608_08287_gb300 import serving, tsdf
from voxels import sort_blocks

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def bank():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    torch.cuda.set_device(0)
    return serving.FrameBank(torch, n_frames=4, step=40)


def alone(plan, bank):
    spec = serving.SESSION_CLASSES[plan.res]
    v = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    for k in range(len(plan.arrivals)):
        depth_h, rgb_h, intr, pose, _ = bank.get(plan.res, plan.frame0 + k)
        assert v.fuse(depth_h.cuda(), intr, pose, rgb_h.cuda()) == "OK"
    return v


def same(a, b):
    ac, ax = sort_blocks(*a.export())
    bc, bx = sort_blocks(*b.export())
    assert np.array_equal(ac, bc), "block-key sets differ"
    assert np.array_equal(ax[:, 1], bx[:, 1]), "weights differ"
    if len(ac):
        assert float(np.max(np.abs(ax[:, [0, 2, 3, 4]] - bx[:, [0, 2, 3, 4]]))) <= TOL
    return len(ac)


@pytest.mark.parametrize("kind", ["batched", "batched_graph", "per_frame"])
def test_each_session_same_alone_and_in_the_mix(bank, kind):
    plans = serving.plan_sessions(10, window=0.6, min_dur=0.2, max_dur=0.5, seed=99)
    if kind == "per_frame":
        srv = serving.PerFrameServer(torch, bank, plans, reuse_volumes=False)
    else:
        srv = serving.BatchedServer(torch, bank, plans, max_batch=16,
                                    use_graph=(kind == "batched_graph"), reuse_volumes=False)
    res, st = srv.run()
    assert st == "OK"
    assert res.frames == sum(len(p.arrivals) for p in plans) > 20
    assert len(res.latencies_ms) == res.frames and np.all(res.latencies_ms > 0)
    for p in srv.plans:
        same(srv.finished[p.sid], alone(p, bank))
    srv.close()


def test_volume_reuse_between_sessions(bank):
    """Sessions that share a pooled volume one after the other start empty."""
    plans = serving.plan_sessions(8, window=0.8, min_dur=0.1, max_dur=0.25, seed=5,
                                  budget_bytes=2 * serving.volume_bytes((640, 480)))
    srv = serving.BatchedServer(torch, bank, plans, max_batch=8)
    res, st = srv.run()
    assert st == "OK" and res.frames == sum(len(p.arrivals) for p in plans)
    srv.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_native_server_same_alone_and_in_the_mix(bank, mode):
    """tsdf_server (C++ continuous batching, mode 0; per-frame baseline, mode 1)."""
    plans = serving.plan_sessions(12, window=0.6, min_dur=0.2, max_dur=0.5, seed=77)
    res, st, vols = serving.native_replay(torch, bank, plans, mode, max_batch=16,
                                          reuse_volumes=False, keep_volumes=True)
    assert st == "OK"
    assert res.frames == sum(len(p.arrivals) for p in plans) > 20
    assert np.all(res.latencies_ms > 0)
    for p in plans:
        if len(p.arrivals):
            assert vols[p.sid].status() == "OK"
            same(vols[p.sid], alone(p, bank))


def test_native_server_reused_volumes_start_empty(bank):
    """Sessions that share a pooled volume one after another: the last session
    on each volume equals that session fused alone (the volume was reset)."""
    plans = serving.plan_sessions(16, window=1.0, min_dur=0.1, max_dur=0.3, seed=31)
    where, counts = serving.assign_volumes(plans)
    assert sum(counts.values()) < len([p for p in plans if len(p.arrivals)])  # reuse happens
    res, st, vols = serving.native_replay(torch, bank, plans, 0, max_batch=8,
                                          keep_volumes=True)
    assert st == "OK"
    last = {}
    for p in sorted([p for p in plans if len(p.arrivals)], key=lambda p: p.arrivals[0]):
        last[where[p.sid]] = p
    for key, p in last.items():
        same(vols[p.sid], alone(p, bank))
