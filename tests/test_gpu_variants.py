"""The paper's variants of the data structure, on the GPU, against the oracle.

* Slot-derived block index (Section 6, "Deriving the location from the slot"):
  the pool index of a block is its table slot, the pool is sized to the table.
  The result is the same volume (C-13: which pool index a block gets is free),
  so it must match the oracle exactly as the counter-indexed volume does, for
  every strategy, up to a load factor of 0.92, and overflow must be reported.
* The bounded probe (Section 7: a probe loop with a compile-time trip count,
  MAX_PROBE = 8 in the printed Triton probe): a NEGATIVE control. At a high
  load factor it must lose blocks or contributions while every status stays
  OK -- the silent loss the paper measures -- and the unbounded probe on the
  same frames must not.
* The table diagnostics (occupancy, probe lengths, total weight) against
  values recomputed on the host from the table's own bytes, and volume copy.

Frames: the room orbit at 160x120 (intrinsics scaled from 640x480), every
sixth frame, voxel 1 cm, truncation 4 cm; 42 frames put 30,180 blocks into a
2^15-slot table (load 0.92); the 48th frame overflows it. At that load the
multiply-xor hash of these spatially coherent blocks leaves long clusters:
linear probing then averages ~300 probes per key, thousands at the worst.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2608_08287_gb300 import synth, tsdf
from test_gpu_parity import MODES, assert_same_volume, to_dev

pytestmark = pytest.mark.gpu

SLOTS = 1 << 15
SPEC = synth.VolumeSpec(0.01, 0.04, SLOTS, SLOTS)
N_HIGH = 42            # frames to load 0.92
N_OVER = 50            # enough frames to overflow 2^15 slots


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    oracle.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def orbit():
    """(frames, oracle statuses, oracle block counts, oracle volume after N_HIGH)."""
    frames = [synth.room_frame(6 * k, width=160, height=120) for k in range(N_OVER)]
    ov = oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SPEC.table_slots,
                             SPEC.pool_blocks)
    statuses, counts = [], []
    snapshot = None
    for k, f in enumerate(frames):
        statuses.append(ov.fuse_frame(f))
        counts.append(ov.block_count())
        if k == N_HIGH - 1:
            snapshot = ov.export(double=True)
    return frames, statuses, counts, snapshot


def volume(spec=SPEC, **opts):
    v = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    for k, x in opts.items():
        assert v.set_option(k, x) == "OK", (k, x)
    return v


def assert_matches_export(gv, ref):
    from voxels import sort_blocks
    oc, ox = ref
    gc, gx = sort_blocks(*gv.export())
    assert np.array_equal(gc, oc), "block-key sets differ"
    assert np.array_equal(gx[:, 1], ox[:, 1].astype(np.float32)), "weights differ"
    assert float(np.max(np.abs(gx[:, 0] - ox[:, 0]))) <= 1e-5
    assert float(np.max(np.abs(gx[:, 2:] - ox[:, 2:]))) <= 1e-5
    return len(gc)


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_slot_index_orbit_to_load_092(orbit, mode):
    frames, statuses, counts, ref = orbit
    gv = volume(slot_index=1, **MODES[mode])
    for k in range(N_HIGH):
        d, c = to_dev(frames[k])
        st = gv.fuse(d, frames[k].intr, frames[k].pose, c)
        assert st == statuses[k] == "OK", (k, st)
        assert gv.block_count() == counts[k], k
    n = assert_matches_export(gv, ref)
    assert n / SLOTS > 0.9
    stats = gv.table_stats()
    assert stats["occupied_slots"] == stats["blocks"] == n
    assert stats["weight_sum"] == int(ref[1][:, 1].sum())


def test_slot_index_overflow_and_reset(orbit):
    frames, statuses, counts, _ = orbit
    first_bad = next(k for k, s in enumerate(statuses) if s != "OK")
    assert statuses[first_bad] == "TABLE_FULL"   # the pool is the table
    gv = volume(slot_index=1)
    for k in range(first_bad + 1):
        d, c = to_dev(frames[k])
        st = gv.fuse(d, frames[k].intr, frames[k].pose, c)
        assert st == statuses[k], (k, st, statuses[k])
    d, c = to_dev(frames[0])
    assert gv.fuse(d, frames[0].intr, frames[0].pose, c) == "POISONED"
    # a reset zeroes the blocks scattered over the slot-indexed pool
    assert gv.reset() == "OK"
    ov = oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SLOTS, SLOTS)
    for k in (3, 4):
        d, c = to_dev(frames[k])
        assert gv.fuse(d, frames[k].intr, frames[k].pose, c) == ov.fuse_frame(frames[k]) == "OK"
    assert_same_volume(gv, ov)


def test_slot_index_option_rules(orbit):
    frames = orbit[0]
    v = volume(synth.VolumeSpec(0.01, 0.04, SLOTS, SLOTS // 2))
    assert v.set_option("slot_index", 1) == "INVALID_ARG"   # pool must equal the table
    v = volume()
    d, c = to_dev(frames[0])
    assert v.fuse(d, frames[0].intr, frames[0].pose, c) == "OK"
    assert v.set_option("slot_index", 1) == "INVALID_ARG"   # blocks already stored
    assert v.set_option("slot_index", 0) == "OK"            # no change is fine
    assert v.reset() == "OK"
    assert v.set_option("slot_index", 1) == "OK"
    assert v.set_option("slot_index", 2) == "INVALID_ARG"


def test_slot_index_batched(orbit):
    """Slot-indexed volumes through the batched kernels."""
    frames = orbit[0]
    vols = [volume(slot_index=1) for _ in range(3)]
    ovs = [oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SLOTS, SLOTS) for _ in vols]
    batch = tsdf.Batch(8)
    for step in range(2):
        items = []
        for i, (gv, ov) in enumerate(zip(vols, ovs)):
            f = frames[7 * i + step]
            d, c = to_dev(f)
            items.append((gv, d, c, f.intr, f.pose))
            assert ov.fuse_frame(f) == "OK"
        assert batch.fuse_async(items) == "OK"
        assert batch.status(len(items))[0] == "OK"
    for gv, ov in zip(vols, ovs):
        assert_same_volume(gv, ov)


def test_bounded_probe_negative_control(orbit):
    """Bound 8 loses data at load 0.92 with every status OK; unbounded does not."""
    frames, statuses, counts, ref = orbit
    lost_at = {}
    for bound in (8, 0):
        gv = volume(probe_bound=bound, fuse_mode=0, allocate_mode=0, integrate_mode=0)
        for k in range(N_HIGH):
            d, c = to_dev(frames[k])
            assert gv.fuse(d, frames[k].intr, frames[k].pose, c) == "OK"   # always silent
        stats = gv.table_stats()
        lost_at[bound] = (counts[N_HIGH - 1] - stats["blocks"],
                          int(ref[1][:, 1].sum()) - stats["weight_sum"])
    assert lost_at[0] == (0, 0)
    blocks_lost, contributions_lost = lost_at[8]
    assert blocks_lost > 0 and contributions_lost > 0, lost_at


def test_bounded_probe_exact_at_low_load(orbit):
    """One frame into a 2^18-slot table (load < 0.01): probes stay short, the
    bounded probe loses nothing."""
    frames, statuses, counts, _ = orbit
    spec = synth.VolumeSpec(0.01, 0.04, 1 << 18, 1 << 15)
    gv = volume(spec, probe_bound=8)
    ov = oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                             spec.pool_blocks)
    d, c = to_dev(frames[0])
    assert gv.fuse(d, frames[0].intr, frames[0].pose, c) == ov.fuse_frame(frames[0]) == "OK"
    assert gv.table_stats()["probe_max"] <= 8
    assert_same_volume(gv, ov)


def _host_probe_lengths(table_bytes, slots):
    """Probe length of every occupied slot, from the table's raw bytes."""
    ent = np.frombuffer(table_bytes, dtype=np.uint64).reshape(slots, 2)
    keys = ent[:, 0]
    occ = np.nonzero(keys != np.uint64(0xFFFFFFFFFFFFFFFF))[0]
    k = keys[occ]
    m = np.uint64((1 << 21) - 1)
    bias = 1 << 20
    bx = ((k >> np.uint64(42)) & m).astype(np.int64) - bias
    by = ((k >> np.uint64(21)) & m).astype(np.int64) - bias
    bz = (k & m).astype(np.int64) - bias
    home = np.array([tsdf.tsdf_block_slot(int(x), int(y), int(z), slots)
                     for x, y, z in zip(bx, by, bz)], dtype=np.int64)
    return ((occ.astype(np.int64) - home) & (slots - 1)) + 1


@pytest.mark.parametrize("slot_index", [0, 1])
def test_table_stats_against_table_bytes(orbit, slot_index):
    frames, statuses, counts, _ = orbit
    nbytes = tsdf.tsdf_volume_bytes(SLOTS, SLOTS)
    mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    gv = tsdf.Volume(SPEC.voxel_size, SPEC.truncation, SLOTS, SLOTS, memory=mem)
    if slot_index:
        assert gv.set_option("slot_index", 1) == "OK"
    ov = oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SLOTS, SLOTS)
    for k in range(30):
        d, c = to_dev(frames[k])
        assert gv.fuse(d, frames[k].intr, frames[k].pose, c) == ov.fuse_frame(frames[k]) == "OK"
    stats = gv.table_stats()
    torch.cuda.synchronize()
    lay = gv.layout()
    table = mem[lay.table_offset:lay.table_offset + 16 * SLOTS].cpu().numpy().tobytes()
    lengths = _host_probe_lengths(table, SLOTS)
    assert stats["occupied_slots"] == len(lengths) == ov.block_count() == stats["blocks"]
    assert stats["probe_sum"] == int(lengths.sum())
    assert stats["probe_max"] == int(lengths.max())
    _, ox = ov.export(double=True)
    assert stats["weight_sum"] == int(ox[:, 1].sum())


def test_volume_copy(orbit):
    frames = orbit[0]
    a = volume()
    b = volume()
    ov = oracle.OracleVolume(SPEC.voxel_size, SPEC.truncation, SLOTS, SLOTS)
    for k in (0, 1):
        d, c = to_dev(frames[k])
        assert a.fuse(d, frames[k].intr, frames[k].pose, c) == ov.fuse_frame(frames[k]) == "OK"
    assert b.copy_from(a) == "OK"
    ca, xa = a.export()
    cb, xb = b.export()
    assert np.array_equal(ca, cb) and np.array_equal(xa, xb)   # a byte copy
    d, c = to_dev(frames[2])
    assert b.fuse(d, frames[2].intr, frames[2].pose, c) == ov.fuse_frame(frames[2]) == "OK"
    assert_same_volume(b, ov)
    # shapes and index modes must agree
    other = volume(synth.VolumeSpec(0.01, 0.04, SLOTS, SLOTS // 2))
    assert other.copy_from(a) == "INVALID_ARG"
    k14 = volume(slot_index=1)
    assert k14.copy_from(a) == "INVALID_ARG"
    assert a.copy_from(a) == "INVALID_ARG"
