"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Acceptance (paper Section 3.3 "Correctness": same block count, no dropped
points; means recovered from sums, Section 2.2):
  * the allocated block-key set is identical (compared as a set: slot and pool
    order are free);
  * the integer-valued weights are identical;
  * tsdf and colour means agree within 1e-5 absolute (float32 sums in a
    different order against the oracle's double sums; weights per voxel stay
    far below the 1e3 contributions at which float32 order error could reach
    1e-5 for values bounded by 1);
  * the status codes are identical.
"""
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


def to_dev(frame, with_rgb=True):
    d = torch.from_numpy(np.ascontiguousarray(frame.depth)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(frame.rgb)).cuda() if with_rgb else None
    return d, c


def gpu_volume(spec, **opts):
    v = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    for k, x in opts.items():
        assert v.set_option(k, x) == "OK"
    return v


def oracle_volume(spec):
    return oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                               spec.pool_blocks)


def assert_same_volume(gv, ov, with_rgb=True):
    gc, gx = sort_blocks(*gv.export())
    oc, ox = ov.export(double=True)
    assert gc.shape == oc.shape, (gc.shape, oc.shape)
    assert np.array_equal(gc, oc), "block-key sets differ"
    assert np.array_equal(gx[:, 1], ox[:, 1].astype(np.float32)), "weights differ"
    err_t = float(np.max(np.abs(gx[:, 0] - ox[:, 0]))) if len(gc) else 0.0
    assert err_t <= TOL, err_t
    if with_rgb:
        err_c = float(np.max(np.abs(gx[:, 2:] - ox[:, 2:]))) if len(gc) else 0.0
        assert err_c <= TOL, err_c
    else:
        assert not np.any(gx[:, 2:])
    assert gv.block_count() == ov.block_count()
    return len(gc)


def fuse_both(frames, spec, with_rgb=True, **opts):
    gv = gpu_volume(spec, **opts)
    ov = oracle_volume(spec)
    for f in frames:
        d, c = to_dev(f, with_rgb)
        sg = gv.fuse(d, f.intr, f.pose, c)
        so = ov.fuse_frame(f, with_rgb=with_rgb)
        assert sg == so, (sg, so)
    return gv, ov


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------
def test_plane_sphere_160x120():
    gv, ov = fuse_both([synth.plane_sphere_frame()], synth.PLANE_SPHERE_160)
    n = assert_same_volume(gv, ov)
    assert n == ov.last_stats["unique_blocks"] > 500


def test_room_640x480_full_frame():
    """The benchmark's workload, in the launch configuration it times."""
    gv, ov = fuse_both([synth.room_frame(0)], synth.ROOM_640)
    n = assert_same_volume(gv, ov)
    assert n == ov.last_stats["unique_blocks"] > 5000


# (voxel, truncation) pairs covering half bands M = 4, 3, 4, 5, 2, 8: the
# unrolled walks (M = 2, 4, 8) and the generic loop (M = 3, 5)
BANDS = [(0.05, 0.2), (0.1, 0.3), (0.03, 0.12), (0.02, 0.1), (0.04, 0.08), (0.01, 0.08)]


# (fuse, allocate, integrate) modes: the fused kernel, and the two-stage path
# with each stage A and stage B strategy (stage B's tile strategy after both
# the tile and the paper's stage A); then the fused tile kernel with the
# threads per point set explicitly to 1, 2, 4 and 8 (the default chooses
# them per frame: 4 for the tiny and 160x120 frames, 1 at 640x480)
MODES = [dict(fuse_mode=2),
         dict(fuse_mode=1),
         dict(fuse_mode=0, allocate_mode=2, integrate_mode=1),
         dict(fuse_mode=0, allocate_mode=1, integrate_mode=1),
         dict(fuse_mode=0, allocate_mode=0, integrate_mode=0),
         dict(fuse_mode=0, allocate_mode=1, integrate_mode=0),
         dict(fuse_mode=0, allocate_mode=1, integrate_mode=2),
         dict(fuse_mode=0, allocate_mode=0, integrate_mode=2),
         dict(fuse_mode=2, threads_per_point=1),
         dict(fuse_mode=2, threads_per_point=2),
         dict(fuse_mode=2, threads_per_point=4),
         dict(fuse_mode=2, threads_per_point=8)]
SPLIT = [m for m in range(len(MODES)) if MODES[m].get("threads_per_point", 0) > 1]
SINGLE = [m for m in range(len(MODES)) if m not in SPLIT]


def half_band(v, tau):
    return int(np.rint(np.float32(tau) / np.float32(v)))


def allowed(mode, band=None, policy=0):
    """The split walk exists for the default probe load and half bands 2, 4, 8."""
    if mode in SINGLE:
        return True
    return policy == 0 and (band is None or half_band(*band) in (2, 4, 8))


@pytest.mark.parametrize("seed", range(64))
def test_random_tiny_frames(seed):
    f = synth.random_frame(2000 + seed, width=16 + seed % 5, height=12 + seed % 3)
    v, tau = BANDS[seed % len(BANDS)]
    spec = synth.VolumeSpec(v, tau, 1 << 12, 1 << 12)
    gv, ov = fuse_both([f], spec, **MODES[SINGLE[(seed // len(BANDS)) % len(SINGLE)]])
    assert_same_volume(gv, ov)


SPLIT_BANDS = [b for b in BANDS if half_band(*b) in (2, 4, 8)]


@pytest.mark.parametrize("seed", range(24))
def test_random_tiny_frames_split_walk(seed):
    """Random depth (holes, NaN, spikes) with the walk split over threads:
    every span boundary of every half band, on ragged tiny frames."""
    f = synth.random_frame(3000 + seed, width=13 + seed % 7, height=9 + seed % 4)
    v, tau = SPLIT_BANDS[seed % len(SPLIT_BANDS)]
    spec = synth.VolumeSpec(v, tau, 1 << 12, 1 << 12)
    gv, ov = fuse_both([f], spec, **MODES[SPLIT[seed % len(SPLIT)]])
    assert_same_volume(gv, ov)


@pytest.mark.parametrize("mode", [SINGLE[0]] + SPLIT)
def test_ragged_tiles_and_odd_sizes(mode):
    """Image sizes that are not multiples of the tile (16x16, or 16 x 16/T
    with T threads per point), down to 1x1."""
    for (w, h) in [(1, 1), (17, 3), (33, 31), (100, 7), (161, 121)]:
        f = synth.room_frame(5, width=w, height=h)
        spec = synth.VolumeSpec(0.02, 0.08, 1 << 14, 1 << 12)
        gv, ov = fuse_both([f], spec, **MODES[mode])
        assert_same_volume(gv, ov)


def test_multi_frame_accumulation():
    frames = [synth.room_frame(i * 7, width=160, height=120) for i in range(8)]
    gv, ov = fuse_both(frames, synth.VolumeSpec(0.01, 0.04, 1 << 16, 1 << 14))
    assert_same_volume(gv, ov)


def test_without_colour():
    gv, ov = fuse_both([synth.plane_sphere_frame()], synth.PLANE_SPHERE_160, with_rgb=False)
    assert_same_volume(gv, ov, with_rgb=False)


def test_empty_and_invalid_frames():
    spec = synth.VolumeSpec(0.01, 0.04, 1 << 10, 1 << 8)
    zero = synth.Frame(depth=np.zeros((24, 32), np.float32), rgb=np.zeros((24, 32, 3), np.uint8),
                       intr=np.array([30, 30, 16, 12], np.float32), pose=np.eye(4, dtype=np.float32))
    nan = synth.Frame(depth=np.full((24, 32), np.nan, np.float32), rgb=zero.rgb, intr=zero.intr,
                      pose=zero.pose)
    gv, ov = fuse_both([zero, nan], spec)
    assert assert_same_volume(gv, ov) == 0


# ----------------------------------------------------------------------------
# variants must not change the result
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("policy,mode", [(p, m) for p in (0, 1, 2) for m in range(len(MODES))
                                         if allowed(m, policy=p)])
def test_probe_load_policies_and_modes(policy, mode):
    gv, ov = fuse_both([synth.room_frame(3, width=320, height=240)],
                       synth.VolumeSpec(0.005, 0.02, 1 << 16, 1 << 15), probe_load=policy,
                       **MODES[mode])
    assert_same_volume(gv, ov)


@pytest.mark.parametrize("band,mode", [(b, m) for b in BANDS for m in range(len(MODES))
                                       if allowed(m, band=b)])
def test_half_bands_on_room(band, mode):
    v, tau = band
    gv, ov = fuse_both([synth.room_frame(21, width=200, height=150)],
                       synth.VolumeSpec(v, tau, 1 << 16, 1 << 14), **MODES[mode])
    assert_same_volume(gv, ov)


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_room_640x480_every_mode(mode):
    gv, ov = fuse_both([synth.room_frame(40)], synth.ROOM_640, **MODES[mode])
    assert_same_volume(gv, ov)


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_multi_frame_every_mode(mode):
    frames = [synth.room_frame(i * 11, width=320, height=240) for i in range(4)]
    gv, ov = fuse_both(frames, synth.VolumeSpec(0.005, 0.02, 1 << 18, 1 << 16), **MODES[mode])
    assert_same_volume(gv, ov)


def tie_frame(pose):
    """Exact binary geometry: samples and projections land on voxel and pixel
    boundaries (the oracle pins the same frame against the dense brute force)."""
    H = W = 8
    vals = (np.arange(H * W) % 13 + 20).astype(np.float32) / np.float32(16.0)
    depth = vals.reshape(H, W)
    depth[3, 3] = np.nextafter(depth[3, 3], np.float32(9))
    depth[4, 5] = np.nextafter(depth[4, 5], np.float32(0))
    return synth.Frame(depth=depth, rgb=np.full((H, W, 3), 100, np.uint8),
                       intr=np.array([8.0, 8.0, 3.5, 3.5], dtype=np.float32),
                       pose=pose.astype(np.float32))


def ulp_frame():
    """Depths one to three ulps either side of voxel boundaries (v = 1 cm)."""
    H, W = 6, 7
    d = np.empty(H * W, dtype=np.float32)
    for i in range(H * W):
        x = np.float32(1.23) + np.float32(0.01) * np.float32(i % 5)
        for _ in range(i % 7 - 3):
            x = np.nextafter(x, np.float32(9))
        for _ in range(3 - i % 7):
            x = np.nextafter(x, np.float32(0))
        d[i] = x
    return synth.Frame(depth=d.reshape(H, W), rgb=np.zeros((H, W, 3), np.uint8),
                       intr=np.array([6.0, 6.0, 3.0, 2.5], np.float32),
                       pose=np.eye(4, dtype=np.float32))


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_floating_point_contract_on_boundaries(mode):
    """The decisions that depend on floating point (voxel of a sample, pixel of
    a centre, the occlusion test) on inputs built to sit on or within an ulp
    of the boundaries: the block set and the weights are bit-exact."""
    import math
    turned = synth.make_pose(synth.rotation(math.pi / 2), [0.25, -0.5, 0.125])
    for f, (v, tau) in ((tie_frame(np.eye(4)), (0.125, 0.5)), (tie_frame(turned), (0.125, 0.5)),
                        (ulp_frame(), (0.01, 0.04))):
        gv, ov = fuse_both([f], synth.VolumeSpec(v, tau, 1 << 14, 1 << 14), **MODES[mode])
        assert assert_same_volume(gv, ov) > 0


def test_split_walk_option_rules():
    v = gpu_volume(synth.VolumeSpec(0.01, 0.04, 1 << 12, 1 << 12))      # half band 4
    for t in (3, 16, -1):
        assert v.set_option("threads_per_point", t) == "INVALID_ARG"
    assert v.set_option("probe_load", 1) == "OK"                      # automatic: allowed
    assert v.set_option("threads_per_point", 2) == "INVALID_ARG"       # default load only
    assert v.set_option("threads_per_point", 0) == "OK"
    assert v.set_option("probe_load", 0) == "OK"
    assert v.set_option("threads_per_point", 4) == "OK"
    assert v.set_option("probe_load", 2) == "INVALID_ARG"
    assert v.set_option("threads_per_point", 1) == "OK"
    assert v.set_option("probe_load", 2) == "OK"
    m3 = gpu_volume(synth.VolumeSpec(0.1, 0.3, 1 << 12, 1 << 12))      # half band 3
    assert m3.set_option("threads_per_point", 2) == "INVALID_ARG"
    assert m3.set_option("threads_per_point", 1) == "OK"
    assert m3.set_option("threads_per_point", 0) == "OK"


@pytest.mark.parametrize("fuse_mode", [0, 1])
def test_split_walk_is_ignored_by_other_fuse_modes(fuse_mode):
    f = synth.room_frame(9, width=160, height=120)
    gv, ov = fuse_both([f], synth.VolumeSpec(0.01, 0.04, 1 << 14, 1 << 13),
                       threads_per_point=8, fuse_mode=fuse_mode)
    assert_same_volume(gv, ov)


def test_stage_split_and_async_match_sync():
    f = synth.room_frame(11, width=320, height=240)
    spec = synth.VolumeSpec(0.005, 0.02, 1 << 16, 1 << 15)
    d, c = to_dev(f)
    a = gpu_volume(spec)
    assert tsdf.tsdf_allocate_async(a.handle, d, f.width, f.height, f.intr, f.pose) == "OK"
    assert tsdf.tsdf_integrate_async(a.handle, d, f.width, f.height, f.intr, f.pose, c) == "OK"
    assert a.status() == "OK"
    b = gpu_volume(spec)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert b.fuse(d, f.intr, f.pose, c, stream=s, sync=False) == "OK"
    assert b.status(stream=s) == "OK"
    h = gpu_volume(spec)
    depth_h = torch.from_numpy(f.depth).pin_memory()
    rgb_h = torch.from_numpy(f.rgb).pin_memory()
    assert h.fuse_host(depth_h, f.intr, f.pose, rgb_h) == "OK"
    ov = oracle_volume(spec)
    ov.fuse_frame(f)
    for v in (a, b, h):
        assert_same_volume(v, ov)


def test_volume_in_caller_memory_and_reset():
    spec = synth.PLANE_SPHERE_160
    nbytes = tsdf.tsdf_volume_bytes(spec.table_slots, spec.pool_blocks)
    mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    gv = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks,
                     memory=mem)
    f1, f2 = synth.plane_sphere_frame(seed=5), synth.plane_sphere_frame(seed=6)
    d1, c1 = to_dev(f1)
    d2, c2 = to_dev(f2)
    assert gv.fuse(d1, f1.intr, f1.pose, c1) == "OK"
    assert gv.reset() == "OK"
    assert gv.block_count() == 0
    assert gv.fuse(d2, f2.intr, f2.pose, c2) == "OK"
    ov = oracle_volume(spec)
    ov.fuse_frame(f2)
    assert_same_volume(gv, ov)
    lay = gv.layout()
    assert lay.base == mem.data_ptr() and lay.bytes == nbytes


# ----------------------------------------------------------------------------
# load and overflow (Section 7.2: never lose a block silently)
# ----------------------------------------------------------------------------
def high_load_frames(slots, target=0.93, v=0.01, width=160, height=120, step=3):
    """Orbit frames whose union of blocks fills `slots` to at least `target` load
    without exceeding it (counted with the oracle)."""
    probe = oracle_volume(synth.VolumeSpec(v, 4 * v, 1 << 22, 1 << 22))
    frames = []
    for i in range(0, 300, step):
        f = synth.room_frame(i, width=width, height=height)
        probe.fuse_frame(f)
        if probe.block_count() > slots:
            break
        frames.append(f)
        if probe.block_count() >= target * slots:
            break
    return frames


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_high_load_factor_zero_lost_blocks(mode):
    """Table and pool sized so the final load factor exceeds 0.9: the unbounded
    probe keeps every block (the bounded probe of Section 7.2 loses blocks from a
    load of 0.071 on)."""
    slots = 1 << 12
    frames = high_load_frames(slots)
    spec = synth.VolumeSpec(0.01, 0.04, slots, slots)
    gv, ov = fuse_both(frames, spec, **MODES[mode])
    n = assert_same_volume(gv, ov)
    assert n / slots > 0.9, n / slots


@pytest.mark.parametrize("mode", range(len(MODES)))
@pytest.mark.parametrize("pool", [1, 4, 16, "D-1"])
def test_pool_overflow_reported(pool, mode):
    f = synth.plane_sphere_frame()
    spec = synth.PLANE_SPHERE_160
    D = fuse_both([f], spec)[1].block_count()
    p = D - 1 if pool == "D-1" else pool
    small = synth.VolumeSpec(spec.voxel_size, spec.truncation, spec.table_slots, p)
    gv = gpu_volume(small, **MODES[mode])
    d, c = to_dev(f)
    assert gv.fuse(d, f.intr, f.pose, c) == "POOL_FULL"
    assert gv.block_count() == p
    assert gv.fuse(d, f.intr, f.pose, c) == "POISONED"
    assert gv.reset() == "OK"
    big = gpu_volume(spec)
    assert big.fuse(d, f.intr, f.pose, c) == "OK"


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_table_overflow_reported(mode):
    f = synth.plane_sphere_frame()
    spec = synth.VolumeSpec(0.01, 0.04, 64, 64)
    gv = gpu_volume(spec, **MODES[mode])
    ov = oracle_volume(spec)
    d, c = to_dev(f)
    assert ov.fuse_frame(f) == "TABLE_FULL"
    assert gv.fuse(d, f.intr, f.pose, c) == "TABLE_FULL"
    assert gv.block_count() == 64


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_publish_timeout_is_bounded(mode):
    """An entry whose key matches a block the frame needs but whose index is never
    published (Section 2.3, the publication window). The waiters give up after
    the configured limit and the call returns an error; the GPU stays usable."""
    f = synth.plane_sphere_frame()
    spec = synth.PLANE_SPHERE_160
    ov = oracle_volume(spec)
    ov.fuse_frame(f)
    coords, _ = ov.export()
    bx, by, bz = (int(x) for x in coords[len(coords) // 2])
    nbytes = tsdf.tsdf_volume_bytes(spec.table_slots, spec.pool_blocks)
    mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    gv = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks,
                     memory=mem)
    assert gv.set_option("publish_timeout_ns", 20_000_000) == "OK"
    for k, x in MODES[mode].items():
        assert gv.set_option(k, x) == "OK"
    torch.cuda.synchronize()
    lay = gv.layout()
    slot = tsdf.tsdf_block_slot(bx, by, bz, spec.table_slots)
    key = tsdf.tsdf_block_key(bx, by, bz)
    ent = np.zeros(2, dtype=np.uint64)
    ent[0] = np.uint64(key)
    ent[1] = np.uint64(0x00000000FFFFFFFF)  # idx = -1 (unpublished), pad = 0
    off = lay.table_offset + 16 * slot
    mem[off:off + 16].copy_(torch.from_numpy(ent.view(np.uint8)))
    d, c = to_dev(f)
    assert gv.fuse(d, f.intr, f.pose, c) == "PUBLISH_TIMEOUT"
    assert gv.fuse(d, f.intr, f.pose, c) == "POISONED"
    assert gv.reset() == "OK"
    assert gv.fuse(d, f.intr, f.pose, c) == "OK"
    assert_same_volume(gv, ov)


def test_layout_sums_match_export():
    """The pool layout the header documents: per voxel a 16-byte record {tsdf
    sum, weight, red sum, green sum}, and a separate array of blue sums; the
    export's means are those sums divided by the weight."""
    f = synth.room_frame(4, width=320, height=240)
    spec = synth.VolumeSpec(0.005, 0.02, 1 << 16, 1 << 15)
    nbytes = tsdf.tsdf_volume_bytes(spec.table_slots, spec.pool_blocks)
    assert nbytes >= spec.pool_blocks * 512 * 20
    mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    gv = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks,
                     memory=mem)
    d, c = to_dev(f)
    assert gv.fuse(d, f.intr, f.pose, c) == "OK"
    coords, vox = gv.export()          # pool order: block j is pool index j
    n = len(coords)
    lay = gv.layout()
    sums = mem[lay.voxel_sums_offset:lay.voxel_sums_offset + 16 * 512 * n].cpu().numpy()
    sums = sums.view(np.float32).reshape(n, 512, 4)
    blue = mem[lay.blue_sums_offset:lay.blue_sums_offset + 4 * 512 * n].cpu().numpy()
    blue = blue.view(np.float32).reshape(n, 512)
    w = sums[:, :, 1]
    assert np.array_equal(w, vox[:, 1])
    hit = w > 0
    assert np.array_equal(sums[:, :, 0][hit] / w[hit], vox[:, 0][hit])
    assert np.array_equal(sums[:, :, 2][hit] / (w[hit] * 255), vox[:, 2][hit])
    assert np.array_equal(sums[:, :, 3][hit] / (w[hit] * 255), vox[:, 3][hit])
    assert np.array_equal(blue[hit] / (w[hit] * 255), vox[:, 4][hit])
    assert not np.any(sums[~hit]) and not np.any(blue[~hit])


def test_block_coordinates_match_table():
    """Every published index points at a coordinate row that matches its key."""
    f = synth.room_frame(2, width=320, height=240)
    spec = synth.VolumeSpec(0.005, 0.02, 1 << 16, 1 << 15)
    nbytes = tsdf.tsdf_volume_bytes(spec.table_slots, spec.pool_blocks)
    mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    gv = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks,
                     memory=mem)
    d, c = to_dev(f)
    assert gv.fuse(d, f.intr, f.pose, c) == "OK"
    lay = gv.layout()
    table = mem[lay.table_offset:lay.table_offset + 16 * spec.table_slots].cpu().numpy()
    table = table.view(np.uint64).reshape(-1, 2)
    used = table[:, 0] != np.uint64(tsdf.EMPTY_KEY)
    idx = (table[used, 1] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    n = gv.block_count()
    assert used.sum() == n and sorted(idx.tolist()) == list(range(n))
    coords = mem[lay.coords_offset:lay.coords_offset + 12 * n].cpu().numpy().view(np.int32)
    coords = coords.reshape(-1, 3)
    for key, i in zip(table[used, 0].tolist(), idx.tolist()):
        assert tsdf.tsdf_block_key(*(int(x) for x in coords[i])) == key
