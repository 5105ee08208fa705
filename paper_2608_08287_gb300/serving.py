"""Continuous-batching fusion server for many reconstruction sessions.

Many independent sessions (cameras) stream depth + colour frames. Each
session owns a hash-blocked TSDF volume resident on the device for its
lifetime; sessions are admitted when their volume's bytes fit a device-memory
budget, and wait in arrival order otherwise. The server runs a loop:

  * frames whose arrival time has passed join their session's queue;
  * whenever fewer than two batches are in flight, every admitted session that
    has a queued frame and nothing in flight contributes its OLDEST frame (so
    each session's frames stay in order), the frames are copied host to
    device into staging slots, and one ``tsdf_fuse_batch_async`` call fuses
    them all (allocate + integrate for every session: two persistent launches,
    optionally replayed from a CUDA graph);
  * completed batches (polled CUDA events) give each frame its latency,
    completion minus arrival.

Frames that arrive while the GPU is busy are admitted as soon as a batch
slot frees: this is continuous batching, not a queue in front of one-frame
launches. ``PerFrameServer`` is the baseline: the same schedule, one
copy + ``tsdf_fuse_frame_async`` per frame on one stream.

All fusion runs in libtsdf's kernels; this module schedules and marshals.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import synth, tsdf

# Session classes by camera resolution: coarser voxels for coarser cameras, so
# that a whole orbit of the room fits each class's pool.
SESSION_CLASSES = {
    (160, 120): synth.VolumeSpec(0.02, 0.08, 1 << 16, 1 << 14),
    (320, 240): synth.VolumeSpec(0.01, 0.04, 1 << 18, 1 << 16),
    (640, 480): synth.VolumeSpec(0.005, 0.02, 1 << 20, 1 << 18),
}


@dataclass
class SessionPlan:
    sid: int
    res: tuple
    request: float          # when the session asks to start (s)
    duration: float         # how long it streams once admitted (s)
    frame0: int             # offset into the frame bank
    admit: float = math.nan  # when it was admitted (set by the schedule)
    arrivals: np.ndarray = field(default_factory=lambda: np.zeros(0))


def volume_bytes(res):
    spec = SESSION_CLASSES[res]
    return tsdf.tsdf_volume_bytes(spec.table_slots, spec.pool_blocks)


def plan_sessions(n_sessions=256, fps=30.0, window=10.0, seed=20261207, min_dur=5.0,
                  max_dur=10.0, budget_bytes=None):
    """Seeded session requests, admission by memory (first come, first served),
    and Poisson frame arrivals (exponential gaps, mean 1/fps) while admitted."""
    u = synth.uniform(seed, 41, n_sessions * 4).reshape(n_sessions, 4)
    res_list = list(SESSION_CLASSES)
    plans = []
    for i in range(n_sessions):
        dur = min_dur + (max_dur - min_dur) * u[i, 0]
        req = (window - dur) * u[i, 1]
        plans.append(SessionPlan(i, res_list[int(u[i, 2] * 3) % 3], float(req), float(dur),
                                 int(u[i, 3] * 1e6)))
    # admission simulation: memory is held from admission to admission + duration
    budget = float("inf") if budget_bytes is None else budget_bytes
    order = sorted(plans, key=lambda p: p.request)
    active = []  # (end time, bytes)
    used = 0
    # process requests in time order, freeing memory as sessions end
    pending = collections.deque(order)
    queue = collections.deque()
    clock = 0.0
    while pending or queue:
        nxt_req = pending[0].request if pending else math.inf
        nxt_end = min(active)[0] if active else math.inf
        if queue and (used + volume_bytes(queue[0].res) <= budget):
            p = queue.popleft()
            p.admit = clock
            used += volume_bytes(p.res)
            active.append((p.admit + p.duration, volume_bytes(p.res)))
            continue
        if nxt_req <= nxt_end:
            clock = nxt_req
            queue.append(pending.popleft())
        elif nxt_end < math.inf:
            clock = nxt_end
            active.sort()
            _, b = active.pop(0)
            used -= b
        else:
            break  # a session larger than the whole budget can never run
    for i, p in enumerate(plans):
        if math.isnan(p.admit):
            continue
        gaps = -np.log1p(-synth.uniform(seed, 1000 + i, int(fps * p.duration * 3) + 16)) / fps
        t = p.admit + np.cumsum(gaps)
        p.arrivals = t[t < min(p.admit + p.duration, window)]
    return plans


class FrameBank:
    """Pre-rendered room-orbit frames per resolution, in pinned host memory."""

    def __init__(self, torch, n_frames=24, step=12, resolutions=None, pool=None):
        self.res = list(resolutions or SESSION_CLASSES)
        self.n = n_frames
        self.frames = {}
        jobs = [(r, k) for r in self.res for k in range(n_frames)]
        if pool is not None:
            rendered = pool.starmap(_render, [(r[0], r[1], k * step) for r, k in jobs])
        else:
            rendered = [_render(r[0], r[1], k * step) for r, k in jobs]
        for (r, k), (depth, rgb, intr, pose) in zip(jobs, rendered):
            # intrinsics and pose kept as ready-made C structs for the launch calls
            self.frames.setdefault(r, []).append(
                (torch.from_numpy(depth).pin_memory(), torch.from_numpy(rgb).pin_memory(),
                 tsdf.intrinsics(intr), tsdf.pose_struct(pose),
                 int(np.count_nonzero(depth > 0))))

    def get(self, res, k):
        return self.frames[res][k % self.n]


def _render(w, h, frame):
    f = synth.room_frame(frame, width=w, height=h)
    return f.depth, f.rgb, f.intr, f.pose


@dataclass
class Result:
    latencies_ms: np.ndarray
    points: int
    frames: int
    wall_s: float
    batches: int = 0

    def summary(self):
        lat = self.latencies_ms
        return {"frames": int(self.frames), "points": int(self.points),
                "pts_per_s": round(self.points / self.wall_s, 1) if self.wall_s else 0.0,
                "frames_per_s": round(self.frames / self.wall_s, 1) if self.wall_s else 0.0,
                "p50_ms": round(float(np.percentile(lat, 50)), 4) if len(lat) else None,
                "p99_ms": round(float(np.percentile(lat, 99)), 4) if len(lat) else None,
                "max_ms": round(float(np.max(lat)), 4) if len(lat) else None,
                "batches": int(self.batches), "wall_s": round(self.wall_s, 3)}


def peak_concurrency(plans):
    """Largest number of sessions of each class admitted at the same time."""
    peaks = {}
    for r in SESSION_CLASSES:
        ev = []
        for p in plans:
            if p.res == r and len(p.arrivals):
                ev += [(p.admit, 1), (p.admit + p.duration, -1)]
        cur = best = 0
        for _, d in sorted(ev, key=lambda e: (e[0], e[1])):
            cur += d
            best = max(best, cur)
        peaks[r] = best
    return peaks


class _Base:
    """Shared state: the schedule, staging rings, and per-class volume pools.

    A session takes a volume from its class's pool (reset on the stream) when
    its first frame is launched and returns it when its last frame completes.
    Pools hold the schedule's peak concurrency plus two per class, or one
    volume per session with ``reuse_volumes=False``."""

    def __init__(self, torch, bank, plans, max_inflight_frames=256, reuse_volumes=True):
        self.torch = torch
        self.bank = bank
        self.plans = [p for p in plans if len(p.arrivals)]
        self.stream = torch.cuda.Stream()
        self.ring = {}
        for r in bank.res:
            w, h = r
            self.ring[r] = collections.deque(
                (torch.empty((h, w), dtype=torch.float32, device="cuda"),
                 torch.empty((h, w, 3), dtype=torch.uint8, device="cuda"))
                for _ in range(max_inflight_frames))
        if reuse_volumes:
            counts = {r: n + 2 for r, n in peak_concurrency(self.plans).items()}
        else:
            counts = collections.Counter(p.res for p in self.plans)
        self.pool = {}
        for r in SESSION_CLASSES:
            spec = SESSION_CLASSES[r]
            self.pool[r] = collections.deque(
                tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
                for _ in range(counts.get(r, 0)))
        self.assigned = {}
        self.finished = {}            # sid -> volume (reuse_volumes=False keeps them)
        self.reuse = reuse_volumes
        ev = [(t, p.sid, k) for p in self.plans for k, t in enumerate(p.arrivals)]
        ev.sort()
        self.arrivals = ev
        self.plan_of = {p.sid: p for p in self.plans}
        self.remaining = {p.sid: len(p.arrivals) for p in self.plans}

    def volume_for(self, sid):
        """The session's volume, taking (and resetting) one from its pool on
        first use; None if the pool is empty right now."""
        v = self.assigned.get(sid)
        if v is None:
            res = self.plan_of[sid].res
            if not self.pool[res]:
                return None
            v = self.pool[res].popleft()
            if v.reset(self.stream.cuda_stream) != "OK":
                raise RuntimeError("tsdf_volume_reset failed")
            self.assigned[sid] = v
        return v

    def frame_done(self, sid):
        self.remaining[sid] -= 1
        if self.remaining[sid] == 0:
            v = self.assigned.pop(sid)
            if self.reuse:
                self.pool[self.plan_of[sid].res].append(v)
            else:
                self.finished[sid] = v

    def close(self):
        for q in self.pool.values():
            for v in q:
                v.close()
        for v in list(self.assigned.values()) + list(self.finished.values()):
            v.close()


class BatchedServer(_Base):
    """Continuous batching: at most one frame per session per batch, two
    batches in flight."""

    def __init__(self, torch, bank, plans, max_batch=128, use_graph=True, **kw):
        super().__init__(torch, bank, plans, **kw)
        self.max_batch = max_batch
        self.batch = tsdf.Batch(max_batch, use_graph=1 if use_graph else 0)

    def run(self, speed=1.0):
        torch = self.torch
        queues = collections.defaultdict(collections.deque)
        busy = set()                      # sessions with a frame in flight
        inflight = collections.deque()    # (event, [(sid, arrival, points, staging)])
        lat, points, n_frames, n_batches = [], 0, 0, 0
        ai = 0
        n_total = len(self.arrivals)
        t0 = time.perf_counter()
        while n_frames < n_total:
            now = (time.perf_counter() - t0) * speed
            while ai < n_total and self.arrivals[ai][0] <= now:
                t, sid, k = self.arrivals[ai]
                queues[sid].append((t, k))
                ai += 1
            while inflight and inflight[0][0].query():
                ev, items = inflight.popleft()
                done = (time.perf_counter() - t0) * speed
                for sid, t_arr, pts, slot, res in items:
                    lat.append((done - t_arr) * 1e3 / speed)
                    points += pts
                    n_frames += 1
                    busy.discard(sid)
                    self.ring[res].append(slot)
                    self.frame_done(sid)
            if len(inflight) < 2:
                ready = [sid for sid, q in queues.items() if q and sid not in busy]
                if ready:
                    ready.sort(key=lambda s: queues[s][0][0])
                    ready = [sid for sid in ready[:self.max_batch]
                             if self.ring[self.plan_of[sid].res]
                             and self.volume_for(sid) is not None]
                if ready:
                    items, frames = [], []
                    with torch.cuda.stream(self.stream):
                        for sid in ready:
                            t_arr, k = queues[sid].popleft()
                            plan = self.plan_of[sid]
                            depth_h, rgb_h, intr, pose, pts = self.bank.get(plan.res,
                                                                            plan.frame0 + k)
                            slot = self.ring[plan.res].popleft()
                            slot[0].copy_(depth_h, non_blocking=True)
                            slot[1].copy_(rgb_h, non_blocking=True)
                            frames.append((self.assigned[sid], slot[0], slot[1], intr, pose))
                            items.append((sid, t_arr, pts, slot, plan.res))
                            busy.add(sid)
                    st = self.batch.fuse_async(frames, stream=self.stream.cuda_stream)
                    if st != "OK":
                        raise RuntimeError(f"tsdf_fuse_batch_async: {st}")
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                    inflight.append((ev, items))
                    n_batches += 1
                    continue
            if not inflight and ai < n_total:
                # idle until the next arrival
                wait = self.arrivals[ai][0] / speed - (time.perf_counter() - t0)
                if wait > 0.0005:
                    time.sleep(wait - 0.0003)
        wall = time.perf_counter() - t0
        st, per = self.batch.status(self.max_batch, stream=self.stream.cuda_stream)
        return Result(np.array(lat), points, n_frames, wall, n_batches), st


class PerFrameServer(_Base):
    """Baseline: one host-to-device copy and one tsdf_fuse_frame_async per frame,
    in arrival order, on one stream."""

    def run(self, speed=1.0):
        torch = self.torch
        inflight = collections.deque()
        lat, points, n_frames = [], 0, 0
        ai = 0
        n_total = len(self.arrivals)
        t0 = time.perf_counter()
        while n_frames < n_total:
            now = (time.perf_counter() - t0) * speed
            while inflight and inflight[0][0].query():
                ev, sid, t_arr, pts, slot, res = inflight.popleft()
                done = (time.perf_counter() - t0) * speed
                lat.append((done - t_arr) * 1e3 / speed)
                points += pts
                n_frames += 1
                self.ring[res].append(slot)
                self.frame_done(sid)
            if ai < n_total and self.arrivals[ai][0] <= now and self.ring_free(ai) and \
                    self.volume_for(self.arrivals[ai][1]) is not None:
                t_arr, sid, k = self.arrivals[ai]
                ai += 1
                plan = self.plan_of[sid]
                depth_h, rgb_h, intr, pose, pts = self.bank.get(plan.res, plan.frame0 + k)
                slot = self.ring[plan.res].popleft()
                with torch.cuda.stream(self.stream):
                    slot[0].copy_(depth_h, non_blocking=True)
                    slot[1].copy_(rgb_h, non_blocking=True)
                    st = self.assigned[sid].fuse(slot[0], intr, pose, slot[1],
                                                stream=self.stream.cuda_stream, sync=False)
                    if st != "OK":
                        raise RuntimeError(f"tsdf_fuse_frame_async: {st}")
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                inflight.append((ev, sid, t_arr, pts, slot, plan.res))
                continue
            if not inflight and ai < n_total:
                wait = self.arrivals[ai][0] / speed - (time.perf_counter() - t0)
                if wait > 0.0005:
                    time.sleep(wait - 0.0003)
        wall = time.perf_counter() - t0
        return Result(np.array(lat), points, n_frames, wall, n_frames), "OK"

    def ring_free(self, ai):
        sid = self.arrivals[ai][1]
        return bool(self.ring[self.plan_of[sid].res])


# ----------------------------------------------------------------------------
# native serving core (tsdf_server): the same schedule replayed in C++
# ----------------------------------------------------------------------------
def assign_volumes(plans):
    """Static volume-pool assignment from the schedule: a session reuses a volume
    of its class once the volume's previous session has had its last frame
    arrive (the server keeps each volume's frames in order, so the new session
    queues behind the old one's tail). Returns ({sid: (class, index)}, counts)."""
    free_at = collections.defaultdict(list)   # class -> [time the volume frees]
    out = {}
    for p in sorted([p for p in plans if len(p.arrivals)], key=lambda p: p.arrivals[0]):
        pool = free_at[p.res]
        best = None
        for i, t in enumerate(pool):
            if t <= p.arrivals[0] and (best is None or pool[best] > t):
                best = i
        if best is None:
            pool.append(0.0)
            best = len(pool) - 1
        pool[best] = float(p.arrivals[-1])
        out[p.sid] = (p.res, best)
    return out, {r: len(v) for r, v in free_at.items()}


def native_replay(torch, bank, plans, mode, max_batch=128, use_graph=True, speed=1.0,
                  reuse_volumes=True, keep_volumes=False, max_inflight=4):
    """Replay the schedule through tsdf_server (mode 0: continuous batching,
    mode 1: one frame per launch), at most max_inflight launches in flight.
    Returns (Result, status, volumes by sid or None). Frames come from the
    bank's pinned host buffers."""
    plans = [p for p in plans if len(p.arrivals)]
    if reuse_volumes:
        where, counts = assign_volumes(plans)
    else:
        where = {p.sid: (p.res, i) for i, p in enumerate(plans)}
        counts = collections.Counter(p.res for p in plans)
        counts = {r: len(plans) for r in counts}
    vols = {}
    for r, n in counts.items():
        spec = SESSION_CLASSES[r]
        vols[r] = [tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots,
                               spec.pool_blocks) for _ in range(n)]
    ev = sorted((t, p.sid, k) for p in plans for k, t in enumerate(p.arrivals))
    plan_of = {p.sid: p for p in plans}
    reqs = (tsdf.tsdf_request * len(ev))()
    points = 0
    for i, (t, sid, k) in enumerate(ev):
        p = plan_of[sid]
        depth_h, rgb_h, intr, pose, pts = bank.get(p.res, p.frame0 + k)
        r, j = where[sid]
        q = reqs[i]
        q.volume = vols[r][j].handle.value
        q.depth = depth_h.data_ptr()
        q.rgb = rgb_h.data_ptr()
        q.width = p.res[0]
        q.height = p.res[1]
        q.intr = intr
        q.pose = pose
        q.arrival_s = t / speed
        q.tag = i
        q.reset_volume = 1 if k == 0 else 0
        points += pts
    stream = torch.cuda.Stream()
    max_px = max(w * h for w, h in bank.res)
    server = tsdf.tsdf_server_create(mode, max_batch, max_inflight, max_px,
                                     max_inflight * max_batch + 8, use_graph, stream.cuda_stream)
    try:
        st, comp = tsdf.tsdf_server_replay(server, reqs)
    finally:
        tsdf.tsdf_server_destroy(server)
    lat = np.array([(c.done_s - c.arrival_s) * 1e3 for c in comp[:len(ev)]])
    wall = max(c.done_s for c in comp[:len(ev)]) if len(ev) else 0.0
    res = Result(lat, points, len(ev), wall, 0)
    by_sid = None
    if keep_volumes:
        by_sid = {sid: vols[r][j] for sid, (r, j) in where.items()}
    else:
        for vs in vols.values():
            for v in vs:
                v.close()
    return res, st, by_sid
