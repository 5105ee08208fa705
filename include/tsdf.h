/*
 * tsdf.h -- C ABI of libtsdf, hash-blocked TSDF fusion on GB300 (sm_103a).
 *
 * The operation is the paper's integration of one depth frame into a
 * hash-blocked TSDF volume (Section 2, "The workload"):
 *   stage A, allocate (Section 2.2 "Allocate", Listing 1 in Section 2.3): every
 *     valid depth point walks its truncation band along its view ray, maps each
 *     voxel that passes the occlusion test to its 8^3 block, and makes sure the
 *     block exists in an open-addressed, linearly probed hash table of 16-byte
 *     entries (64-bit packed key + 32-bit block index, Section 2.1), claiming a
 *     slot with a 64-bit compare-exchange and a pool index with a counter;
 *   stage B, update (Section 2.2 "Update"): the same walk and test, a table
 *     lookup, and weighted SUMS added to five parallel float arrays of the block
 *     pool (signed distance, weight, red, green, blue; Section 2.1).
 * Means are recovered on read-out (Section 2.2), here by tsdf_export_blocks.
 *
 * Geometry (fixed where the paper is silent; identical in every entry point):
 *   pixel (u, v) is a pixel centre; its camera ray is ((u-cx)/fx, (v-cy)/fy, 1);
 *   the band holds 2M+1 samples at range offsets (k-M)*voxel_size, k = 0..2M,
 *   M = lrintf(truncation / voxel_size), along the unit ray; each distinct voxel
 *   is taken once per point; a voxel is accepted when its centre is in front of
 *   the camera, projects (nearest pixel) inside the image onto a valid depth d',
 *   and lies no more than `truncation` behind it; the stored value is
 *   clamp((d - z_centre) / truncation, -1, 1), evaluated at the voxel centre
 *   (Section 4.1); weight 1 per contribution. All integer decisions are taken in
 *   IEEE single precision with a fixed operation order, so they are reproducible.
 *
 * Memory: one device allocation per volume, laid out as
 *   header (block counter, error word) | table (table_slots x 16 B) |
 *   block coordinates (pool_blocks x 3 int32) |
 *   voxel sums (pool_blocks x 512 x {tsdf sum, weight, red sum, green sum},
 *   16 B per voxel) | blue sums (pool_blocks x 512 float32).
 * The paper keeps the five sums in five parallel float arrays (Section 2.1);
 * here four of them sit together so that one 16-byte vector reduction adds
 * them, and the fifth (blue) has an array of its own: 20 bytes per voxel as in
 * the paper. A block with pool index i owns voxels [i*512, (i+1)*512) of both
 * arrays; the voxel (lx, ly, lz) of a block is local index lx + 8*ly + 64*lz.
 * Block coordinates are floor(voxel / 8) and must lie in [-2^20, 2^20); the
 * packed key is (bx+2^20)<<42 | (by+2^20)<<21 | (bz+2^20) (Section 2.1).
 *
 * Streams: every `stream` argument is a cudaStream_t passed as void*
 * (NULL = the legacy default stream). Device pointers must be on the device
 * that was current when the volume was created, and that device must be
 * current when the volume is used.
 *
 * Errors: every call returns a status; nothing throws across the ABI. Table or
 * pool overflow is never silent: the fusion call reports it and the volume is
 * POISONED (later fusion calls return TSDF_ERR_POISONED and do nothing) until
 * tsdf_volume_reset. The probe is unbounded in the paper's sense (it scans
 * until it finds the key or an empty slot); a scan of the whole table reports
 * TSDF_ERR_TABLE_FULL instead of looping.
 */
#ifndef TSDF_H_
#define TSDF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsdf_volume tsdf_volume; /* opaque, owned by the library */

typedef enum tsdf_status {
  TSDF_OK = 0,
  TSDF_ERR_INVALID_ARG = 1,      /* bad argument; nothing was enqueued */
  TSDF_ERR_OUT_OF_MEMORY = 2,    /* a device or pinned allocation failed */
  TSDF_ERR_POOL_FULL = 3,        /* more blocks than pool_blocks (Section 3.4) */
  TSDF_ERR_TABLE_FULL = 4,       /* a probe scanned every slot without room */
  TSDF_ERR_PUBLISH_TIMEOUT = 5,  /* a block index was never published */
  TSDF_ERR_BOUNDS = 6,           /* reserved for bounds-checked kernels; never set now */
  TSDF_ERR_POISONED = 7,         /* volume holds an earlier error; reset it */
  TSDF_ERR_CUDA = 8              /* a CUDA runtime call failed */
} tsdf_status;

typedef struct tsdf_intrinsics {
  float fx, fy, cx, cy; /* pinhole, pixels */
} tsdf_intrinsics;

typedef struct tsdf_pose {
  float m[16]; /* row-major 4x4 camera-to-world; last row 0 0 0 1 (not read) */
} tsdf_pose;

/* Device addresses of a volume's arrays, for inspection and tests. */
typedef struct tsdf_layout {
  void* base;              /* start of the volume's allocation */
  size_t bytes;            /* its size, = tsdf_volume_bytes(...) */
  uint32_t* block_count;   /* device: blocks claimed (may exceed pool on overflow) */
  uint32_t* error_word;    /* device: sticky error bits, see TSDF_ERRBIT_* */
  void* table;             /* device: table_slots entries {uint64 key; int32 idx; int32 pad} */
  int32_t* block_coords;   /* device: pool_blocks x {bx, by, bz} (unused with TSDF_OPT_SLOT_INDEX) */
  float* voxel_sums;       /* device: pool_blocks x 512 x {tsdf, weight, red, green} sums */
  float* blue_sums;        /* device: pool_blocks x 512 blue sums */
  uint32_t table_slots;
  uint32_t pool_blocks;
  size_t table_offset, coords_offset, voxel_sums_offset, blue_sums_offset; /* from base */
} tsdf_layout;

/* Sticky bits of the device error word. PUBLISH_TIMEOUT is also set when
 * stage B finds a block that was claimed but whose index was never
 * published. */
#define TSDF_ERRBIT_POOL_FULL 1u
#define TSDF_ERRBIT_TABLE_FULL 2u
#define TSDF_ERRBIT_PUBLISH_TIMEOUT 4u
#define TSDF_ERRBIT_BOUNDS 8u

/* The empty key and the unpublished index of a table entry (Section 2.3). */
#define TSDF_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull
#define TSDF_UNPUBLISHED (-1)

/* Options (tsdf_volume_set_option). */
typedef enum tsdf_option {
  /* How an insert (stage A, or the fused kernels) reads a probed entry before
   * any compare-exchange (Section 6.2: a GPU-scope atomic load bypasses L1, a
   * plain load may hit in it).
   * 0 = plain load cached in L1 (default), 1 = L2 only (.cg), 2 = relaxed
   * GPU-scope atomic load. */
  TSDF_OPT_PROBE_LOAD = 0,
  /* Upper bound on the wait for a block index to be published, nanoseconds
   * (default 1e9). The wait gives up with TSDF_ERR_PUBLISH_TIMEOUT. */
  TSDF_OPT_PUBLISH_TIMEOUT_NS = 1,
  /* Stage B strategy of the two-stage path (TSDF_OPT_FUSE_MODE 0): 0 = each
   * thread looks up its blocks in the table (a one-entry cache per point) and
   * adds the five sums of every accepted voxel with two fire-and-forget
   * reductions (a 16-byte vector of {tsdf, weight, red, green} and the blue
   * scalar), the paper's update stage (default); 1 = each warp dedupes its
   * points' blocks with __match_any_sync and looks them up once,
   * warp-cooperatively, then the same additions; 2 = the distinct blocks of
   * each 16x16 pixel tile are collected in shared memory and looked up once
   * per tile, warp-cooperatively (long probe chains scanned by the whole
   * warp), then the same additions with each index taken from the tile's
   * list. Batches take 0 and 1. */
  TSDF_OPT_INTEGRATE_MODE = 2,
  /* Launch shape: threads per CTA for both stages (256). */
  TSDF_OPT_THREADS = 3,
  /* Stage A strategy of the two-stage path (TSDF_OPT_FUSE_MODE 0):
   * 0 = the paper's protocol as printed (every warp-distinct
   * key inserted as the walk finds it; a thread that finds its key waits for
   * the index to be published); 1 = the distinct keys of each 16x16 pixel
   * tile, via a shared-memory set, inserted warp-cooperatively after one
   * barrier (default); 2 = the distinct keys of each warp inserted
   * warp-cooperatively, no shared memory. In 1 and 2 counter increments are
   * aggregated per warp and no thread waits: nothing in stage A consumes an
   * index, and the kernel boundary publishes every index before stage B. */
  TSDF_OPT_ALLOCATE_MODE = 4,
  /* What tsdf_fuse_frame* launch: 0 = stage A then stage B (two kernels,
   * Section 2.2, with the strategies above); 1 = one fused kernel in which
   * each warp walks its points once, inserts its distinct blocks (waiting,
   * bounded, for indices published by others) and adds its sums; 2 = one
   * fused kernel per 16x16 pixel tile (default): the walk runs once, the
   * tile's distinct blocks are inserted warp-cooperatively and their indices
   * kept in shared memory, then every accepted voxel's sums are added with
   * no further table probe. Results are identical up to the order of
   * floating-point additions. Safe without a grid barrier because a point
   * only touches blocks whose indices it has resolved. */
  TSDF_OPT_FUSE_MODE = 5,
  /* Batches only, with TSDF_OPT_BATCH_STREAMS 0: cap on resident CTAs per SM
   * of the persistent batched kernels (0 = as many as fit, default). */
  TSDF_OPT_CTAS_PER_SM = 6,
  /* Batches only, with TSDF_OPT_BATCH_STREAMS 0: 1 = capture each
   * configuration's copy-and-launch sequence in a CUDA graph once and replay
   * it for batches of at least 2048 tiles; smaller batches are launched
   * directly with a grid of their own size (default 0: always launch
   * directly). */
  TSDF_OPT_USE_GRAPH = 7,
  /* 1 = a block's pool index is its table slot (Section 6, "Deriving the
   * location from the slot"): the slot winner only counts the block, a thread
   * that finds its key has the index at once, nothing is published and no
   * thread waits. Requires pool_blocks == table_slots (the pool is sized to
   * the table) and a volume with nothing fused since creation or the last
   * reset; TSDF_ERR_INVALID_ARG otherwise. The block_coords array is then
   * unused (the key holds the coordinate) and tsdf_export_blocks returns the
   * blocks in slot order. Overflow can only be TSDF_ERR_TABLE_FULL.
   * 0 = counter-assigned indices (default). */
  TSDF_OPT_SLOT_INDEX = 8,
  /* NEGATIVE CONTROL, never for real use: 0 = unbounded probe (default);
   * B > 0 = every insert and lookup gives up after B probes WITHOUT reporting
   * it, so blocks and contributions can be lost silently -- the behaviour of a
   * probe loop with a compile-time trip count (Section 7, the bounded probe
   * of the Triton arm). It exists to measure that loss against the unbounded
   * probe. Values above table_slots act as unbounded. */
  TSDF_OPT_PROBE_BOUND = 9,
  /* Threads per depth point in the fused tile kernel (TSDF_OPT_FUSE_MODE 2;
   * other modes ignore it): 1 = each thread walks its point's whole band;
   * 2, 4 or 8 = the point's 2M+1 band samples are split into that many
   * contiguous spans, one per thread, so a frame runs on that many times more
   * threads (for small frames that do not fill the GPU); 0 (default) =
   * chosen per frame: the largest of 1, 2 and 4 whose CTAs (one per
   * 16 x 16/TPP pixels) fit the GPU at four per SM, where the split walk
   * exists (default probe load, half band 2, 4 or 8), else 1. The result is
   * the same for every value. Values above 1 need the default
   * TSDF_OPT_PROBE_LOAD and a half band M = round(truncation / voxel_size)
   * of 2, 4 or 8; TSDF_ERR_INVALID_ARG otherwise, and setting another probe
   * load while it is above 1 is rejected too. Not a batch option. */
  TSDF_OPT_THREADS_PER_POINT = 10,
  /* Batches only, with TSDF_OPT_FUSE_MODE 0 (two stages): which stages a call
   * launches. 3 = stage A then stage B (default); 1 = stage A alone; 2 =
   * stage B alone, for frames whose stage A ran before (a separate call on
   * the same frames) -- so that each stage can be timed on its own. Other
   * fuse modes ignore it. */
  TSDF_OPT_BATCH_STAGES = 11,
  /* Batches only: 0 = every frame of a call in one persistent launch per
   * stage (the batched kernels; TSDF_OPT_CTAS_PER_SM and TSDF_OPT_USE_GRAPH
   * apply); k = 1..16 = every frame in a launch of its own -- the
   * single-frame kernels, with the batch's strategy options and the threads
   * per point that the automatic choice of a volume would give one frame of
   * all the call's tiles (1 when they fill the GPU) -- the frames taken
   * largest first and dealt round-robin over k streams the batch owns, which
   * wait for `stream` before their first launch and which `stream` waits for
   * after their last (concurrent kernels fill the GPU where one small frame
   * cannot). Default 8. The result is the same for every value. */
  TSDF_OPT_BATCH_STREAMS = 12
} tsdf_option;

/* ---------------------------------------------------------------------------
 * Volumes
 * ------------------------------------------------------------------------- */

/* Bytes of device memory a volume with these sizes occupies (0 if invalid). */
size_t tsdf_volume_bytes(uint32_t table_slots, uint32_t pool_blocks);

/* Create a volume in library-allocated device memory (cudaMalloc on the
 * current device), initialised empty. table_slots must be a power of two >= 2,
 * 1 <= pool_blocks <= table_slots, voxel_size > 0, truncation >= voxel_size and
 * truncation / voxel_size <= 16. The paper sizes the table at the next power of
 * two above twice the pool (Section 2.1); any pool_blocks <= table_slots is
 * accepted, so load factors up to 1 can be studied. On error *out is NULL. */
tsdf_status tsdf_volume_create(float voxel_size, float truncation, uint32_t table_slots,
                               uint32_t pool_blocks, tsdf_volume** out);

/* Same, in caller-owned device memory of at least tsdf_volume_bytes() bytes,
 * 256-byte aligned (e.g. a torch tensor). The library never frees it; the
 * caller keeps it alive until tsdf_volume_destroy. The harness-owned memory of
 * Section 3.1 ("handed pointers into memory allocated once by the harness").
 * Initialisation is enqueued on `stream`. */
tsdf_status tsdf_volume_create_in(void* dev_mem, size_t bytes, float voxel_size,
                                  float truncation, uint32_t table_slots,
                                  uint32_t pool_blocks, void* stream,
                                  tsdf_volume** out);

/* Empty the volume (table, counter, error word, used part of the pool) and
 * clear the poisoned state. Enqueued on `stream`. */
tsdf_status tsdf_volume_reset(tsdf_volume* vol, void* stream);

/* Release the volume (and its memory if the library allocated it). Waits for
 * the device to finish using it. NULL is ignored. */
void tsdf_volume_destroy(tsdf_volume* vol);

tsdf_status tsdf_volume_set_option(tsdf_volume* vol, tsdf_option opt, int64_t value);
tsdf_status tsdf_volume_layout(const tsdf_volume* vol, tsdf_layout* out);

/* ---------------------------------------------------------------------------
 * Fusion
 * ------------------------------------------------------------------------- */

/* Fuse one frame: stage A then stage B (by default both in one fused kernel,
 * see TSDF_OPT_FUSE_MODE; the result is the same), enqueued on `stream`, then
 * wait for the stream and return the volume's status (as tsdf_volume_status).
 * depth_dev: height*width float32, row-major, device memory; a pixel is valid
 *   iff finite and > 0. rgb_dev: height*width*3 uint8 (interleaved), device
 *   memory, or NULL to skip the colour sums. Both are only read, and only
 *   during the call. width, height in [1, 32768]. */
tsdf_status tsdf_fuse_frame(tsdf_volume* vol, const float* depth_dev, int width, int height,
                            const tsdf_intrinsics* intr, const tsdf_pose* pose,
                            const uint8_t* rgb_dev, void* stream);

/* As tsdf_fuse_frame but only enqueues; errors surface through
 * tsdf_volume_status. depth_dev and rgb_dev must stay valid until the stream
 * reaches the end of the work. */
tsdf_status tsdf_fuse_frame_async(tsdf_volume* vol, const float* depth_dev, int width,
                                  int height, const tsdf_intrinsics* intr,
                                  const tsdf_pose* pose, const uint8_t* rgb_dev,
                                  void* stream);

/* End-to-end variant with HOST inputs: copies depth (and rgb when not NULL)
 * to device staging owned by the volume (grown on first use, kept until
 * destroy), fuses, and returns the status, all ordered on `stream`. Host
 * buffers in pinned memory make the copies asynchronous. */
tsdf_status tsdf_fuse_frame_host(tsdf_volume* vol, const float* depth_host, int width,
                                 int height, const tsdf_intrinsics* intr,
                                 const tsdf_pose* pose, const uint8_t* rgb_host,
                                 void* stream);

/* Largest frame (width * height) tsdf_fuse_frame_host_noalloc accepts. */
#define TSDF_NOALLOC_MAX_PIXELS (1u << 20)

/* As tsdf_fuse_frame_host, but allocates nothing. (The paper has no
 * counterpart; this is for callers of this library.) Callers that cannot let
 * the library call cudaMalloc -- a real-time loop that must not stall on an
 * allocation, a process whose device memory is fully budgeted by its own
 * allocator, a plugin host that forbids plugins to own device memory -- use
 * this call: the frame is staged in one fixed array compiled into the library
 * (TSDF_NOALLOC_MAX_PIXELS * 7 bytes, 7 MiB, held by every GPU that loads the
 * library until the process exits) instead of volume-owned staging.
 * width * height above TSDF_NOALLOC_MAX_PIXELS returns TSDF_ERR_INVALID_ARG
 * and does nothing. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture. Every call on a device shares the one array:
 * calls whose work overlaps on the GPU (two host threads, or two streams)
 * race on it and must be serialised by the caller. Each call waits for
 * `stream` before returning, on success and on every error after its copies
 * are enqueued, so consecutive calls from one thread are safe. The frame is
 * validated (as tsdf_fuse_frame does) before anything is copied. The array
 * keeps the last frame; each call overwrites what it reads. The looked-up
 * address is cached for the life of the CUDA context: cudaDeviceReset between
 * calls is not supported. */
tsdf_status tsdf_fuse_frame_host_noalloc(tsdf_volume* vol, const float* depth_host, int width,
                                         int height, const tsdf_intrinsics* intr,
                                         const tsdf_pose* pose, const uint8_t* rgb_host,
                                         void* stream);

/* Stage A alone (Section 2.2 "Allocate"): enqueue block allocation. */
tsdf_status tsdf_allocate_async(tsdf_volume* vol, const float* depth_dev, int width,
                                int height, const tsdf_intrinsics* intr,
                                const tsdf_pose* pose, void* stream);

/* Stage B alone (Section 2.2 "Update"): enqueue integration into blocks that
 * stage A allocated for the same frame. A contribution whose block is absent
 * (only possible after an overflow) is skipped. */
tsdf_status tsdf_integrate_async(tsdf_volume* vol, const float* depth_dev, int width,
                                 int height, const tsdf_intrinsics* intr,
                                 const tsdf_pose* pose, const uint8_t* rgb_dev,
                                 void* stream);

/* Wait for `stream`, read the device error word and map it to a status
 * (POOL_FULL, then TABLE_FULL, then PUBLISH_TIMEOUT, then BOUNDS). Any error
 * poisons the volume. */
tsdf_status tsdf_volume_status(tsdf_volume* vol, void* stream);

/* Number of allocated blocks, min(claimed, pool_blocks). Waits for `stream`. */
tsdf_status tsdf_volume_block_count(tsdf_volume* vol, void* stream, uint32_t* n);

/* ---------------------------------------------------------------------------
 * Batched fusion: one frame for each of many volumes (independent sessions)
 * per launch. Not in the paper, whose harness fuses one frame per launch; the
 * per-frame computation is the same.
 * ------------------------------------------------------------------------- */

typedef struct tsdf_batch tsdf_batch; /* opaque, owned by the library */

/* One frame of a batch. All pointers as for tsdf_fuse_frame_async. */
typedef struct tsdf_frame {
  tsdf_volume* volume;
  const float* depth; /* device, height x width float32 */
  const uint8_t* rgb; /* device, height x width x 3, or NULL */
  int width, height;
  tsdf_intrinsics intr;
  tsdf_pose pose;
} tsdf_frame;

/* A batch context for up to max_frames frames per call, on the current
 * device: two session tables (device + pinned host, double-buffered), a
 * status buffer, and the streams of TSDF_OPT_BATCH_STREAMS (8 at creation).
 * One host thread at a time may call into a batch context. */
tsdf_status tsdf_batch_create(int max_frames, tsdf_batch** out);
void tsdf_batch_destroy(tsdf_batch* batch);

/* TSDF_OPT_PROBE_LOAD, TSDF_OPT_ALLOCATE_MODE (1 or 2), TSDF_OPT_INTEGRATE_MODE,
 * TSDF_OPT_FUSE_MODE (default 2, as for volumes), TSDF_OPT_CTAS_PER_SM,
 * TSDF_OPT_USE_GRAPH, TSDF_OPT_BATCH_STAGES, TSDF_OPT_BATCH_STREAMS (setting
 * it above the streams the batch has creates the missing streams and their
 * events: TSDF_ERR_CUDA if that fails). */
tsdf_status tsdf_batch_set_option(tsdf_batch* batch, tsdf_option opt, int64_t value);

/* Enqueue the fusion of n frames (1 <= n <= max_frames), each into a distinct
 * volume, on `stream`: with TSDF_OPT_BATCH_STREAMS k > 0 (the default) one
 * launch per frame over the batch's k streams, forked from and joined back
 * into `stream`; with 0, allocation of every frame, then integration of every
 * frame (two persistent launches), or one fused launch. Returns after
 * enqueueing; it may first wait for the batch's launch before last (the
 * session tables are double-buffered). Frame buffers must stay valid until
 * the stream completes. Any poisoned volume rejects the whole call. */
tsdf_status tsdf_fuse_batch_async(tsdf_batch* batch, const tsdf_frame* frames, int n,
                                  void* stream);

/* Wait for `stream` and report the status of every frame of the last batch
 * (per_frame may be NULL; otherwise n >= that batch's size; per_frame[i] is
 * frames[i]'s). Returns the error of the first frame, in the call's order,
 * that has one, and poisons the volumes that have one. */
tsdf_status tsdf_batch_status(tsdf_batch* batch, void* stream, tsdf_status* per_frame, int n);

/* ---------------------------------------------------------------------------
 * Streaming host input (not in the paper, whose harness fuses frames already
 * in device memory, Section 4): a sequence of frames given in HOST memory,
 * fused in order, each frame's host-to-device copy overlapping the fusion of
 * the frame before it.
 * ------------------------------------------------------------------------- */

/* Fuse frames[0..n-1] in order, frames[i] into frames[i].volume (the same
 * volume may take several frames, or each frame its own). Here depth and rgb
 * are HOST pointers (height x width float32; height x width x 3 uint8 or
 * NULL); in pinned memory the copies run asynchronously and overlap the
 * kernels, otherwise they are staged by the CUDA runtime. Each frame is
 * copied on a copy stream owned by frames[0].volume into one of its two
 * staging slots (frame i into slot i mod 2, after the kernel of frame i-2 has
 * finished reading it), then fused on `stream` exactly as
 * tsdf_fuse_frame_async fuses it, and its volume's error word is copied back
 * into pinned memory (right after the frame when a later frame of the call
 * goes into the same volume, else after the last frame). The call waits
 * once, for the whole sequence, then
 * writes status[i] for every frame: OK, the frame's error (which poisons its
 * volume), POISONED for a volume poisoned before the call or by an earlier
 * frame of it. Returns the first non-OK status, else OK.
 * Every frame is validated (as tsdf_fuse_frame does) before anything is
 * enqueued; a frame that fails validation returns its error and enqueues
 * nothing. The staging slots, the copy stream, its events and the pinned
 * status words are made on the first call (or grown when a call needs larger
 * slots or more frames) and kept until frames[0].volume is destroyed; a call
 * on that volume must not overlap another such call. Host buffers may be
 * reused when the call returns. The volumes must be on the current device. */
tsdf_status tsdf_fuse_frames_host(const tsdf_frame* frames, int n, tsdf_status* status,
                                  void* stream);

/* ---------------------------------------------------------------------------
 * Autotuning (not in the paper): time the strategies on the caller's frames
 * and keep the fastest. Times are medians of `reps` repetitions (1..1000)
 * after one warm-up, CUDA events on `stream`, L2 evicted before each.
 * ------------------------------------------------------------------------- */

typedef struct tsdf_tuning {
  int allocate_mode, integrate_mode, fuse_mode, probe_load; /* the chosen strategy */
  int ctas_per_sm, use_graph; /* batches: the chosen launch shape (0 for a volume) */
  int candidates;             /* configurations timed */
  float best_ms;              /* median time of the chosen configuration */
  float default_ms;           /* median time of the default configuration */
  int threads_per_point;      /* volumes: the chosen TSDF_OPT_THREADS_PER_POINT, 0 = automatic
                                 (1 for a batch) */
  int batch_streams;          /* batches: the chosen TSDF_OPT_BATCH_STREAMS (0 for a volume) */
} tsdf_tuning;

/* Tune `vol` for this frame: every stage A x stage B strategy, the fused
 * kernels, the probe loads and (where the half band allows it) 2, 4 and 8
 * threads per point in the fused tile kernel, each fusing the frame into a
 * scratch copy of the
 * volume's current state (restored before every repetition). The volume's
 * contents are not modified; its options are set to the fastest
 * configuration, which *out describes. Needs device memory for one more
 * volume of the same size (TSDF_ERR_OUT_OF_MEMORY otherwise). If the frame
 * overflows the volume the overflow status is returned and nothing is set.
 * Waits for `stream`. */
tsdf_status tsdf_autotune_frame(tsdf_volume* vol, const float* depth_dev, int width, int height,
                                const tsdf_intrinsics* intr, const tsdf_pose* pose,
                                const uint8_t* rgb_dev, int reps, void* stream,
                                tsdf_tuning* out);

/* Tune `batch` for these frames: the strategies, then the CTAs-per-SM cap of
 * the persistent grid (1..4 or all), then graph replay on or off (all with
 * TSDF_OPT_BATCH_STREAMS 0), then one launch per frame over 4, 8 and 16
 * streams with the best strategy. Every
 * frame's volume must be empty (nothing fused since creation or reset;
 * TSDF_ERR_INVALID_ARG otherwise): the volumes are reset before each
 * repetition and are left empty. The batch's options are set to the fastest
 * configuration, which *out describes. Waits for `stream`. */
tsdf_status tsdf_batch_autotune(tsdf_batch* batch, const tsdf_frame* frames, int n, int reps,
                                void* stream, tsdf_tuning* out);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of frames from many sessions (not in the
 * paper). A server owns device staging for its in-flight frames, a batch
 * context and a clock; frames are submitted with their arrival times and
 * tsdf_server_poll drives everything: it retires finished launches and, while
 * fewer than max_inflight launches are in flight, launches the head frame of
 * every session (volume) with nothing in flight, oldest first, up to
 * max_batch per launch. A session's frames run in submission order.
 * ------------------------------------------------------------------------- */

typedef struct tsdf_server tsdf_server; /* opaque, owned by the library */

/* One frame to serve. depth/rgb are HOST buffers (pinned for asynchronous
 * copies) that must stay valid until the frame's completion is reported. */
typedef struct tsdf_request {
  tsdf_volume* volume;
  const float* depth;   /* host, height x width float32 */
  const uint8_t* rgb;   /* host, height x width x 3, or NULL */
  int width, height;
  tsdf_intrinsics intr;
  tsdf_pose pose;
  double arrival_s;     /* on the server's clock (replay: seconds from its start) */
  uint64_t tag;         /* caller's identifier, returned with the completion */
  int reset_volume;     /* 1 = empty the volume before this frame (a new session) */
} tsdf_request;

typedef struct tsdf_completion {
  uint64_t tag;
  double arrival_s;
  double done_s;        /* when the server saw the frame's launch complete */
  tsdf_status status;   /* launch status (volume errors: tsdf_volume_status) */
} tsdf_completion;

/* mode 0: continuous batching (a launch of several frames uses
 * tsdf_fuse_batch_async, with a batch context for each launch stream; a
 * launch of one frame takes the single-frame path); each
 * session's head frame is copied into staging as soon as a slot is free, on
 * a copy stream the server owns, and a launch waits only for its own frames'
 * copies; each launch in flight runs on one of max_inflight streams the
 * server owns, after the work enqueued on `stream` before it, so that a
 * launch runs beside those already in flight. mode 1: one frame per launch
 * with its copy just before it, all on `stream` (the baseline).
 * max_frame_pixels bounds a frame's size; staging_frames (>= max_batch)
 * device staging slots of that size are allocated here (mode 0 also makes
 * the copy stream, one event per slot, the launch streams and their batch
 * contexts), and nothing
 * is allocated afterwards. use_graph as TSDF_OPT_USE_GRAPH. */
tsdf_status tsdf_server_create(int mode, int max_batch, int max_inflight, int max_frame_pixels,
                               int staging_frames, int use_graph, void* stream,
                               tsdf_server** out);
void tsdf_server_destroy(tsdf_server* server);
/* Seconds since the server was created (steady clock). */
double tsdf_server_clock(const tsdf_server* server);
tsdf_status tsdf_server_submit(tsdf_server* server, const tsdf_request* request);
/* Retire and launch; writes up to `capacity` completions, returns how many
 * (-1 if server is NULL). */
int tsdf_server_poll(tsdf_server* server, tsdf_completion* out, int capacity);
/* Frames submitted and not yet reported complete. */
int tsdf_server_pending(const tsdf_server* server);
/* Replay n requests sorted by arrival (arrival_s = seconds from the start of
 * the replay, tags unique) in real time: each is submitted when the server's
 * clock reaches it, the loop polls until all complete, and out[i] receives
 * request i's completion (times in seconds from the start). Returns the
 * first launch error, else TSDF_OK. */
tsdf_status tsdf_server_replay(tsdf_server* server, const tsdf_request* requests, int n,
                               tsdf_completion* out);

/* ---------------------------------------------------------------------------
 * Read-out (Section 2.2: means recovered at extraction)
 * ------------------------------------------------------------------------- */

/* Copy every allocated block to host memory, in pool order (slot order with
 * TSDF_OPT_SLOT_INDEX): coords_host gets
 * n x {bx, by, bz}; voxels_host gets n x 5 x 512 float32, per block the
 * channels {tsdf mean, weight, red mean, green mean, blue mean} (means are
 * sum / weight where weight > 0, else 0; colours in [0, 1]). If capacity < n
 * nothing is copied and TSDF_ERR_INVALID_ARG is returned; *n_out is always n.
 * Either host pointer may be NULL to query n. Waits for `stream`. */
tsdf_status tsdf_export_blocks(tsdf_volume* vol, int32_t* coords_host, float* voxels_host,
                               uint32_t capacity, uint32_t* n_out, void* stream);

/* Surface extraction: marching tetrahedra over the allocated blocks (the
 * extraction stage of Section 2, which the paper runs once in CUDA C++ and
 * excludes from its comparison; Section 2 also reports that most of its
 * measured time was the device-to-host copy, so the two are timed apart).
 *   - grid points are voxel centres (g + 1/2) * voxel_size; every voxel g
 *     whose 8 corners g + {0,1}^3 all have weight > 0 spans a cube; a corner's
 *     value is its mean tsdf;
 *   - each cube is split into the 6 tetrahedra around its diagonal from corner
 *     0 to corner 7 (corner c = g + (c&1, c>>1&1, c>>2&1));
 *   - a corner is inside when its value is < 0; each tetrahedron edge with
 *     ends on both sides holds a vertex p_lo + t (p_hi - p_lo),
 *     t = v_lo / (v_lo - v_hi), lo the corner whose offset bits are a subset
 *     of the other's;
 *   - one lone corner gives one triangle, a pair gives two; every triangle is
 *     wound so its normal points towards positive values (free space).
 * A triangle is 9 float32 (x, y, z of three vertices, metres); its cell record
 * is 4 int32 {gx, gy, gz, 2*tetrahedron + k}: the cube's voxel and which
 * triangle of which tetrahedron it is. Triangle order is unspecified. */

typedef struct tsdf_extract_timing {
  float compute_ms;   /* the extraction kernel (CUDA events) */
  float d2h_ms;       /* the device-to-host copies of the result */
  uint64_t d2h_bytes; /* bytes copied to the host */
} tsdf_extract_timing;

/* Enqueue the extraction into device buffers: at most `capacity` triangles
 * and cell records are written (either pointer may be NULL; cells_dev must be
 * 16-byte aligned, TSDF_ERR_INVALID_ARG otherwise), and *count_dev (device)
 * receives the total number of triangles, which may exceed capacity.
 * Nothing is allocated; nothing waits. */
tsdf_status tsdf_extract_mesh_async(tsdf_volume* vol, float* triangles_dev, int32_t* cells_dev,
                                    uint32_t capacity, uint32_t* count_dev, void* stream);

/* Extract to host memory: triangles_host gets n x 9 floats, cells_host
 * n x 4 int32 (either may be NULL; both NULL or capacity 0 only counts).
 * *n_out is always n. If capacity < n nothing is copied and
 * TSDF_ERR_INVALID_ARG is returned. *timing (nullable) receives the kernel
 * and copy times. Allocates device scratch for the result; waits for
 * `stream`. */
tsdf_status tsdf_extract_mesh(tsdf_volume* vol, float* triangles_host, int32_t* cells_host,
                              uint32_t capacity, uint32_t* n_out, tsdf_extract_timing* timing,
                              void* stream);

/* Diagnostics of a volume's table and pool (a read-out, not part of fusion).
 * A key's probe length is its distance from its home slot plus one: the
 * number of entries an unbounded probe reads to find it (Section 3.1, linear
 * probing). weight_sum is the sum of every voxel weight, i.e. the number of
 * contributions the volume has received (weights are 1 per contribution). */
typedef struct tsdf_table_stats {
  uint64_t occupied_slots; /* entries holding a key */
  uint64_t probe_sum;      /* sum of the keys' probe lengths */
  uint32_t probe_max;      /* longest probe length (0 when empty) */
  uint32_t blocks;         /* min(claimed, pool_blocks), as tsdf_volume_block_count */
  uint64_t weight_sum;     /* sum of all voxel weights of the allocated blocks */
} tsdf_table_stats;

/* Fill *out for `vol`. Enqueues two kernels on `stream` and waits for it. */
tsdf_status tsdf_volume_table_stats(tsdf_volume* vol, void* stream, tsdf_table_stats* out);

/* Copy the whole state of `src` (header, table, coordinates, pool, poisoned
 * flag) into `dst`, device to device on `stream` (not waited for). Both must
 * have the same voxel size, truncation, table_slots, pool_blocks and
 * TSDF_OPT_SLOT_INDEX setting and live on the current device; options other
 * than the slot index are not copied. For snapshots and restores (e.g. timing
 * a fusion repeatedly from the same state). */
tsdf_status tsdf_volume_copy(tsdf_volume* dst, const tsdf_volume* src, void* stream);

/* Checkpoint and resume (not in the paper): a volume's whole state -- its
 * device allocation, laid out as at the top of this header, and the poisoned
 * flag -- in caller-owned host memory, behind a 64-byte header recording the
 * voxel size, truncation, table_slots, pool_blocks and TSDF_OPT_SLOT_INDEX
 * setting. tsdf_export_blocks returns means, which do not restore the sums
 * bit for bit; a checkpoint does.
 *
 * tsdf_volume_checkpoint_bytes: the bytes a checkpoint of `vol` takes,
 * 64 + tsdf_volume_bytes(table_slots, pool_blocks); 0 for NULL.
 *
 * tsdf_volume_save: write the checkpoint into `host` (at least that many
 * bytes). The copy is ordered after the work already on `stream` and waited
 * for, so `host` is complete on return. TSDF_ERR_INVALID_ARG for a NULL
 * pointer, a short buffer, or a device other than the volume's current.
 *
 * tsdf_volume_load: replace the state of `vol` with a checkpoint. It must
 * come from a volume with the same voxel size, truncation, table_slots,
 * pool_blocks and slot-index setting, and be complete (TSDF_ERR_INVALID_ARG
 * otherwise, also for a buffer that is not a checkpoint); nothing is changed
 * then. Options other than the slot index are the volume's own. The copy is
 * ordered on `stream` and waited for; `host` is only read during the call. */
size_t tsdf_volume_checkpoint_bytes(const tsdf_volume* vol);
tsdf_status tsdf_volume_save(const tsdf_volume* vol, void* host, size_t bytes, void* stream);
tsdf_status tsdf_volume_load(tsdf_volume* vol, const void* host, size_t bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Exact integer helpers (the device code uses the same definitions)
 * ------------------------------------------------------------------------- */

/* Packed 64-bit key of block (bx, by, bz), each in [-2^20, 2^20) (Section 2.1). */
uint64_t tsdf_block_key(int32_t bx, int32_t by, int32_t bz);

/* Home slot of a block: (bx*73856093 ^ by*19349669 ^ bz*83492791) mod 2^32,
 * masked to table_slots - 1 (multiply-xor hash of Section 3.1, constants of
 * Teschner et al. 2003). table_slots must be a power of two. */
uint32_t tsdf_block_slot(int32_t bx, int32_t by, int32_t bz, uint32_t table_slots);

const char* tsdf_status_string(tsdf_status s);

/* Library version, and the number of kernel launches this process has
 * enqueued through the library (for accounting in benchmarks). */
const char* tsdf_version(void);
uint64_t tsdf_launch_count(void);

/* Sets the largest number of bytes the L2 cache fetches from DRAM on a miss
 * (CUDA's cudaLimitMaxL2FetchGranularity: 0, 32, 64 or 128) for the CUDA
 * context of the current device, which this process shares with every other
 * library in it; *previous (may be NULL) receives the value it replaces.
 * Section 2.2's updates touch the five sums of scattered voxels: with 32, an
 * L2 miss fetches only its own 32-byte sector, so the pool is read at sector
 * granularity (no bytes fetched beside the touched sectors); the kernels'
 * results do not depend on it. The limit lasts as long as the context, and
 * is a hint the driver may round. Returns INVALID_ARG for other values,
 * CUDA on a failed call. Not in the paper. */
tsdf_status tsdf_set_l2_fetch_bytes(int bytes, int* previous);

#ifdef __cplusplus
}
#endif

#endif /* TSDF_H_ */
