/*
 * psweep.h — C ABI of the GB300 fisheye plane-sweep + TSDF fusion library
 * (libpsweep.so).
 *
 * The library computes the data-parallel hot path of "Real-Time Dense Mapping
 * for Self-Driving Vehicles using Fisheye Cameras" (Cui et al.):
 *   - multi-scale fisheye plane-sweep stereo with a windowed ZNCC cost
 *     (Sec. III-A: plane sweeping, fronto-parallel and ground-parallel plane
 *     sets, ZNCC matching cost, multi-scale strategy),
 *   - masking of dynamic-object boxes in the depth map (Sec. III overview,
 *     Sec. III-B),
 *   - TSDF fusion of fisheye depth maps into voxel blocks (Sec. III-C,
 *     Eq. 1 back-projection, Eq. 2 running average, local map).
 *
 * Conventions (all entry points):
 *   - Pixel centres sit at integer coordinates; images are row-major with
 *     u = column, v = row; the camera frame is x right, y down, z forward.
 *   - Intensities are uint8; the method works on I / 255.
 *   - Depth is the range along the pixel's unit viewing ray (|X|), float32,
 *     with 0 meaning "no depth".
 *   - A pose {R, t} maps source to destination coordinates,
 *     X_dst = R X_src + t, R row-major.
 *   - Pointers documented "device" must point to memory of the current CUDA
 *     device; "host" pointers are ordinary CPU memory.  The caller owns every
 *     buffer it passes; the library owns its handles' scratch memory, which
 *     is allocated only in *_create and freed only in *_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls documented "asynchronous" only enqueue work on it.
 *   - Every int-returning call returns a PS_* status.  On a non-zero status
 *     ps_last_error() gives a message for the calling thread.  Device-side
 *     failures (hash table or block pool full, bounded probe gave up) are
 *     latched in the handle and reported by the next synchronising call
 *     (ps_sync_status for any handle; tsdf_status, tsdf_extract,
 *     tsdf_count for a TSDF; psbatch_status for a batch).  No call traps
 *     the device.
 */
#ifndef PSWEEP_H
#define PSWEEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PS_OK 0
#define PS_ERR_ARG 1        /* invalid argument: null pointer, bad size, unsupported option */
#define PS_ERR_OOM 2        /* device or host allocation failed in *_create */
#define PS_ERR_CAPACITY 3   /* TSDF hash table or voxel-block pool is full */
#define PS_ERR_CUDA 4       /* a CUDA runtime call failed */
#define PS_ERR_TIMEOUT 5    /* a bounded device loop (hash probing) gave up */
#define PS_ERR_STATE 6      /* a device-side invariant failed: one handle's work counters were
                               advanced by overlapping calls (e.g. two streams at once) */

/* Unified omnidirectional camera (Sec. III-C, Eq. 1, after Mei) with
 * radial-tangential distortion of the normalised coordinates:
 *   x_d = x (1 + k1 r^2 + k2 r^4) + 2 p1 x y + p2 (r^2 + 2 x^2)
 *   y_d = y (1 + k1 r^2 + k2 r^4) + p1 (r^2 + 2 y^2) + 2 p2 x y,
 *   u = fx x_d + cx, v = fy y_d + cy.
 * r2_max bounds x^2 + y^2 of accepted undistorted coordinates (keeps the
 * polynomial one-to-one); a point projects only where its unit-sphere z
 * exceeds -min(xi, 1/xi). */
typedef struct {
    double xi, fx, fy, cx, cy, k1, k2, p1, p2, r2_max;
    int32_t width, height;
} ps_camera;

typedef struct {
    double R[9];
    double t[3];
} ps_pose;

#define PS_PLANES_FRONTO 0  /* n = (0,0,1); inverse depth uniform on [1/b, 1/a], index 0 farthest */
#define PS_PLANES_GROUND 1  /* n . X = h, h uniform on [a, b], index 0 at h = a; n = ground normal */

/* One set of sweep planes (Sec. III-A: one set parallel to the reference
 * image plane, one set parallel to the ground from the extrinsic
 * calibration). */
typedef struct {
    int32_t family;
    int32_t count;          /* >= 1 */
    double a, b;            /* fronto: near, far (m); ground: lowest, highest offset (m) */
    double n[3];            /* ground normal in the reference frame (normalised by the library) */
} ps_plane_set;

#define PS_LEVEL_DOWNSAMPLE 0  /* all images box-averaged by `factor` */
#define PS_LEVEL_CROP 1        /* centred crop_w x crop_h window of the reference at full
                                  resolution, matched against full-resolution matching images */
#define PS_MAX_SETS 4
#define PS_MAX_CAMS 4
#define PS_MAX_LEVELS 2

/* One resolution level of the multi-scale strategy (Sec. III-A). */
typedef struct {
    int32_t kind;
    int32_t factor;         /* DOWNSAMPLE: 1, 2 or 4 (image sizes must divide) */
    int32_t crop_w, crop_h; /* CROP: window size; offset ((W - crop_w)/2, (H - crop_h)/2) */
    int32_t window;         /* side of the square ZNCC window: 5, 7 or 9 */
    int32_t n_sets;         /* 1 .. PS_MAX_SETS */
    ps_plane_set sets[PS_MAX_SETS];
} ps_level;

/* Depth map filtering (Sec. III-A, "Depth map filtering"), all zero = off.
 * Per level, a pixel is an outlier when its best cost exceeds alpha of its
 * image part (alpha_upper for pixels whose centre lies above the
 * full-resolution row split_row, alpha_lower below; split_row < 0 means half
 * the height; the paper uses 0.05 and 0.3) or when its second-best cost is
 * below ratio_min times the best (the paper's uniqueness ratio; it gives no
 * value).  After merging, a pixel keeps its depth only if at least a
 * fraction delta of the other pixels of its window x window neighbourhood
 * inside the image have a depth within gamma of it (the paper: gamma 0.5 m,
 * delta 0.3).  The boxes are applied last. */
typedef struct {
    int32_t enable;
    int32_t window;         /* odd, 1 .. 15 */
    double alpha_upper, alpha_lower;
    double split_row;
    double ratio_min;
    double gamma, delta;
} ps_filter;

typedef struct {
    ps_camera ref;                 /* reference camera at full resolution */
    int32_t n_cams;                /* matching cameras, 1 .. PS_MAX_CAMS */
    const ps_camera* cams;         /* host, n_cams entries */
    const ps_pose* ref_to_cam;     /* host, n_cams entries: X_cam = R X_ref + t */
    int32_t n_levels;              /* 1 .. PS_MAX_LEVELS: at most one DOWNSAMPLE and one CROP */
    const ps_level* levels;        /* host */
    ps_filter filter;              /* depth map filtering; zero-initialised = off */
    int32_t image_half;            /* 1: matching images stored as FP16 (arithmetic stays FP32) */
} ps_sweep_desc;

/* Half-open pixel rectangle [x0, x1) x [y0, y1) in full-resolution
 * reference pixels: a dynamic-object detection (Sec. III-B). */
typedef struct {
    int32_t x0, y0, x1, y1;
} ps_box;

/* Optional per-level outputs, each a device array of the level's size
 * (DOWNSAMPLE: (H/factor) x (W/factor); CROP: crop_h x crop_w), any may be
 * NULL.  best_cost / second_cost: lowest and second-lowest aggregated cost
 * over the planes (+inf where none); plane_idx: winning plane (-1 = none);
 * depth: the level's range map before merging. */
typedef struct {
    float* depth;
    float* best_cost;
    float* second_cost;
    int32_t* plane_idx;
} ps_level_out;

typedef struct psweep_s psweep_t;
typedef struct tsdf_s tsdf_t;

/* Validate the rig and levels, build the per-level ray tables (Eq. 1 per
 * reference pixel), plane tables and scratch images.  The only sweep call
 * that allocates.  On success *out receives the handle; on failure *out is
 * NULL and the status says why (PS_ERR_ARG, PS_ERR_OOM, PS_ERR_CUDA). */
int psweep_create(const ps_sweep_desc* desc, psweep_t** out);

/* Depth map of the reference camera for one synchronised frame (Sec. III-A):
 * per level, warp each matching image through every plane, ZNCC cost over
 * the window, minimum over matching cameras, winner-take-all with parabolic
 * sub-plane refinement; then, when the descriptor enables it, the per-level
 * cost filters; merge the levels at full resolution (crop depth where valid,
 * else the downsampled level's depth at (u/factor, v/factor)); the
 * continuity filter; and zero the pixels inside the boxes.
 *   images    host array of 1 + n_cams device pointers: [0] reference, then
 *             the matching cameras, each a contiguous uint8 H x W image of
 *             its camera's full-resolution size.
 *   boxes     host array of n_boxes boxes (may be NULL when n_boxes == 0).
 *   depth_out device float32 H x W (reference full resolution).
 *   level_out host array of n_levels entries or NULL.
 * Asynchronous on `stream`; allocates nothing. */
int psweep_depth(psweep_t* h, const uint8_t* const* images, const ps_box* boxes, int32_t n_boxes,
                 float* depth_out, const ps_level_out* level_out, void* stream);

void psweep_destroy(psweep_t* h);

/* Copy the handle's own level outputs (depth, best and second-best cost,
 * plane index per level pixel, as the last psweep_depth call without
 * level_out or the last batch run over this handle left them) into the
 * caller's buffers (level_out: host array of n_levels entries; NULL members
 * are skipped).  Asynchronous on `stream`; allocates nothing. */
int psweep_level_outputs(psweep_t* h, const ps_level_out* level_out, void* stream);

/* ---------------------------------------------------------------------
 * Plane-sharded sweep.  The plane hypotheses of a level are independent
 * until the winner-take-all (Sec. III-A: every plane's warped images and
 * costs stand alone; the depth is the plane of least cost), so one frame's
 * sweep splits into consecutive plane ranges swept on different GPUs, each
 * reducing its range to a per-pixel record; one exchange of the records
 * (an all-gather of 7 floats per pixel per level) and psweep_merge_records
 * on every GPU give exactly psweep_depth's outputs.  The paper pipelines
 * the stages of its system over three computers (Sec. IV-A); this is the
 * data-parallel split of the sweep stage itself.
 *
 * Sweep planes [plane_lo[l], plane_hi[l]) of each level l (host int32
 * arrays of n_levels entries; an empty range is allowed) and write each
 * pixel's record of that range:
 *   records  host array of n_levels device pointers, each 7 x H_l x W_l
 *            float32 planes: best cost, second best, the best plane's
 *            neighbour costs inside the range (+inf at its ends), the
 *            range's first and last plane cost, the best plane's index as
 *            int32 bits (-1 = none).
 * Asynchronous on `stream`; allocates nothing. */
#define PS_MAX_PARTS 16
int psweep_depth_planes(psweep_t* h, const uint8_t* const* images, const int32_t* plane_lo,
                        const int32_t* plane_hi, float* const* records, void* stream);

/* Merge the records of n_parts consecutive plane ranges (part p of level l
 * starts at plane part_lo[p * n_levels + l]; part 0 at plane 0, the last
 * part ends at the level's plane count; starts never fall) into each
 * level's winner-take-all with the sub-plane fit, then merge the levels,
 * filter and mask exactly as psweep_depth does.  records: host array of
 * n_parts * n_levels device pointers in the same order (NULL allowed for
 * empty parts).  The outputs are bit-identical to psweep_depth on the same
 * images.  Asynchronous on `stream`; allocates nothing. */
int psweep_merge_records(psweep_t* h, int32_t n_parts, const int32_t* part_lo, const float* const* records,
                         const ps_box* boxes, int32_t n_boxes, float* depth_out, const ps_level_out* level_out,
                         void* stream);

/* TSDF volume (Sec. III-C).  Voxels hold {D, w}: D in [-1, 1] is the
 * truncated signed distance normalised by mu (positive in front of
 * surfaces), w the number of fused observations capped at w_max.
 * Blocks are 8^3 voxels.  dense_dim != 0 gives a fixed grid of
 * dense_dim[0] x dense_dim[1] x dense_dim[2] voxels (multiples of 8) at
 * `origin`; otherwise blocks are allocated on demand in a hash table of
 * hash_slots (power of two) slots backed by a pool of pool_blocks blocks,
 * keyed by block index floor((X - origin) / (8 voxel_size)).  local_half
 * != 0 restricts allocation to blocks whose centre lies within
 * local_half of the local-map centre passed to tsdf_integrate. */
typedef struct {
    ps_camera cam;            /* camera of the fused depth maps (full resolution) */
    double voxel_size;
    double mu;
    double w_max;
    int32_t block_dim;        /* must be 8 */
    int32_t dense_dim[3];
    double origin[3];
    double local_half[3];
    int64_t hash_slots;
    int64_t pool_blocks;
} ps_tsdf_desc;

/* Allocates the voxel pool (zeroed), hash table and per-frame scratch and
 * builds the depth camera's ray table (Eq. 1 per pixel). */
int tsdf_create(const ps_tsdf_desc* desc, tsdf_t** out);

/* Fuse one depth map (Sec. III-C): allocate the blocks crossed by the
 * segment [d - mu, d + mu] (starting no closer than the camera centre)
 * along every valid pixel's ray, inside the local map; list the allocated
 * blocks a pixel of this frame can update; apply Eq. 2 to their voxels:
 * with eta = d(nearest pixel of the voxel's projection) - |X_d|, voxels with
 * eta >= -mu get D <- (w D + min(1, eta/mu)) / (w + 1), w <- min(w + 1, w_max).
 *   depth         device float32 H x W range map of the desc's camera (0 = no depth).
 *   world_to_cam  host, pose of the camera for this frame.
 *   local_center  host double[3] or NULL (required when local_half != 0).
 * Asynchronous on `stream`; allocates nothing.  A full hash table or pool
 * is latched (PS_ERR_CAPACITY) and the affected blocks are skipped. */
int tsdf_integrate(tsdf_t* t, const float* depth, const ps_pose* world_to_cam, const double* local_center,
                   void* stream);

/* Synchronises `stream`; *n_blocks = number of allocated blocks.  Returns
 * the latched device status (then clears it). */
int tsdf_count(tsdf_t* t, int64_t* n_blocks, void* stream);

/* Synchronises `stream`; *n_blocks = number of blocks on the visible-block
 * list of the last tsdf_integrate call (the blocks whose voxels Eq. 2 was
 * applied to, Sec. III-C), 0 before the first call.  For measurement: the
 * integration stage reads and writes 16 bytes per voxel of these blocks.
 * Returns PS_OK or PS_ERR_ARG (NULL argument); the latched status is left
 * for tsdf_count / tsdf_status. */
int tsdf_listed(tsdf_t* t, int64_t* n_blocks, void* stream);

/* Synchronises `stream` and copies out every allocated block, in pool-slot
 * order (for a dense grid: block bx + nbx (by + nby bz)): keys (device int32, capacity x 3 block indices), D and W (device
 * float32, capacity x 512 voxels each, voxel index x + 8 y + 64 z).
 * Voxels with w < min_weight are reported with W = 0 and D = 0 (Sec. III-C:
 * only voxels with at least 3 observations are kept; pass 0 for all).
 * *n_out = number of blocks written (min(count, capacity)).  Returns the
 * latched device status, or PS_ERR_CAPACITY if capacity < count. */
int tsdf_extract(tsdf_t* t, float min_weight, int32_t* keys, float* D, float* W, int64_t capacity,
                 int64_t* n_out, void* stream);

/* Synchronises `stream`, returns and clears the latched device status. */
int tsdf_status(tsdf_t* t, void* stream);

/* Ownership of the map by hash partition, for fusing one sequence on
 * n_parts GPUs (Sec. III-C: every voxel block is updated only from the
 * depth map and its own state, so disjoint block sets fuse independently):
 * from the next tsdf_integrate on, this map allocates only the blocks whose
 * key hashes to `part` (high half of a 64-bit mix of the key, modulo
 * n_parts); every GPU fuses the same broadcast depth map into its own
 * part, and the union of the parts equals the map one GPU would build,
 * voxel for voxel.  n_parts = 1 restores the whole map.  Hashed maps only
 * (a dense grid gets PS_ERR_ARG).  Blocks already allocated stay. */
int tsdf_set_partition(tsdf_t* t, int32_t n_parts, int32_t part);

/* Surface points of the map (Sec. III-C; the paper evaluates the map as a
 * point set): for every voxel a and its +x, +y and +z neighbour b (in the
 * same block or the next block along that axis) that both have at least
 * max(min_weight, 1) observations and whose D change sign (positive against
 * zero or negative), the point X_a + t (X_b - X_a) with t = D_a / (D_a - D_b),
 * X = origin + (i + 1/2) voxel_size, in world coordinates.
 *   points  device float32 capacity x 3.
 *   edges   device int32 capacity x 4 (global voxel index of a, axis) or NULL.
 * Unspecified order.  *n_out = points found; if that exceeds capacity only
 * the first `capacity` are written and the call returns PS_ERR_CAPACITY
 * (capacity 0 counts them).  Synchronises `stream`. */
int tsdf_extract_points(tsdf_t* t, float min_weight, float* points, int32_t* edges, int64_t capacity,
                        int64_t* n_out, void* stream);

/* Local-map swap-out (Sec. III-C: blocks that are no longer in the local map
 * are swapped out of GPU memory).  Every allocated block whose centre lies
 * outside the local-map box around local_center (half extents local_half of
 * the descriptor) is copied to the caller's buffers (device; keys capacity x 3,
 * D and W capacity x 512, in an unspecified order), removed from the hash
 * table, and its pool slot freed for reuse by later allocations.  At most
 * `capacity` blocks leave per call; if more lie outside, the rest stay and the
 * call returns PS_ERR_CAPACITY.  *n_out = blocks written.  Hashed maps with a
 * local map only.  Synchronises `stream`. */
int tsdf_swap_out(tsdf_t* t, const double* local_center, int32_t* keys, float* D, float* W, int64_t capacity,
                  int64_t* n_out, void* stream);

/* Insert or overwrite n blocks (device keys n x 3, D and W n x 512, the layout
 * tsdf_extract and tsdf_swap_out produce): checkpoint resume and swap-in.
 * Hashed maps only.  Asynchronous on `stream`; a full pool is latched
 * (PS_ERR_CAPACITY) and the blocks that found no slot are skipped. */
int tsdf_load(tsdf_t* t, const int32_t* keys, const float* D, const float* W, int64_t n, void* stream);

void tsdf_destroy(tsdf_t* t);

/* One frame end to end from host memory: copy the 1 + n_cams host images
 * (uint8, pinned memory gives asynchronous copies) to library-owned device
 * buffers, run psweep_depth, fuse the depth map with tsdf_integrate (t may
 * be NULL to skip fusion; its camera must be the reference camera) at pose
 * world_to_ref, and
 * copy the full-resolution depth map back to host_depth_out (float32 H x W,
 * may be NULL).  Synchronises `stream` before returning. */
int psweep_frame_host(psweep_t* h, tsdf_t* t, const uint8_t* const* host_images, const ps_box* boxes,
                      int32_t n_boxes, const ps_pose* world_to_ref, const double* local_center,
                      float* host_depth_out, void* stream);

/* Frame pipeline.  The paper ran depth estimation and fusion on separate
 * computers at the same time, each on a different frame (Sec. IV-A).  On
 * one GPU the sweep fills every SM, so the overlap comes from the copies:
 * frames from host memory go through a copy-in stream (host images ->
 * pinned staging -> device), a compute stream (psweep_depth, then
 * tsdf_integrate) and a copy-out stream (the depth map back to pinned
 * staging), with two frames in flight, so the copies and the host-side
 * staging of the neighbouring frames overlap the GPU work of the current
 * one.  Every frame gets exactly what psweep_frame_host gives it.
 *   ps_pipe_create  t may be NULL (no fusion); allocates two sets of device
 *                   and pinned staging buffers, three streams, six events.
 *   ps_pipe_push    enqueues one frame (arguments as psweep_frame_host) and
 *                   returns; it first waits for the frame pushed two calls
 *                   earlier, whose depth map is then copied to that call's
 *                   host_depth_out (host float32 H x W, may be NULL).  The
 *                   host images may be reused when the call returns.
 *   ps_pipe_flush   waits for every pushed frame and delivers its depth map.
 * While frames are in flight, do not use the pipeline's sweep or TSDF
 * handle elsewhere; flush first. */
typedef struct ps_pipe_s ps_pipe_t;
int ps_pipe_create(psweep_t* h, tsdf_t* t, ps_pipe_t** out);
int ps_pipe_push(ps_pipe_t* p, const uint8_t* const* host_images, const ps_box* boxes, int32_t n_boxes,
                 const ps_pose* world_to_ref, const double* local_center, float* host_depth_out);
int ps_pipe_flush(ps_pipe_t* p);
void ps_pipe_destroy(ps_pipe_t* p);

/* Stage timing for measurement tools.  psweep_profile(h, capacity) with
 * capacity > 0 creates 2 x stages x capacity CUDA events (this allocates:
 * call it outside timed or captured regions) and makes the next `capacity`
 * psweep_depth calls record events around their stages on their stream:
 * stage 0 level preparation (downsampling, quad images), stage 1 the sweep
 * kernel, stage 2 the merge.  capacity 0 turns recording off and frees the
 * events.  psweep_profile_read synchronises those events and returns the
 * summed milliseconds per stage (host double[3]) and the number of calls
 * recorded, then restarts the count.  tsdf_profile / tsdf_profile_read do
 * the same for tsdf_integrate with 4 stages: 0 depth maximum, 1 block
 * allocation, 2 visible-block list, 3 integration. */
int psweep_profile(psweep_t* h, int32_t capacity);
int psweep_profile_read(psweep_t* h, double* stage_ms, int32_t* n_calls);
int tsdf_profile(tsdf_t* t, int32_t capacity);
int tsdf_profile_read(tsdf_t* t, double* stage_ms, int32_t* n_calls);

/* Allocation-free fusion into a caller-owned dense grid (the paper has no
 * counterpart; this is a convenience of the library).  Some callers cannot
 * allocate GPU memory while they run: real-time loops whose memory is
 * planned once up front (an allocation there can stall or fail at an
 * unplanned moment), and hosts whose device memory belongs to another
 * allocator (memory taken behind its back is memory it cannot account
 * for).  This call fuses one depth map exactly like tsdf_integrate on
 * a dense grid, but the voxels are the caller's and the library's working
 * memory (block list, counters, depth maximum) is one fixed static device
 * array of PS_STATIC_SCRATCH_BYTES (about 1.3 MB), which every GPU that
 * loads the library keeps until the process exits.  No memory is allocated.
 *   voxels        device float32: n_blocks x 512 {D, w} pairs; block
 *                 b = bx + nbx (by + nby bz) of the grid, voxel x + 8 y + 64 z
 *                 inside a block (the order tsdf_extract reports for a dense
 *                 map).  Zero it to start an empty map.
 *   dims          host int32[3]: voxels per axis, multiples of 8, at most
 *                 PS_STATIC_MAX_BLOCKS blocks in all (larger grids get
 *                 PS_ERR_ARG and a message naming the limit).  The library
 *                 sees only pointers: voxels must hold dims' blocks and
 *                 depth cam's H x W values (the Python binding checks both).
 *   origin        host double[3]; voxel_size, mu, w_max as in ps_tsdf_desc.
 *   depth         device float32 H x W range map of cam (0 = no depth).
 *   cam           host, the depth map's camera; world_to_cam host pose.
 * Asynchronous on `stream`; a device-side failure has no handle to be
 * latched in, and none can occur on a dense grid (argument errors are
 * returned at once).  The first call on each device looks up the static
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call
 * reuses the same array (it keeps the last call's contents; the call clears
 * what must start at zero), so calls that overlap on the GPU, from other
 * streams or host threads, race on it: serialise them. */
#define PS_STATIC_MAX_BLOCKS 65536
#define PS_STATIC_SCRATCH_BYTES (256 + PS_STATIC_MAX_BLOCKS * 20)
int tsdf_integrate_dense_static(float* voxels, const int32_t* dims, const double* origin, double voxel_size,
                                double mu, double w_max, const float* depth, const ps_camera* cam,
                                const ps_pose* world_to_cam, void* stream);

/* ---------------------------------------------------------------------
 * Batched sweeps.  The paper computes one depth map per synchronised frame
 * of one rig; a batch computes the depth maps of many sweep handles (other
 * rigs, image sizes, plane counts, camera counts, levels and filters) with
 * the same results as psweep_depth on each, in ONE persistent kernel
 * launch.  Every step of psweep_depth (level images, reference statistics,
 * the sweep's tile x plane-chunk work items, merge, filters, boxes) is a
 * work item of that kernel, taken from a device queue built at
 * psbatch_create.  An item that needs other items' results waits for them
 * on the GPU with a bounded spin; the queue order puts every item after
 * the items it needs, so the waits end, and a wait longer than its limit
 * (wait_limit_ms) gives up, skips the rest of the batch and is reported as
 * PS_ERR_TIMEOUT by psbatch_status.  With use_graph the per-run launch sequence (one
 * copy of the run's pointers and boxes, two memsets, the kernel) is
 * captured into a CUDA graph on the first run and replayed afterwards.
 *
 * A batch uses the level buffers of its sweep handles: while a batch may
 * run, do not run psweep_depth on its handles concurrently, and destroy the
 * batch before its handles.  Every handle may appear once. */
typedef struct psbatch_s psbatch_t;

#define PS_BATCH_SHORTEST_FIRST 0 /* queue sweeps by ascending work: lowest mean latency */
#define PS_BATCH_GIVEN_ORDER 1    /* queue sweeps in the order given */

typedef struct {
    int32_t tile_h;       /* output rows per tile: 16 or 24 (0 = 24); tiles are 64 columns wide */
    int32_t kp;           /* planes warped per camera before their window sums: 1 or 2 (0 = 2) */
    int32_t plane_chunk;  /* most planes per sweep work item, 1..4096 (0 = 32) */
    int32_t order;        /* PS_BATCH_SHORTEST_FIRST or PS_BATCH_GIVEN_ORDER */
    int32_t use_graph;    /* non-zero: replay the run as a CUDA graph (needs a non-NULL stream) */
    int32_t grid;         /* persistent CTAs (0 = one per SM; at most one per SM) */
    int32_t wait_limit_ms;     /* time limit of one dependency wait, 1..60000 (0 = 2000) */
    int32_t drill_unmet_wait;  /* failure drill, for tests of the error path only: non-zero makes
                                  every merge item wait for one tile more than its sweep has, so
                                  that the first such wait runs out after wait_limit_ms, the rest
                                  of the batch is skipped and psbatch_status reports
                                  PS_ERR_TIMEOUT with the context still usable */
} ps_batch_opts;

/* Build the queue and device tables for sweeps[0 .. n) (host array of
 * handles, 1 <= n <= 4096).  opts may be NULL (defaults).  Allocates; the
 * only batch call that does. */
int psbatch_create(psweep_t* const* sweeps, int32_t n, const ps_batch_opts* opts, psbatch_t** out);

/* Depth maps of every sweep of the batch, each as psweep_depth would give it.
 *   images     host array: for each sweep in turn, 1 + n_cams device image
 *              pointers as for psweep_depth (concatenated).
 *   boxes      host array of every sweep's boxes, concatenated (may be NULL
 *              when no sweep has boxes); n_boxes host int32[n] (NULL = none),
 *              each at most 256.
 *   depth_out  host array of n device float32 maps (H x W of each sweep's
 *              reference camera).
 * Asynchronous on `stream`; serialise runs of one batch on one stream.
 * Allocates nothing (the first graph run instantiates the graph). */
int psbatch_run(psbatch_t* b, const uint8_t* const* images, const ps_box* boxes, const int32_t* n_boxes,
                float* const* depth_out, void* stream);

/* Synchronises with the last run and reads its device clock stamps:
 * done_ms host double[n] (may be NULL): time from the start of the kernel to
 * the completion of each sweep's depth map; *span_ms (may be NULL): the
 * same for the last sweep.  PS_ERR_TIMEOUT if the run gave up. */
int psbatch_timing(psbatch_t* b, double* done_ms, double* span_ms);

/* Synchronises with the last run: PS_OK or PS_ERR_TIMEOUT. */
int psbatch_status(psbatch_t* b);

/* Work items of the batch's queue by kind (host int32[6]: reference rows,
 * quad rows, statistics rows, sweep items, merge rows, continuity rows). */
int psbatch_queue_stats(psbatch_t* b, int32_t* counts);

void psbatch_destroy(psbatch_t* b);

/* Autotuner: for each of n_cand candidate options, build a batch of the
 * given sweeps, run it once untimed and `reps` times timed (CUDA events on
 * `stream`, a synchronise around each), and write the median milliseconds to
 * ms_out[i] (host double[n_cand]).  *best receives the index of the fastest
 * candidate.  The inputs are those of psbatch_run; depth_out is written.
 * Allocates and synchronises: call it outside timed regions. */
int psbatch_autotune(psweep_t* const* sweeps, int32_t n, const uint8_t* const* images, const ps_box* boxes,
                     const int32_t* n_boxes, float* const* depth_out, const ps_batch_opts* candidates,
                     int32_t n_cand, int32_t reps, int32_t* best, double* ms_out, void* stream);

/* ---------------------------------------------------------------------
 * Differentiable forms (the paper has none: its winner-take-all depth and
 * its fusion are used forward only; these make the sweep and the fusion
 * usable inside gradient-based calibration or learning).
 *
 * Soft-argmin depth over the plane hypotheses of one full-resolution level
 * (Sec. III-A costs on real-valued images):
 *   C_k   = min over matching cameras of (1 - ZNCC) / 2 (lowest camera index
 *           on a tie; invalid windows as in psweep_depth)
 *   s_k   = exp(-C_k / T) / sum over valid k' of exp(-C_k' / T)
 *   range = 1 / sum_k s_k rho_k,  rho_k = (n_k . r) / d_k, the inverse range
 *           of plane k along the pixel's unit ray r (Eq. 1)
 *   cost  = -T log sum over valid k of exp(-C_k / T)   (soft minimum)
 * Both are 0 where no plane is valid.  psdiff_backward gives the gradient of
 * L = sum g_range * range + g_cost * cost with respect to every image and
 * to a left perturbation (w, v) of each ref_to_cam pose:
 * T_j <- exp([w]x, v) T_j, i.e. X_j <- X_j + w x X_j + v to first order. */
typedef struct psdiff_s psdiff_t;

typedef struct {
    ps_camera ref;
    int32_t n_cams;          /* 1 .. PS_MAX_CAMS */
    const ps_camera* cams;   /* host array of n_cams */
    ps_level level;          /* kind PS_LEVEL_DOWNSAMPLE, factor 1; window 5, 7 or 9 */
    double temperature;      /* T > 0 */
} ps_diff_desc;

/* Builds the reference ray table (Eq. 1) and the plane table; allocates. */
int psdiff_create(const ps_diff_desc* desc, psdiff_t** out);

/* images: host array of 1 + n_cams device float32 images (reference first,
 * each H x W of its camera), real-valued intensities.  ref_to_cam: host
 * array of n_cams poses (per call: they may be the variables of an
 * optimisation).  range, cost (may be NULL): device float32 H x W.  aux:
 * device float32 H x W x 3 that psdiff_backward needs (may be NULL when no
 * backward follows).  Asynchronous on `stream`. */
int psdiff_forward(psdiff_t* h, const float* const* images, const ps_pose* ref_to_cam, float* range, float* cost,
                   float* aux, void* stream);

/* Same images and poses as the forward whose aux is passed.  g_range,
 * g_cost: device float32 H x W (either may be NULL).  g_images: host array
 * of 1 + n_cams device float32 buffers shaped like the images (entries may
 * be NULL), ADDED to.  g_pose: device double[6 n_cams], (w, v) per camera,
 * ADDED to (may be NULL).  Asynchronous; the costs are recomputed per tile,
 * nothing of the forward but aux is kept. */
int psdiff_backward(psdiff_t* h, const float* const* images, const ps_pose* ref_to_cam, const float* aux,
                    const float* g_range, const float* g_cost, float* const* g_images, double* g_pose,
                    void* stream);

void psdiff_destroy(psdiff_t* h);

/* Gradient of one fusion step into a caller-owned dense grid (the step
 * tsdf_integrate_dense_static performs; Eq. 2 with unit observation
 * weight): voxels_in is the grid BEFORE the step (same layout), g_D_out the
 * gradient with respect to the D of every voxel after it (float32 per
 * voxel; weights are counts and carry none).  Writes g_D_in (float32 per
 * voxel, may be NULL); ADDS to g_depth (device float32 H x W of cam, may be
 * NULL) and g_pose (device double[6], a left perturbation (w, v) of
 * world_to_cam, may be NULL).  An observed voxel (eta >= -mu) passes
 * w / (w + 1) of its gradient to D_in; if eta < mu also 1 / (mu (w + 1)) to
 * its pixel's depth and minus that along X_c / |X_c| to the camera-frame
 * point.  Asynchronous on `stream`; allocates nothing. */
int tsdf_dense_fuse_backward(const float* voxels_in, const int32_t* dims, const double* origin, double voxel_size,
                             double mu, double w_max, const float* depth, const ps_camera* cam,
                             const ps_pose* world_to_cam, const float* g_D_out, float* g_D_in, float* g_depth,
                             double* g_pose, void* stream);

/* Checked build (libpsweep_check.so, compiled with -DPS_CHECK; there is no
 * sanitizer on every machine this runs on): the kernels test the accesses
 * whose addresses come from data (image gathers at projected coordinates,
 * pixel indices, voxel-block pool slots from the hash table, work items of
 * the persistent queues), skip a failing access and record a bit:
 * 1 gather outside the image, 2 pixel outside the image, 4 pool slot outside
 * the pool, 8 work item outside its level or queue.  ps_check_read
 * synchronises the device and returns (and clears) the bits recorded since
 * the last read; in the normal build it always returns 0 bits, and
 * ps_version says which build is loaded. */
int ps_check_read(uint32_t* bits);

/* Message for the calling thread's last non-zero status ("" if none). */
const char* ps_last_error(void);

/* Synchronises `stream` and returns the device status latched in a handle
 * since the last read (then clears it), for any handle the library made:
 * psweep_t (a plane-chunk completion counted more often than the tile has
 * chunks: PS_ERR_STATE, which overlapping calls on one handle cause),
 * tsdf_t (full hash table or pool: PS_ERR_CAPACITY; probing gave up:
 * PS_ERR_TIMEOUT) or psbatch_t (a wait gave up: PS_ERR_TIMEOUT;
 * PS_ERR_STATE as for a sweep).  The handle's type is read from its first
 * word; a pointer that is no live handle of this library is undefined
 * behaviour (PS_ERR_ARG when the word does not match a handle type).
 * Paper: Sec. III (the per-frame pipeline needs each stage's outcome). */
int ps_sync_status(void* handle, void* stream);

/* Library version string. */
const char* ps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PSWEEP_H */
