/*
 * pat_bp.h -- C ABI of the GB300 fast-marching back-projection library.
 *
 * Method (Wang & Jing, "A fast marching method based back projection algorithm
 * for photoacoustic tomography in heterogeneous media"):
 *   - Sec. II-B: travel times T_s(r) from every sensor s to every pixel r solve
 *     the eikonal equation |grad T|^2 = 1/c^2 by fast marching, run once per
 *     speed map with the sensor as the point source (ray paths are reversible).
 *   - Sec. II-C, Eq. (BP): every pixel sums over the sensors the integrand
 *     b_s(t) = 2 p_s(t) - 2 t dp_s/dt sampled at t = T_s(r), weighted by w_s.
 *   - Sec. III: the travel-time table is computed off line once; the per-frame
 *     ("on-line") work is the back projection only.
 *
 * Conventions shared by every entry point:
 *   - No exception crosses the ABI; every call returns a pat_status.  CUDA
 *     errors map to PAT_ERR_CUDA; a device-side wait that ran out of time maps
 *     to PAT_ERR_TIMEOUT when the status is read (pat_bp_sync).
 *   - "host" pointers are ordinary CPU memory, "dev" pointers are device
 *     memory of the current CUDA device.  The library copies every host input
 *     it keeps; it never frees caller memory.
 *   - Grid nodes: node (i, j, k) sits at origin + (i, j, k) * dx (metres), x
 *     fastest in every array; 2-D grids use n[2] = 1.
 *   - Signals are [F][N_s][N_t] row-major; sample k of every row is at t = k dt
 *     (t = 0 is the laser pulse, the initial condition of Sec. II-A).
 */
#ifndef PAT_BP_H
#define PAT_BP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PAT_OK = 0,
  PAT_ERR_INVALID = 1,   /* bad argument (sizes, pointers, geometry)          */
  PAT_ERR_OOM = 2,       /* device or host allocation failed                 */
  PAT_ERR_CUDA = 3,      /* a CUDA runtime call failed                       */
  PAT_ERR_TIMEOUT = 4,   /* a bounded device or host wait ran out            */
  PAT_ERR_BUSY = 5,      /* admission refused for now (serving)              */
  PAT_ERR_NOT_FOUND = 6, /* unknown ticket / subject (serving)               */
  PAT_PENDING = 7        /* request still in flight (serving)                */
} pat_status;

typedef enum { PAT_F32 = 0, PAT_BF16 = 1, PAT_F16 = 2 } pat_dtype;

typedef struct {
  int ndim;          /* 2 or 3                                               */
  int n[3];          /* nodes along x, y, z (n[2] = 1 when ndim == 2)         */
  double dx;         /* node spacing (m), > 0                                 */
  double origin[3];  /* position of node (0,0,0) (m)                          */
} pat_grid;

typedef struct pat_bp_s* pat_bp_t;
typedef void* pat_stream_t; /* a cudaStream_t; NULL = legacy default stream */

/* Flags of pat_bp_create. */
#define PAT_FLAG_COMPACT_OUT 0x1u /* out is [F][N_pix] in raster order of the mask
                                     instead of the dense [F][grid] image        */
#define PAT_FLAG_TILE_128 0x10u   /* force 128 pixels per tile                   */
#define PAT_FLAG_TILE_256 0x20u   /* force 256 pixels per tile                   */
#define PAT_FLAG_HOST_MIRROR 0x100u /* keep a pinned host copy of the table so the
                                       device copy can be evicted and restored    */
#define PAT_FLAG_FMM_SECOND_ORDER 0x400u /* build the table with the printed
                                            second-order stencil of Sec. II-B
                                            (one-sided difference (3T_i - 4T_{i-1}
                                            + T_{i-2}) / 2h where the two upwind
                                            nodes are accepted and monotone)     */
#define PAT_FLAG_GPU_TABLE 0x800u /* solve the arrival times of the table on the
                                    current CUDA device (first-order scheme:
                                    block-iterative fixed point of the same
                                    Godunov update, equal bit for bit to the
                                    host march, so the table is the same);
                                    not with PAT_FLAG_FMM_SECOND_ORDER        */
#define PAT_FLAG_STAGED_SINGLE 0x200u /* single frames through the staged (TMA
                                         pipeline) gather too; by default one
                                         frame takes the unstaged kernel, which
                                         gives the same bits                     */
#define PAT_FLAG_NO_WINDOW 0x1000u /* unstaged single frames of a stored table
                                      gather the integrand from L2 instead of
                                      from shared-memory windows (the default
                                      whenever every window of the table has at
                                      most 288 samples); same bits, for
                                      comparisons                               */

/* Read-only facts about a handle (pat_bp_info). */
typedef struct {
  int64_t n_pix;        /* reconstructed (mask) pixels                        */
  int64_t grid_total;   /* nodes of the dense grid                            */
  int n_sensors, n_samples, n_samples_pad;
  int tile_pix;         /* P: pixels per tile                                 */
  int n_tiles;
  int window;           /* W: samples of one sensor a tile can touch          */
  int split;            /* sensor segments per tile (64 sensors each)         */
  int sensor_warps;     /* warps that share a tile's sensors inside one CTA   */
  int64_t table_bytes;  /* device bytes of the delay data: the travel-time
                           table, or the anchors and pixel terms (constant c)  */
  double build_seconds; /* wall time of the table (or anchor) build           */
  int delays;           /* 0 fast-marching table, 1 constant speed            */
  double c0;            /* the constant speed (m/s) when delays == 1, else 0  */
  int solid_angle;      /* 1 after pat_bp_set_solid_angle (exact BP weights)  */
  int gpu_table;        /* 1 if the table's times were solved on the GPU      */
} pat_bp_info_t;

const char* pat_status_str(pat_status s);

/* Message of the last failed call on this host thread ("" if none). */
const char* pat_last_error(void);

/* pat_bp_create -- the off-line step of Sec. III: fast-marching travel times
 * (Sec. II-B, first-order Godunov upwind update, one FP64 run per sensor on
 * the host, all host cores), stored on the device as FP32 sample offsets
 * u = T/dt - base from an int32 base per (pixel tile, sensor).
 *   speed_host    [n_z][n_y][n_x] sound speed (m/s) at the nodes, all > 0
 *   grid          geometry of speed_host (and of the dense output)
 *   sensors_host  [n_sensors][3] positions (m); each inside the grid box
 *   mask_host     [grid] nonzero = reconstruct that pixel; NULL = all nodes
 *   weights_host  [n_sensors] w_s of Eq. (BP); NULL = 1/n_sensors each
 *   dt, n_samples sample interval (s, > 0) and samples per signal (2..32768)
 *   flags         PAT_FLAG_* (0 = defaults)
 *   out           receives the handle (owns all device memory it allocates)
 * Uses the current CUDA device.  Blocking.  Errors: PAT_ERR_INVALID for bad
 * geometry, PAT_ERR_OOM, PAT_ERR_CUDA. */
pat_status pat_bp_create(const float* speed_host, const pat_grid* grid,
                         const double* sensors_host, int n_sensors,
                         const uint8_t* mask_host, const float* weights_host,
                         double dt, int n_samples, unsigned flags, pat_bp_t* out);

/* pat_bp_create_constant -- the conventional back projection that Sec. III
 * compares against: Eq. (BP) with the time of flight computed analytically
 * for a constant sound speed (Sec. II-C), t_sj = |r_j - r_s| / c0 (Sec. III
 * uses c0 = 1560 m/s).  No travel-time table is built or stored: the gather
 * kernel evaluates every delay from a 32-byte anchor per (pixel tile, sensor)
 * and 16 bytes per pixel (FP32, a few 1e-6 samples from the exact delay).
 *   c0            sound speed (m/s), finite and > 0
 *   sensors_host  [n_sensors][3] positions (m), anywhere (inside the grid box
 *                 or not); for a 2-D grid only x and y are used
 *   other arguments as pat_bp_create (the grid gives the pixel positions and
 *                 the output geometry)
 * Every other call (reconstruct, preprocess/gather, host round trip, plans,
 * autotuning, eviction) accepts the handle; pat_bp_table returns its bases and
 * slots but no offsets, and a plan takes only handles of one delay source.
 * Blocking.  Errors: PAT_ERR_INVALID, PAT_ERR_OOM, PAT_ERR_CUDA. */
pat_status pat_bp_create_constant(double c0, const pat_grid* grid, const double* sensors_host,
                                  int n_sensors, const uint8_t* mask_host,
                                  const float* weights_host, double dt, int n_samples,
                                  unsigned flags, pat_bp_t* out);

/* pat_bp_set_solid_angle -- switch a handle to the exact back projection that
 * Eq. (BP) approximates (Sec. II-C notes the approximation assumes a circular
 * scan with a radius much larger than the imaged region): every term is
 * weighted by the share of the full angle that the sensor's element subtends
 * at the pixel,
 *     w_s(r) = elem_s (n_s . (r - r_s)) / |r - r_s|^d / omega0,
 * d = 2 for a 2-D grid (plane angle; x and y only) and 3 for a 3-D grid.  This
 * replaces the per-sensor weights of the handle.  The kernel evaluates w from
 * 32 bytes per (pixel tile, sensor) and 16 per pixel (FP32, relative error a
 * few 1e-7); for a closed array the weights of a pixel inside it sum to 1.
 *   normals_host  [n_sensors][3] element normals pointing into the imaged
 *                 region (normalised here; a zero normal is an error)
 *   elem_host     [n_sensors] element length (2-D, m) or area (3-D, m^2), >= 0
 *   omega0        the full angle: 2 pi for a closed curve (2-D), 4 pi for a
 *                 closed surface, 2 pi for a plane or a hemisphere's half space
 * A pixel on a sensor has no finite weight.  Every reconstruction path takes
 * the handle (single frames, batches, plans whose handles all have weights,
 * serving, the no-allocation entry); a frame has the same bits alone and in a
 * batch.  Host mirrors are updated.  Blocking (synchronises the device).
 * Errors: PAT_ERR_INVALID (bad arguments, evicted handle), PAT_ERR_OOM,
 * PAT_ERR_CUDA. */
pat_status pat_bp_set_solid_angle(pat_bp_t h, const double* normals_host, const double* elem_host,
                                  double omega0);

/* pat_bp_reconstruct -- the on-line step: Eq. (BP) for n_frames frames that
 * share the handle's table.
 *   signals_dev   [n_frames][n_sensors][n_samples] of dtype; for PAT_BF16 and
 *                 PAT_F16 the pressure is code * scale
 *   scales_dev    [n_frames][n_sensors] FP32 per-row scales; required for the
 *                 16-bit dtypes, optional (NULL = 1) for PAT_F32
 *   out_dev       [n_frames][grid] dense image (zeros outside the mask), or
 *                 [n_frames][n_pix] with PAT_FLAG_COMPACT_OUT
 *   stream        CUDA stream; the call is asynchronous on it
 * FP32 signals are preprocessed into FP32 integrands; 16-bit signals into
 * 16-bit (value, slope) pairs with a per-row FP32 scale.  Accumulation is FP32.
 * The first call with more frames than any earlier call grows the handle's
 * integrand buffer (a device allocation); pat_bp_reserve avoids that.
 * Calls on one handle must not overlap on the GPU (they share that buffer).
 * The caller keeps signals/out alive until the stream passes this point. */
pat_status pat_bp_reconstruct(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                              const float* scales_dev, int n_frames, float* out_dev,
                              pat_stream_t stream);

/* pat_bp_preprocess / pat_bp_gather -- the two kernels of pat_bp_reconstruct
 * as separate calls (same arguments, same buffers): pat_bp_preprocess forms
 * the Eq. (BP) integrand of n_frames frames into the handle's buffer;
 * pat_bp_gather back-projects the last preprocessed n_frames frames into
 * out_dev.  pat_bp_reconstruct == preprocess then gather on one stream. */
pat_status pat_bp_preprocess(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                             const float* scales_dev, int n_frames, pat_stream_t stream);
pat_status pat_bp_gather(pat_bp_t h, int n_frames, float* out_dev, pat_stream_t stream);

/* pat_bp_reconstruct_noalloc -- pat_bp_reconstruct without any device
 * allocation, for callers that may not allocate device memory: hosts that own
 * all device memory in their own pool or budget, and per-frame loops that
 * must not call the CUDA allocator (its calls can synchronise the device and
 * add latency jitter).  The paper has no counterpart; this is an interface
 * convenience.  Same arguments and result as pat_bp_reconstruct.  All scratch
 * (integrand, multipliers, partial sums, counters, tickets) comes from one
 * file-scope device array of 16 MiB per device, held until the process exits;
 * a reconstruction needing more returns PAT_ERR_INVALID with the byte count
 * (one paper-shaped frame of 512 sensors x 2048 samples needs about 5 MiB).
 * The first call on a device looks up the array's address; make it before any
 * stream capture.  Calls share the array: work of two calls that overlaps on
 * the GPU races, so serialise them.  Each call clears, on its stream, the
 * parts that must start at zero.  Device-side timeouts are reported by
 * pat_bp_sync on the handle. */
pat_status pat_bp_reconstruct_noalloc(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                                      const float* scales_dev, int n_frames, float* out_dev,
                                      pat_stream_t stream);

/* pat_bp_reconstruct_host -- the paper's timed on-line path (Sec. III):
 * signals and scales from host memory in, the image to host memory out.
 * Synchronous; uses the handle's own stream.  Page-locked (pinned) buffers are
 * read and written in place by the kernels (the preprocessing reads the
 * signals across the host link, the last kernel stores the image there), with
 * no staging copy; pageable buffers are copied through device staging buffers.
 * The caller must not modify the buffers during the call. */
pat_status pat_bp_reconstruct_host(pat_bp_t h, const void* signals_host, pat_dtype dtype,
                                   const float* scales_host, int n_frames, float* out_host);

/* pat_bp_reserve -- allocate the integrand buffer for up to max_frames frames
 * of dtype now, so later calls allocate nothing. */
pat_status pat_bp_reserve(pat_bp_t h, int max_frames, pat_dtype dtype);

/* pat_bp_sync -- wait for `stream`, then report a device-side timeout recorded
 * by any earlier launch of this handle (and clear it). */
pat_status pat_bp_sync(pat_bp_t h, pat_stream_t stream);

/* pat_bp_info -- sizes and layout facts of the handle. */
pat_status pat_bp_info(pat_bp_t h, pat_bp_info_t* info);

/* pat_bp_table -- copy the device table back (tests): u_host [n_tiles][n_sensors]
 * [tile_pix] FP32 offsets, base_host [n_tiles][n_sensors] int32 bases, pix_host
 * [n_tiles * tile_pix] output index of each slot (-1 = padding).  Any pointer
 * may be NULL.  u + base is T/dt; entries out of the record hold 1e30.  A
 * constant-speed handle has no offsets: u_host must be NULL for it
 * (PAT_ERR_INVALID otherwise). */
pat_status pat_bp_table(pat_bp_t h, float* u_host, int32_t* base_host, int32_t* pix_host);

/* pat_bp_evict -- free the handle's device table and working buffers (needs
 * PAT_FLAG_HOST_MIRROR); synchronises the device first.  Reconstruction calls
 * fail with PAT_ERR_INVALID until pat_bp_restore. */
pat_status pat_bp_evict(pat_bp_t h);

/* pat_bp_restore -- reallocate the device table and copy it back from the
 * pinned host mirror, asynchronously on stream (no-op when resident). */
pat_status pat_bp_restore(pat_bp_t h, pat_stream_t stream);

/* pat_bp_destroy -- free the handle and its device memory (synchronises). */
pat_status pat_bp_destroy(pat_bp_t h);

/* pat_fmm_host -- the library's own host fast marching (Sec. II-B) from one
 * point source; order 1 (first-order upwind) or 2 (the printed second-order
 * stencil); T_out [grid] receives FP64 arrival times (s).  CPU only. */
pat_status pat_fmm_host(const float* speed_host, const pat_grid* grid, const double* src_xyz,
                        int order, double* T_out);

/* pat_fmm_gpu -- first-order arrival times (Sec. II-B) of n_src point sources
 * (src_xyz [n_src][3]) solved on the current CUDA device: the Godunov system
 * iterated block by block to its fixed point with the host march's
 * arithmetic.  T_out (host) [n_src][grid] receives FP64 times (s), equal to
 * pat_fmm_host(order 1) of each source.  Synchronous; PAT_ERR_INVALID for a
 * source outside the grid box, PAT_ERR_CUDA for a device failure. */
pat_status pat_fmm_gpu(const float* speed_host, const pat_grid* grid, const double* src_xyz,
                       int n_src, double* T_out);

/* pat_table_host -- the table pat_bp_create would upload, built on the host
 * only (no GPU needed): same arguments as pat_bp_create.  info receives the
 * sizes; u_host [n_tiles][n_sensors][tile_pix], base_host [n_tiles][n_sensors]
 * and slot_host [n_tiles * tile_pix] are filled when non-NULL (call once with
 * NULL buffers to learn the sizes).  The split/sensor_warps fields of info
 * are not set.  CPU only, except with PAT_FLAG_GPU_TABLE, which solves the
 * arrival times on the current CUDA device (the result is the same). */
pat_status pat_table_host(const float* speed_host, const pat_grid* grid, const double* sensors_host,
                          int n_sensors, const uint8_t* mask_host, double dt, int n_samples,
                          unsigned flags, pat_bp_info_t* info, float* u_host, int32_t* base_host,
                          int32_t* slot_host);

/* ------------------------------------------------------------------------
 * Many instances in persistent launches (uneven grids, sensor counts, sample
 * counts and frame counts).  A plan fixes the handles and their frame counts
 * and groups the instances by frames per unit FB (the largest power of two up
 * to 8 not above an instance's frame count: FB frames share each pass over a
 * table tile).  Each execution runs one preprocessing launch per group, then
 * one persistent gather launch per group (the first programmatically
 * dependent on the preprocessing), optionally replayed as a CUDA graph.  The
 * summation order of every instance is its handle's own, so each image is
 * bit-identical to that handle's pat_bp_reconstruct of the same frames,
 * whatever else is in the plan or however the launches are shaped.
 * ------------------------------------------------------------------------ */
typedef struct pat_plan_s* pat_plan_t;

#define PAT_PLAN_AUTOTUNE 0x1u /* time candidate launch shapes at the first execution */
#define PAT_PLAN_GRAPH 0x2u    /* capture the launches once, replay a CUDA graph */

typedef struct {
  int n_inst;
  int frames_per_unit;   /* FB: frames that share one pass over a table tile
                            (the largest over the plan's classes)              */
  int sensors_per_stage; /* S                                                  */
  int stages;            /* pipeline depth of the gather                       */
  int smem_budget_kb;    /* shared memory per CTA the shape was sized for      */
  int grid;              /* persistent CTAs of the gather launch               */
  int64_t n_units;       /* work units (frame group, tile, sensor segment)     */
  int tuned;             /* 1 once the autotuner chose the shape               */
  int graph;             /* 1 once a CUDA graph is captured                    */
  double tune_ms;        /* best measured time per execution while tuning      */
  int n_classes;         /* groups of instances with the same FB (one
                            preprocessing and one gather launch each)          */
  int fb_mask;           /* OR of the classes' FB values                       */
} pat_plan_info_t;

/* pat_plan_create -- n (1..64) distinct handles of one device, all with the
 * same tile size, each with n_frames[i] frames per execution, all signals of
 * dtype.  Allocates the per-handle integrand and scratch buffers.  Errors:
 * PAT_ERR_INVALID (duplicates, mixed tile sizes, bad counts), PAT_ERR_OOM. */
pat_status pat_plan_create(const pat_bp_t* handles, const int* n_frames, int n, pat_dtype dtype,
                           unsigned flags, pat_plan_t* out);

/* pat_plan_execute -- signals_dev[i] [n_frames[i]][N_s][N_t], scales_dev[i]
 * (required for 16-bit dtypes, else may be NULL or hold NULLs), outs_dev[i] as
 * in pat_bp_reconstruct.  Asynchronous on stream, except that the first call
 * of an autotuning plan synchronises while it times candidate shapes (that
 * call must not be captured by the caller).  Executions of one plan, and of
 * plans or calls sharing a handle, must not overlap on the GPU.  On the host,
 * an execution holds every handle of the plan (the same lock as the handle's
 * own calls) while it enqueues its work, so handle calls from other threads
 * wait for it instead of changing buffers the launch reads. */
pat_status pat_plan_execute(pat_plan_t plan, const void* const* signals_dev,
                            const float* const* scales_dev, float* const* outs_dev,
                            pat_stream_t stream);

/* pat_plan_sync -- wait for stream and report a device-side timeout of the
 * plan's launches (PAT_ERR_TIMEOUT), clearing it. */
pat_status pat_plan_sync(pat_plan_t plan, pat_stream_t stream);

pat_status pat_plan_info(pat_plan_t plan, pat_plan_info_t* info);
pat_status pat_plan_destroy(pat_plan_t plan);

/* pat_bp_reconstruct_multi -- one-shot plan (no tuning, no graph) executed on
 * stream; same arguments as pat_plan_create + pat_plan_execute. */
pat_status pat_bp_reconstruct_multi(const pat_bp_t* handles, const void* const* signals_dev,
                                    pat_dtype dtype, const float* const* scales_dev,
                                    const int* n_frames, float* const* outs_dev, int n,
                                    pat_stream_t stream);

/* pat_bp_autotune -- time candidate launch shapes for n_frames frames of dtype
 * on these inputs (the output is written with the correct result) and keep the
 * fastest for later pat_bp_reconstruct / pat_bp_gather calls of the handle
 * with the same frames-per-unit grouping.  Synchronous. */
pat_status pat_bp_autotune(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                           const float* scales_dev, int n_frames, float* out_dev,
                           pat_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: frames arrive one request at a time for several registered
 * subjects (speed maps); a scheduler thread keeps tables resident on the
 * device within an HBM budget (least recently used tables are evicted to a
 * pinned host copy and reloaded on demand), batches the pending frames of a
 * subject into one reconstruction, and runs batches of different subjects
 * concurrently on several streams while new requests keep arriving
 * (continuous batching).  Every result is bit-identical to reconstructing
 * that frame alone with pat_bp_reconstruct.
 * ------------------------------------------------------------------------ */
typedef struct pat_srv_s* pat_srv_t;

typedef struct {
  int n_streams;        /* batches in flight at once (default 4)                */
  int max_batch_frames; /* frames of one subject in one batch (default 16)      */
  int max_queue;        /* pending requests before submit says BUSY (def. 4096) */
  int stall_us;         /* test hook: scheduler sleeps this long per cycle (0)  */
} pat_srv_cfg;

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t batches, uploads, evictions;
  double p50_ms, p99_ms, mean_batch_frames;
  size_t resident_bytes, budget_bytes;
} pat_srv_stats_t;

/* pat_srv_create -- hbm_budget: device bytes the resident tables and their
 * working buffers may use; cfg may be NULL (defaults).  Starts the scheduler
 * thread on the current device. */
pat_status pat_srv_create(size_t hbm_budget, const pat_srv_cfg* cfg, pat_srv_t* out);

/* pat_srv_register -- arguments of pat_bp_create; builds the subject's table
 * (host fast marching, or the GPU solver with PAT_FLAG_GPU_TABLE) and keeps a
 * pinned host copy for reloads.  The subject stays resident, with its working
 * buffers for a full batch, if the budget allows; else it is evicted and
 * uploaded when a request needs it.  Every request slot's device staging is
 * sized for a full batch of the subject here, so serving never grows it.
 * Blocking (an allocation can wait for batches in flight). */
pat_status pat_srv_register(pat_srv_t srv, const float* speed_host, const pat_grid* grid,
                            const double* sensors_host, int n_sensors, const uint8_t* mask_host,
                            const float* weights_host, double dt, int n_samples, unsigned flags,
                            int* subject_id);

/* pat_srv_submit -- one frame: signals_host [N_s][N_t] of dtype (scales_host
 * [N_s] for 16-bit dtypes), result written to out_host (dense grid or compact,
 * as the subject's flags say).  Both host buffers must stay valid until
 * pat_srv_poll reports the ticket done.  Errors: PAT_ERR_NOT_FOUND (unknown
 * subject), PAT_ERR_BUSY (queue full), PAT_ERR_INVALID. */
pat_status pat_srv_submit(pat_srv_t srv, int subject, const void* signals_host, pat_dtype dtype,
                          const float* scales_host, float* out_host, uint64_t* ticket);

/* pat_srv_poll -- wait up to timeout_us (0 = do not wait) for the ticket.
 * Returns PAT_PENDING while in flight, else the request's final status (and
 * forgets the ticket); latency_s (may be NULL) receives submit-to-done time.
 * PAT_ERR_NOT_FOUND for an unknown or already reported ticket. */
pat_status pat_srv_poll(pat_srv_t srv, uint64_t ticket, int timeout_us, double* latency_s);

pat_status pat_srv_stats(pat_srv_t srv, pat_srv_stats_t* stats);

/* pat_srv_set_budget -- change the HBM budget of a running server (bytes > 0).
 * Idle resident subjects are evicted to their host copies, least recently
 * used first, until the resident ones fit; subjects with batches in flight
 * stay until those finish, and later admissions keep to the new budget.
 * Blocking (an eviction waits for the device).  PAT_ERR_INVALID for a zero
 * budget. */
pat_status pat_srv_set_budget(pat_srv_t srv, size_t hbm_budget);

/* pat_srv_destroy -- finish everything in flight, stop the scheduler, free. */
pat_status pat_srv_destroy(pat_srv_t srv);

/* pat_probe_l2_to_smem -- diagnostic (no counterpart in the paper): measures,
 * on the current device, the aggregate bandwidth of 1-D bulk copies from an
 * L2-resident buffer into shared memory (one CTA per SM streaming 64 KB
 * chunks of a 64 MB buffer through three slots, about 2 GB), the path the
 * staged gather's table blocks and integrand windows take.  Writes GB/s to
 * *gbps.  Allocates and frees 64 MB of device memory; synchronous.  Errors:
 * PAT_ERR_INVALID, PAT_ERR_CUDA, PAT_ERR_TIMEOUT (a bounded wait gave up). */
pat_status pat_probe_l2_to_smem(double* gbps);

/* pat_test_wait_timeout -- launches one CTA whose mbarrier wait can never
 * complete, bounded by timeout_ns; returns PAT_ERR_TIMEOUT when the kernel
 * gave up and reported it, PAT_OK if it (wrongly) completed.  Exercises the
 * failure path of every bounded device wait without faulting the GPU. */
pat_status pat_test_wait_timeout(uint64_t timeout_ns);

/* pat_test_gather_only -- measurement hook, no counterpart in the paper: after
 * pat_bp_preprocess of one frame, launches the single-frame gather kernel of
 * pat_bp_gather alone on `stream` (asynchronous), without the reduction that
 * sums its per-segment results into the image, so that the gather kernel's own
 * duration can be timed with events around this call.  The image is not
 * written; a following pat_bp_gather recomputes everything.  Errors:
 * PAT_ERR_INVALID (NULL handle, no one-frame preprocess before, or a handle
 * whose single frame takes the staged kernel), PAT_ERR_CUDA. */
pat_status pat_test_gather_only(pat_bp_t h, pat_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PAT_BP_H */
