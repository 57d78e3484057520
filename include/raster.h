/*
 * raster.h -- C ABI of the GB300 RASTER library (libraster.so).
 *
 * RASTER (Ulm et al., "Contraction Clustering (RASTER)") clusters 2-D points
 * in two steps (Alg. 1):
 *   contraction   -- every point (x, y) is projected to the tile
 *                    (floor(x*s), floor(y*s)), s = 10^precision, and the
 *                    points per tile are counted (Alg. 1 first loop,
 *                    Sect. 3.2); tiles with at least tau points are
 *                    "significant" (Alg. 1 second loop);
 *   agglomeration -- significant tiles at Chebyshev distance 1 are joined
 *                    into clusters and clusters of fewer than mu tiles are
 *                    dropped (Alg. 1 while loop; Sect. 3.2, eight neighbours).
 *
 * Conventions fixed by this library (the paper leaves them open):
 *   - ix = floor(RN(x * s)): one IEEE-754 binary64 multiply rounded to nearest
 *     even, then floor (not truncation), evaluated bit-exactly on the GPU;
 *   - a valid tile index lies in [INT32_MIN+1, INT32_MAX-1]; a point with a
 *     non-finite coordinate or an index outside that range is skipped and
 *     reported as RASTER_E_RANGE;
 *   - tile key = (int64_t)ix << 32 | (uint32_t)iy;
 *   - significant: count >= tau; kept: cluster size in tiles >= mu;
 *   - cluster id = key of the cluster's smallest tile in (ix, iy)
 *     lexicographic order (ix first); noise label = RASTER_NOISE.
 * raster_create_ex extends the neighbourhood (Chebyshev or Manhattan
 * distance delta, Sect. 3.2), adds the 2 x 2 group rule of Sect. 3.6, and
 * takes points with three coordinates (its own key format, see
 * raster_params); the defaults above are unchanged.
 *
 * Memory: points and labels are caller buffers; tables and results live in
 * device memory owned by the handle.  "stream" arguments are cudaStream_t
 * values passed as void* (NULL = the legacy default stream).  Calls on one
 * handle must not run concurrently from several host threads.
 *
 * Status: every call returns RASTER_OK (0) or one of the RASTER_E_* codes.
 * Device-side failures (range errors, a full table) are recorded in the
 * handle and reported at the next call that synchronises (agglomerate,
 * status, labels).  No call traps or hangs the GPU: every device loop is
 * bounded and reports exhaustion through a status word.
 */
#ifndef RASTER_H
#define RASTER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RASTER_OK 0
#define RASTER_E_ARG 1         /* invalid argument (bad tau/mu/precision/size/pointer alignment) */
#define RASTER_E_RANGE 2       /* some coordinate was not finite or its tile index out of range */
#define RASTER_E_OOM 3         /* device or pinned host allocation failed */
#define RASTER_E_TABLE_FULL 4  /* a bounded hash probe gave up (table full) */
#define RASTER_E_CUDA 5        /* a CUDA runtime call failed */
#define RASTER_E_INTERNAL 6    /* a bounded device iteration did not converge */
#define RASTER_E_STATE 7       /* call not valid in the handle's state (e.g. labels before agglomerate) */
#define RASTER_E_LIMIT 8       /* input larger than a fixed capacity (raster_count_tiles_static) */

#define RASTER_NOISE INT64_MIN /* label of a point outside every kept cluster */
#define RASTER_INVALID_KEY (INT64_MIN + 1) /* tile key of a point that did not project (raster_contract_keys) */

typedef struct raster_handle raster_handle;

/* Result of raster_agglomerate.  Arrays are DEVICE pointers owned by the
 * handle, valid until the next contract/reset/agglomerate/destroy on it.
 * Row i describes one tile of a kept cluster: its key, its point count and
 * its cluster id.  Row order is unspecified (the set of rows is unique). */
typedef struct {
    const int64_t *key;
    const uint32_t *count;
    const int64_t *cid;
    int64_t n_tiles;        /* rows: tiles in kept clusters */
    int64_t n_clusters;     /* clusters with at least mu tiles */
    int64_t n_distinct;     /* tiles with at least one point (D) */
    int64_t n_significant;  /* tiles with at least tau points (S) */
    int64_t n_points;       /* points submitted to contract (range errors included) */
} raster_clusters;

/* Create a handle for one clustering problem.
 * precision: tile side is 10^-precision (Alg. 1 input "prec"; any finite real,
 *   e.g. 2, 3.5 or 0.73, Sect. 4.1 and App. A); s = 10^precision must be a
 *   normal positive double.  tau >= 1, mu >= 1 (Alg. 1 inputs).
 * On success *out receives the handle (allocated on the current device). */
int raster_create(double precision, uint32_t tau, uint32_t mu, raster_handle **out);

/* Neighbourhood metrics for neighbors(u, delta) (Alg. 1; Sect. 3.2: significant
 * tiles at most a Manhattan or Chebyshev distance of delta steps apart). */
#define RASTER_CHEBYSHEV 0
#define RASTER_MANHATTAN 1
#define RASTER_MAX_DELTA 4

/* Parameters of raster_create_ex.
 *   precision, tau, mu  as for raster_create.
 *   metric   RASTER_CHEBYSHEV or RASTER_MANHATTAN (Sect. 3.2).
 *   delta    1..RASTER_MAX_DELTA: tiles at that distance or less are
 *            neighbours (Alg. 1 input delta).  raster_create uses Chebyshev 1,
 *            the eight neighbours.
 *   groups   0 or 1.  1 adds the post-processing step of Sect. 3.6
 *            ("disadvantageous grid layouts", Fig. 4): every occupied tile of
 *            a group of 2 x 2 tiles holding at least tau points together is
 *            significant too (raster_clusters.n_significant counts them).
 *   dims     coordinates per point: 2 (or 0), or 3 (the generalisation to
 *            higher dimensions of Sect. 3.6).  With 3, every point array of
 *            the handle is n x 3 float64, 8-byte aligned; each tile index
 *            must lie in [-(2^20 - 1), 2^20 - 2] (else RASTER_E_RANGE) and
 *            key = (ix + 2^20) << 42 | (iy + 2^20) << 21 | (iz + 2^20), so
 *            integer key order is (ix, iy, iz) order and cluster ids are the
 *            smallest key; neighbours are taken over all three axes
 *            (Chebyshev 1: the 26 surrounding tiles); groups must be 0. */
typedef struct {
    double precision;
    uint32_t tau, mu;
    uint32_t metric;
    uint32_t delta;
    uint32_t groups;
    uint32_t dims;
} raster_params;

/* Create a handle with the parameters above (Alg. 1 inputs prec, tau, delta,
 * mu).  RASTER_E_ARG for an unknown metric, delta outside 1..RASTER_MAX_DELTA,
 * groups other than 0/1, dims other than 0/2/3, groups with dims 3, a
 * neighbourhood of more than 40 forward offsets (three coordinates allow
 * Chebyshev 1 and Manhattan up to 3), or any argument raster_create refuses.  Every other
 * call works on such a handle as on one from raster_create; the batched,
 * served and fixed-capacity entry points use Chebyshev distance 1 only. */
int raster_create_ex(const raster_params *params, raster_handle **out);

/* Size the tile table for at least n_tiles distinct tiles (like reserving a
 * hash map; the paper's fixed table budget T, Sect. 3.6).  Optional: the
 * table also grows on demand.  Synchronises the handle's stream. */
int raster_reserve(raster_handle *h, int64_t n_tiles);

/* Contraction of one chunk (Alg. 1 first loop; chunked processing, Sect. 3.6).
 * xy: DEVICE pointer to n points as interleaved float64 pairs (x0,y0,x1,y1,..),
 *   16-byte aligned (triples x,y,z, 8-byte aligned, for a handle created
 *   with dims = 3; the same holds for every point array below); caller-owned
 *   and must stay valid until the stream work completes.  n >= 0.  Callable
 *   any number of times; counts accumulate.
 * Work is enqueued on `stream`; the call synchronises once per 2^30 points
 * to read the table's tile count (and grows the table when needed), so xy
 * may be released when it returns.  The total number of points per handle
 * must stay below 2^32. */
int raster_contract(raster_handle *h, const double *xy, int64_t n, void *stream);

/* Contraction as raster_contract (Alg. 1 first loop; the projection of
 * Sect. 3.2), which also writes each point's tile key, so that the labels of
 * the same points can later be read from the keys (raster_key_labels)
 * instead of projecting every point a second time.
 * keys: DEVICE int64[n], 8-byte aligned, caller-owned; keys[i] is the tile of
 * point i in the handle's packing, or RASTER_INVALID_KEY for a point with a
 * non-finite coordinate or a tile index out of range (those points are
 * skipped and reported as RASTER_E_RANGE, as by raster_contract).
 * Asynchronous like raster_contract; keys are complete when the stream
 * reaches the end of the call. */
int raster_contract_keys(raster_handle *h, const double *xy, int64_t n, int64_t *keys, void *stream);

/* Add tiles counted elsewhere: count[i] points to tile key[i], as if those
 * points had been contracted into this handle.  This is the join of partial
 * count maps that P-RASTER performs after its parallel contraction (Sect.
 * 3.5), and the step a sharded run uses when the tiles of a vertical slice
 * arrive at the device that owns it (Alg. 2).
 * key: DEVICE int64 tile keys (8-byte aligned) in the handle's packing (two
 *   int32 indices, or three 21-bit fields for dims = 3); count: DEVICE uint32
 *   (4-byte aligned); both caller-owned, n >= 0 entries; a key may repeat.
 * A key outside the valid index range is skipped (RASTER_E_RANGE, reported
 * like a range error of contraction); counts of 0 are ignored.  Grows the
 * table first so every key fits, and synchronises `stream` twice (to read
 * the points the counts stand for, and the table's tile count).
 * RASTER_E_ARG for bad pointers or if the handle's total points would reach
 * 2^32. */
int raster_contract_tiles(raster_handle *h, const int64_t *key, const uint32_t *count, int64_t n, void *stream);

/* Contraction of one chunk (Alg. 1 first loop; Sect. 3.6) as raster_contract,
 * but xy is in HOST memory (pinned for full speed).  The
 * points are streamed through device staging buffers, copies overlapping the
 * contraction.  Returns once xy may be reused (synchronous). */
int raster_contract_host(raster_handle *h, const double *xy_host, int64_t n, void *stream);

/* Agglomeration (Alg. 1 threshold + while loop) over everything contracted
 * so far, on the stream of the last contract call.  Fills *out (device
 * arrays owned by the handle) and synchronises.  Further contract calls
 * are allowed afterwards (streaming); they invalidate *out. */
int raster_agglomerate(raster_handle *h, raster_clusters *out);

/* Per-point cluster labels (the RASTER* second pass, Sect. 4.1): projects
 * each point again and writes its tile's cluster id, or RASTER_NOISE.
 * Requires a preceding raster_agglomerate with no contract since.
 * xy: DEVICE, n x 2 float64, 16-byte aligned; labels: DEVICE int64[n],
 * caller-owned.  Asynchronous on `stream`, except that the first call after
 * an agglomeration of two-coordinate points whose tile table exceeds 64 MiB
 * synchronises once, to size an index of the kept tiles by 8 x 8-tile block
 * that answers most lookups from L2.  The environment variable
 * RASTER_LABEL_INDEX, read when the handle is created, forces that index on
 * ("1") or off ("0"); the labels are the same either way. */
int raster_point_labels(raster_handle *h, const double *xy, int64_t n, int64_t *labels, void *stream);

/* Per-point cluster labels (RASTER*, Sect. 4.1) from the points' tile keys,
 * as written by raster_contract_keys into this handle: the same labels that
 * raster_point_labels gives for those points, without reading or projecting
 * the coordinates again.  Requires a preceding raster_agglomerate with no
 * contract since.  keys: DEVICE int64[n] (8-byte aligned; any key of the
 * handle's packing is accepted; RASTER_INVALID_KEY is labelled RASTER_NOISE
 * and raises the handle's range flag, as a non-finite point does in
 * raster_point_labels); labels: DEVICE int64[n], caller-owned.  Asynchronous,
 * with the same one-time synchronisation as raster_point_labels. */
int raster_key_labels(raster_handle *h, const int64_t *keys, int64_t n, int64_t *labels, void *stream);

/* Per-point labels (RASTER*, Sect. 4.1) as raster_point_labels, with HOST xy
 * and HOST labels; synchronous. */
int raster_point_labels_host(raster_handle *h, const double *xy_host, int64_t n, int64_t *labels_host,
                             void *stream);

typedef struct {
    int64_t capacity, occupied, probe_sum, probe_max;
} raster_table_stats_t;

/* Diagnostics of the tile table (no counterpart in the paper).  capacity:
 * slots; occupied: tiles in the table (D); probe_sum / probe_max: over the
 * occupied slots, the number of slots a lookup of that tile reads (1 + its
 * distance from its home slot within the 4096-slot bucket).  probe_sum /
 * occupied is the mean probe length of a successful lookup.  Synchronises
 * the handle's stream. */
int raster_table_stats(raster_handle *h, raster_table_stats_t *out);

/* The whole method on HOST points in one call (Alg. 1 and the RASTER* labels,
 * Sect. 4.1): contraction of the n points at HOST xy_host (layout as for
 * raster_contract, added to whatever the handle holds), agglomeration into
 * *out (as raster_agglomerate), and the label of each of the n points into
 * HOST labels_host (int64[n], as raster_point_labels).  The points are copied
 * to the device once, in chunks, each chunk's first contraction pass running
 * while later chunks are still being copied, and they stay on the device (a
 * buffer owned by the handle, reused by later calls, freed by
 * raster_destroy) for the label pass; labels return chunk by chunk behind
 * the label kernels.  If that buffer cannot be allocated the call copies the
 * points twice instead (raster_contract_host, raster_agglomerate,
 * raster_point_labels_host).  Pinned host memory makes the copies
 * asynchronous.  Synchronous; returns what raster_agglomerate returns, or
 * the first error. */
int raster_cluster_host(raster_handle *h, const double *xy_host, int64_t n, int64_t *labels_host,
                        raster_clusters *out, void *stream);

/* RASTER' output (Sect. 3.4; clusters as sets of points, Fig. 2d): the points
 * of every kept tile, grouped by result row.  Requires a preceding
 * raster_agglomerate with no contract since; rows follow the order of that
 * call's raster_clusters.  For the n points at DEVICE xy (n x 2 float64,
 * 16-byte aligned; normally the points that were contracted):
 *   row_start   DEVICE int64[n_tiles + 1]: row r's points are
 *               point_index[row_start[r] .. row_start[r+1]);
 *   point_index DEVICE int64[capacity]: indices (0..n-1) of the points in
 *               kept tiles, grouped by row; order within a row unspecified;
 *   *n_grouped  HOST: number of such points (= row_start[n_tiles]).
 * If capacity < *n_grouped nothing is written to point_index and
 * RASTER_E_ARG is returned; the handle stays usable.  n above 2^32 - 1 is
 * RASTER_E_LIMIT.  Synchronises `stream` once. */
int raster_point_groups(raster_handle *h, const double *xy, int64_t n, int64_t *row_start, int64_t *point_index,
                        int64_t capacity, int64_t *n_grouped, void *stream);

/* The tile table after contraction (acc of Alg. 1): copy every tile with at
 * least one point (key, count) into caller DEVICE buffers of `capacity` rows;
 * *n_out receives D.  Order unspecified.
 * Returns RASTER_E_ARG if capacity < D (nothing is written then).
 * Synchronises.  Used for checkpointing and for tests. */
int raster_export_tiles(raster_handle *h, int64_t *key, uint32_t *count, int64_t capacity, int64_t *n_out);

/* Forget all points (keep the table's capacity) on `stream`; clears errors.
 * Lifecycle call; no counterpart in the paper. */
int raster_reset(raster_handle *h, void *stream);

/* Synchronise and return the handle's recorded status (RASTER_OK if none).
 * Diagnostics; no counterpart in the paper. */
int raster_status(raster_handle *h);

/* The scale s = 10^precision used by project() (Alg. 1; Sect. 3.2), as the one
 * double both the kernels and any other implementation must multiply by. */
double raster_get_scale(const raster_handle *h);

/* Table capacity in slots.  Diagnostics; no counterpart in the paper. */
int64_t raster_table_capacity(const raster_handle *h);

/* Number of kernels this library has launched in this process, over all
 * handles (lets a caller count device launches in a region).  Diagnostics;
 * no counterpart in the paper. */
uint64_t raster_kernel_launches(void);

/* Bounds of the device loops, lowered so that tests can drive the failure
 * paths without faulting a GPU.  No counterpart in the paper.  probe_limit
 * caps the slots one table insertion probes; union_limit caps the steps of
 * one union-find join; a negative value restores the library's own bound
 * (the default).  Lookups keep their full bound, so a lowered limit makes an
 * insertion or a join give up, never hides a tile.  The values are read when
 * a handle (raster_create*), a batch (raster_batch_create) or a served
 * request (raster_server_submit) is created and stay with it; every loop
 * still ends, and an exhausted bound surfaces as RASTER_E_TABLE_FULL or
 * RASTER_E_INTERNAL from that handle, batch instance or request only.
 * Process-wide; not meant for production use.  Returns RASTER_OK. */
int raster_set_test_limits(int32_t probe_limit, int32_t union_limit);

/* Release the handle and its device memory (synchronises).  Lifecycle call;
 * no counterpart in the paper. */
int raster_destroy(raster_handle *h);

/* ---- Batched form: many independent instances, one graph launch ----------
 *
 * Runs contraction and agglomeration (Alg. 1) for `count` independent RASTER
 * problems at once, each with its own points, precision, tau and mu.  All
 * instances share one persistent contraction kernel and one sequence of
 * segmented agglomeration kernels, captured once in a CUDA graph at creation
 * and replayed by every raster_batch_run.  Each instance's result is exactly
 * what a separate handle would produce.  (Per-point labels are not part of
 * the batched form.) */
typedef struct {
    const double *xy;  /* DEVICE, n x 2 interleaved float64, 16-byte aligned; must stay
                          valid and hold the instance's points whenever the batch runs */
    int64_t n;         /* points, >= 0 */
    double precision;  /* tile side 10^-precision */
    uint32_t tau, mu;  /* >= 1 */
} raster_instance;

/* Tuning knobs (0 / -1 = default).  None of them changes any result. */
typedef struct {
    double load;     /* table slots >= n_i / load (power of two), 0 < load <= 0.75 */
    int32_t block;   /* threads per block of the contraction kernel: 128, 256 or 512 */
    int32_t width;   /* points per thread per iteration: 1, 2, 4 or 8 */
    int32_t preagg;  /* 1: merge equal tiles within a warp before inserting; 0: off */
} raster_batch_config;

typedef struct raster_batch raster_batch;

/* Plan the batch of Alg. 1 problems (sizes every table from its n, so no table
 * can overflow), allocate its device memory and capture its graph on the
 * current device.  inst[] is copied; the xy pointers are baked into the graph.
 * RASTER_E_ARG for an invalid instance or knob. */
int raster_batch_create(const raster_instance *inst, int32_t count, const raster_batch_config *cfg,
                        raster_batch **out);

/* Run contraction and agglomeration (Alg. 1) of every instance on `stream`
 * (asynchronous: one graph launch). */
int raster_batch_run(raster_batch *b, void *stream);

/* Wait for the last run; returns the worst status over all instances.
 * Synchronisation call; no counterpart in the paper. */
int raster_batch_wait(raster_batch *b);

/* Clusters (Alg. 1 output) of instance i of the last run, after
 * raster_batch_wait: DEVICE arrays owned by the batch, valid until its next
 * run or destroy.  Returns that instance's own status. */
int raster_batch_result(raster_batch *b, int32_t i, raster_clusters *out);

/* Device bytes held by the batch (tables, scratch and results).  Diagnostics;
 * no counterpart in the paper. */
int64_t raster_batch_device_bytes(const raster_batch *b);

/* Release the batch.  Lifecycle call; no counterpart in the paper. */
int raster_batch_destroy(raster_batch *b);

/* ---- Served form: continuous batching of requests ------------------------
 *
 * A serving engine with a worker thread.  Requests (one Alg. 1 problem each)
 * arrive at any time and send their points in chunks (chunked processing,
 * Sect. 3.6).  Every step the engine admits waiting requests in arrival order
 * while free device memory (cudaMemGetInfo minus the caller's reserve) covers
 * what the request's tile table and result rows add, contracts every ready
 * chunk of every admitted request in one segmented launch, and agglomerates
 * every request whose chunks are all in.  Requests therefore overlap on the
 * device; each result equals that of a separate handle.
 *
 * Memory: tables and rows live in device address ranges reserved at create
 * and backed by physical pages only while a live request uses them.  A
 * request's table (a power of two >= n / 0.75 slots, at least 4096; 16 bytes
 * each) is held from admission until it completes, its result rows
 * (max(1, n / tau), 52 bytes each with the agglomeration's work rows) until
 * the client releases it.  Pages no request holds are kept for reuse and
 * given back when admission needs the memory or the engine has been idle for
 * 0.2 s.  A request that does not fit while no other request is active is
 * completed at once with RASTER_E_OOM. */
typedef struct raster_server raster_server;

typedef struct {
    int64_t table_slots;   /* most tile-table slots held at once; 0: as many as device memory could hold */
    int64_t result_rows;   /* most result rows held at once; 0: as many as device memory could hold
                              (at most 2^31 - 2) */
    int32_t max_active;    /* most requests admitted at once, 1..8192 */
    int64_t reserve_bytes; /* device memory admission leaves free for other users (>= 0) */
} raster_server_config;

typedef struct {
    int64_t steps, points, waiting, active, completed_unpolled, table_slots_used, result_rows_used;
    int64_t device_bytes;  /* physical device memory the engine's tables and rows hold now */
    int64_t refused;       /* requests completed with RASTER_E_OOM */
    int64_t gpu_us;        /* device time of all steps so far (events around each step's work), microseconds */
} raster_server_stats_t;

/* Reserve the address ranges on the current device and start the worker
 * thread; no table or row memory is committed yet.  RASTER_E_ARG for a bad
 * config, RASTER_E_CUDA if the device lacks the virtual memory calls.
 * Lifecycle call; no counterpart in the paper. */
int raster_server_create(const raster_server_config *cfg, raster_server **out);

/* Announce request `request_id` (unique among live requests): an Alg. 1
 * problem of n_total points in n_chunks chunks.  Returns RASTER_E_LIMIT if it
 * could never fit (its table and rows exceed the configured bounds, or the
 * device's memory less the reserve).  Thread-safe. */
int raster_server_submit(raster_server *s, int64_t request_id, double precision, uint32_t tau, uint32_t mu,
                         int64_t n_total, int32_t n_chunks);

/* Give the next chunk of a request (chunked contraction, Sect. 3.6): DEVICE
 * xy, n x 2 float64, 16-byte aligned, caller-owned, valid until the request
 * completes.  The chunk sizes must add up to n_total.  Thread-safe. */
int raster_server_push(raster_server *s, int64_t request_id, const double *xy, int64_t n);

/* Take one completed request (Alg. 1 output), waiting up to wait_ms: its id,
 * its clusters (DEVICE arrays in the engine's arena, valid until released) and
 * its latency from submit to completion.  Returns the request's status, or
 * RASTER_E_STATE when none completed in time.  Thread-safe. */
int raster_server_poll(raster_server *s, int32_t wait_ms, int64_t *request_id, raster_clusters *out,
                       double *latency_ms);

/* Free a completed request's table and rows.  Lifecycle call; no counterpart
 * in the paper. */
int raster_server_release(raster_server *s, int64_t request_id);

/* Engine counters; returns the engine's fatal status (RASTER_OK if none).
 * Diagnostics; no counterpart in the paper. */
int raster_server_stats(raster_server *s, raster_server_stats_t *out);

/* Stop the worker and free everything.  Lifecycle call; no counterpart in the
 * paper. */
int raster_server_destroy(raster_server *s);

/* Largest input accepted by raster_count_tiles_static. */
#define RASTER_STATIC_MAX_POINTS 524288

/* Tile counts without any allocation -- the paper has no counterpart; this is
 * for callers that cannot allocate device memory (code running inside another
 * runtime's memory pool or a fixed memory budget, plugins whose host owns all
 * allocations, paths that must avoid the allocator's implicit synchronisation).
 *
 * Projects the n points at DEVICE xy (interleaved float64 pairs, 16-byte
 * aligned) with s = 10^precision exactly like raster_contract and writes every
 * tile holding at least one point as a row (key, count) into the caller's
 * DEVICE arrays key_out and count_out, which must have room for n rows (a tile
 * count never exceeds n).  Row order is unspecified.  *n_tiles_out (HOST)
 * receives the number of rows.  Synchronises `stream` before returning.
 *
 * The hash table is a fixed 16 MiB array of device memory inside the library
 * (present on every GPU that loads the library, until the process exits); no
 * cudaMalloc, cudaFree or other allocating call is made.  n larger than
 * RASTER_STATIC_MAX_POINTS returns RASTER_E_LIMIT and does nothing.  The first
 * call on a device looks up the array's device address (once per device, with
 * that device current); make that first call before any stream capture.  All
 * calls share the array and each clears it first: calls whose GPU work
 * overlaps (other streams or host threads) race and must be serialised.
 * Returns RASTER_E_RANGE if some point was skipped (non-finite or out of the
 * int32 tile range); the rows of every other tile are still written with
 * their exact counts and *n_tiles_out is set, so the caller may use them.
 * n = 0 returns RASTER_OK with *n_tiles_out = 0 (xy may then be NULL).
 * Returns RASTER_E_ARG for bad arguments. */
int raster_count_tiles_static(const double *xy, int64_t n, double precision, int64_t *key_out,
                              uint32_t *count_out, int64_t *n_tiles_out, void *stream);

/* Static description of a status code.  No counterpart in the paper. */
const char *raster_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* RASTER_H */
