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

/* Size the tile table for at least n_tiles distinct tiles (like reserving a
 * hash map; the paper's fixed table budget T, Sect. 3.6).  Optional: the
 * table also grows on demand.  Synchronises the handle's stream. */
int raster_reserve(raster_handle *h, int64_t n_tiles);

/* Contraction of one chunk (Alg. 1 first loop; chunked processing, Sect. 3.6).
 * xy: DEVICE pointer to n points as interleaved float64 pairs (x0,y0,x1,y1,..),
 *   16-byte aligned; caller-owned and must stay valid until the stream work
 *   completes.  n >= 0.  Callable any number of times; counts accumulate.
 * Asynchronous on `stream`, except that it synchronises when the table has
 * to grow.  The total number of points per handle must stay below 2^32. */
int raster_contract(raster_handle *h, const double *xy, int64_t n, void *stream);

/* As raster_contract, but xy is in HOST memory (pinned for full speed).  The
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
 * caller-owned.  Asynchronous on `stream`. */
int raster_point_labels(raster_handle *h, const double *xy, int64_t n, int64_t *labels, void *stream);

/* As raster_point_labels with HOST xy and HOST labels; synchronous. */
int raster_point_labels_host(raster_handle *h, const double *xy_host, int64_t n, int64_t *labels_host,
                             void *stream);

/* Copy every tile with at least one point (key, count) into caller DEVICE
 * buffers of `capacity` rows; *n_out receives D.  Order unspecified.
 * Returns RASTER_E_ARG if capacity < D (nothing is written then).
 * Synchronises.  Used for checkpointing and for tests. */
int raster_export_tiles(raster_handle *h, int64_t *key, uint32_t *count, int64_t capacity, int64_t *n_out);

/* Forget all points (keep the table's capacity) on `stream`; clears errors. */
int raster_reset(raster_handle *h, void *stream);

/* Synchronise and return the handle's recorded status (RASTER_OK if none). */
int raster_status(raster_handle *h);

/* The scale s = 10^precision used for projection (one double). */
double raster_get_scale(const raster_handle *h);

/* Table capacity in slots (for diagnostics). */
int64_t raster_table_capacity(const raster_handle *h);

/* Number of kernels this library has launched in this process, over all
 * handles (diagnostics: lets a caller count device launches in a region). */
uint64_t raster_kernel_launches(void);

/* Release the handle and its device memory (synchronises). */
int raster_destroy(raster_handle *h);

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
 * int32 tile range), RASTER_E_ARG for bad arguments. */
int raster_count_tiles_static(const double *xy, int64_t n, double precision, int64_t *key_out,
                              uint32_t *count_out, int64_t *n_tiles_out, void *stream);

/* Static description of a status code. */
const char *raster_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* RASTER_H */
