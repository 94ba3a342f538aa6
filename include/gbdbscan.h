/*
 * gbdbscan -- DBSCAN for 2D/3D fp32 points on one GB300 GPU (sm_103a).
 *
 * The method is FDbscan and FDbscan-DenseBox of "Fast tree-based algorithms
 * for DBSCAN for low-dimensional data on GPUs" (Prokopenko, Lebrun-Grandie,
 * Arndt; arXiv 2103.05162):
 *   - the two-phase parallel disjoint-set DBSCAN (Sec. 3.2, Algorithm 3): a
 *     preprocessing phase decides core points, a main phase unions every
 *     eps-pair into a lock-free union-find as it is found, with no neighbour
 *     list stored;
 *   - a linear BVH over Morton-sorted primitives as the search index, each
 *     pair visited once through the leaf-index mask (Sec. 4.1, Figure
 *     "pair traversal");
 *   - DenseBox: grid cells of side eps/sqrt(d) holding at least minPts points
 *     become single leaves of the BVH whose points are all core and in one
 *     cluster (Sec. 4.2);
 *   - synchronisation-free union-find with path halving and a final
 *     compression pass (Sec. 4.3).
 *
 * Definitions (Sec. 2.1). N_eps(x) = { y : dist(x,y) <= eps }, x included.
 * x is core iff |N_eps(x)| >= minPts. Clusters are the connected components
 * of the core points under the eps relation. A non-core point within eps of
 * a core point is a border point and joins one of the clusters of its core
 * neighbours (DBSCAN mode); in DBSCAN* mode border points are noise.
 *
 * Distance test. dist(x,y) <= eps is evaluated as the fp32 squared form with
 * no fused multiply-add, in this order:
 *   dk = fl(x_k - y_k); s = fl(d0*d0); s = fl(s + fl(dk*dk)), k = 1..d-1;
 *   adjacent <=> s <= fl(eps*eps).
 * The paper leaves the rounding open; fixing it makes results reproducible
 * bit for bit.
 *
 * Output labels. labels_out[i] = -1 for noise, otherwise the smallest input
 * index of a core point of i's cluster. Core points and noise are unique;
 * a border point's cluster is any valid one.
 *
 * Conventions for every entry point:
 *   - All functions are extern "C" and return dbscan_status (0 = OK).
 *   - Arguments are checked before anything is enqueued; on error nothing is
 *     enqueued and dbscan_last_error() holds a message (per host thread).
 *   - Device pointers are owned by the caller, who keeps them alive until the
 *     work on the stream (or the server job) has completed.
 *   - Work is enqueued on the given stream (0 = the legacy default stream).
 *     The library owns its device workspaces, one per (device, stream),
 *     grown on demand and freed by dbscan_release_workspaces().
 *   - Sizes: 0 <= n < 2^30 points; 2 <= dim <= 8 (the paper's 2D and 3D
 *     sets and its higher-dimensional ones, Table 1; batches: 2 or 3);
 *     eps > 0 and finite; min_pts >= 1.
 */
#ifndef GBDBSCAN_H
#define GBDBSCAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DBSCAN_OK = 0,
    DBSCAN_ERR_INVALID_ARG = 1,   /* a bad pointer, size or parameter */
    DBSCAN_ERR_OOM = 2,           /* device or host allocation failed */
    DBSCAN_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    DBSCAN_ERR_NONFINITE = 4,     /* an input coordinate is NaN or infinite */
    DBSCAN_ERR_DEVICE_TIMEOUT = 5,/* a bounded device-side wait gave up */
    DBSCAN_ERR_BUSY = 6,          /* server: no slot or budget free (try later) */
    DBSCAN_ERR_NOT_FOUND = 7      /* server: unknown job id */
} dbscan_status;

typedef enum { DBSCAN_MODE_DBSCAN = 0, DBSCAN_MODE_DBSCAN_STAR = 1 } dbscan_mode;
/* DBSCAN_ALGO_AUTO chooses per call (dbscan_run, dbscan_run_host,
 * dbscan_run_multi; not batches) from 2048 sample points and the DenseBox
 * grid (cells of side eps/sqrt(d)): DenseBox when the estimated share of
 * points in cells of >= minPts points, or the estimated mean number of points
 * in a point's cell, reaches its threshold (dbscan_set_auto_threshold), else
 * FDbscan -- DenseBox pays off on data with dense regions (Sec. 5.1, 6). */
typedef enum { DBSCAN_ALGO_FDBSCAN = 0, DBSCAN_ALGO_DENSEBOX = 1, DBSCAN_ALGO_AUTO = 2 } dbscan_algo;

/* opaque CUDA stream (cudaStream_t) */
typedef void* dbscan_stream;

/*
 * Cluster n points (Sec. 3.2 Algorithm 3 with the index of Sec. 4.1 for
 * algo = FDBSCAN, or of Sec. 4.2 for algo = DENSEBOX).
 *   points      device, n*dim fp32, row-major (point i at points[i*dim..]).
 *   labels_out  device, n int32: canonical label or -1 (see above).
 *   core_out    device, n bytes (1 = core point) or NULL.
 * The call enqueues the whole pipeline on `stream` and returns without
 * waiting for the device (the grid of Sec. 4.2, the sort's key width and the
 * automatic algorithm choice are all decided on the device). The caller keeps
 * points and labels_out alive until the stream has finished the work. Argument
 * errors are returned before anything is enqueued. The only host wait is the
 * growth of the stream's workspace (the first call, or a larger n): it waits
 * for the stream before reallocating. Errors found on the device -- a
 * non-finite coordinate (DBSCAN_ERR_NONFINITE; labels_out is then not
 * written) or a radix-sort wait that gave up (DBSCAN_ERR_DEVICE_TIMEOUT) --
 * are reported by the next host sync point on the stream:
 * dbscan_stream_status(), dbscan_run_host(), dbscan_run_sync().
 */
dbscan_status dbscan_run(const float* points, int64_t n, int dim, float eps, int min_pts,
                         int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                         dbscan_stream stream);

/*
 * dbscan_run, then a wait for `stream` and the run's device-side status:
 * errors found on the device (above) are returned by this call.
 */
dbscan_status dbscan_run_sync(const float* points, int64_t n, int dim, float eps, int min_pts,
                              int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                              dbscan_stream stream);

/*
 * The same clustering on host buffers: copies points to the device, runs
 * dbscan_run, copies labels (and core flags if core_out != NULL) back and
 * waits for completion; device-side errors of the run are returned. Host
 * buffers may be pageable or pinned (pinned is faster). Uses a library-owned
 * device staging area per stream.
 */
dbscan_status dbscan_run_host(const float* points_host, int64_t n, int dim, float eps, int min_pts,
                              int mode, int algo, int32_t* labels_host, uint8_t* core_host,
                              dbscan_stream stream);

/*
 * dbscan_run_host without the wait (Sec. 3.2 Algorithm 3, index of Sec. 4.1
 * or 4.2, as dbscan_run): enqueues on `stream` the copy of the points into
 * the stream's staging area, the clustering and the copies of the labels (and
 * core flags) into the host buffers, and returns. Host buffers must be
 * page-locked (cudaHostAlloc, cudaHostRegister, torch pin_memory), so that
 * the copies are asynchronous and overlap the work of other streams: steps
 * enqueued alternately on two streams keep the host link and the kernels busy
 * at once. The caller owns the buffers, keeps them alive and reads the
 * results only after the stream has finished (cudaStreamSynchronize, an
 * event, or dbscan_stream_status, which also returns the run's device-side
 * errors, as for dbscan_run). Calls on one stream reuse its staging area in
 * stream order. Argument errors, and pageable host buffers, are returned
 * (DBSCAN_ERR_INVALID_ARG) before anything is enqueued; like dbscan_run, the
 * call waits only for workspace growth and the autotuner's first call of a
 * kind.
 */
dbscan_status dbscan_run_host_async(const float* points_host, int64_t n, int dim, float eps, int min_pts,
                                    int mode, int algo, int32_t* labels_host, uint8_t* core_host,
                                    dbscan_stream stream);

/*
 * Cluster `count` independent instances in one call (the batched workload).
 *   points      device, concatenated instances; instance b is the rows
 *               offsets[b] .. offsets[b+1]-1 of dims[b] floats each, i.e. its
 *               first coordinate is at points + coord_offsets[b], where
 *               coord_offsets[b] = sum_{c<b} (offsets[c+1]-offsets[c])*dims[c].
 *   offsets     host, count+1 int64 row offsets (offsets[0] = 0, non-decreasing).
 *   dims, eps, min_pts   host, per instance (dims 2 or 3).
 *   labels_out  device, offsets[count] int32; instance b's labels (relative to
 *               the instance: 0 .. n_b-1, or -1) at labels_out + offsets[b].
 *   core_out    device, offsets[count] bytes or NULL.
 * Results are identical to calling dbscan_run per instance.
 */
dbscan_status dbscan_run_batch(const float* points, const int64_t* offsets, const int32_t* dims,
                               const float* eps, const int32_t* min_pts, int32_t count, int mode,
                               int algo, int32_t* labels_out, uint8_t* core_out, dbscan_stream stream);

/*
 * Several minPts over one index (a sweep): for each k < count, writes to
 * labels_out + k*n (and core_out + k*n if core_out is not NULL) exactly what
 * dbscan_run(points, n, dim, eps, min_pts[k], mode, algo, ...) writes (core
 * flags and core labels identical; border labels valid). The index is built
 * once and the neighbour counts are taken once, stopping at the largest
 * minPts instead of each one -- the case the paper names as the exception to
 * early termination (Sec. 3.2); each minPts then runs its own main phase.
 *   min_pts     host, count values >= 1 (any order, repeats allowed).
 *   labels_out  device, count*n int32; core_out device, count*n bytes or NULL.
 * 0 <= count <= 4096; count == 0 or n == 0 returns DBSCAN_OK with no work.
 * Errors as dbscan_run (checked for every min_pts before any work).
 */
dbscan_status dbscan_run_multi(const float* points, int64_t n, int dim, float eps, const int32_t* min_pts,
                               int32_t count, int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                               dbscan_stream stream);

/*
 * Point sets larger than device memory (out-of-core, one GPU; the paper names
 * this as future work, Sec. 6): points and outputs in HOST memory. The set is
 * cut along its widest axis into slabs of at most slab_points points (0: 2^26;
 * a slab is whole bins of 1/65536 of the extent, so one dense bin may exceed
 * it); each slab is clustered on the device with the points within eps of it,
 * twice (exact core flags, then clusters with every point's flag from its own
 * slab), and clusters that meet across slabs are merged on the host.
 * Results as dbscan_run_host (core flags and core labels identical, border
 * labels valid), for n < 2^31; device memory holds one slab at a time.
 *   core_host   host, n bytes (required: the merge uses the core flags).
 * DBSCAN_ERR_INVALID_ARG as dbscan_run, or when a slab with its halo would
 * hold 2^30 points or more; DBSCAN_ERR_NONFINITE for NaN/Inf coordinates.
 * Synchronous: returns when the outputs are written.
 */
dbscan_status dbscan_run_slabs(const float* points_host, int64_t n, int dim, float eps, int min_pts, int mode,
                               int algo, int32_t* labels_host, uint8_t* core_host, int64_t slab_points,
                               dbscan_stream stream);

/*
 * Serving: a request loop that admits clustering jobs as they arrive, by a
 * device-memory budget and a slot limit, and runs admitted jobs concurrently
 * on their own streams. Jobs keep their device state until collected.
 *   dbscan_server_create   budget in bytes of device memory for job state;
 *                          max_slots concurrent jobs (streams).
 *   dbscan_server_submit   queues a job; points/labels_out/core_out are device
 *                          pointers the caller keeps alive until the job is
 *                          done. Returns DBSCAN_ERR_INVALID_ARG for bad
 *                          arguments or jobs that can never fit the budget.
 *   dbscan_server_poll     done_out = 1 once labels are complete; latency is
 *                          seconds from submit to completion (0 while running).
 *                          A finished job's status is returned by poll/wait.
 *   dbscan_server_wait     blocks until the job is done.
 *   dbscan_server_release  forgets a finished job (frees its id).
 *   dbscan_server_destroy  drains all jobs, then frees everything.
 *   dbscan_server_set_batching  continuous batching: a slot that takes a job
 *                          of at most max_job_points points also takes the
 *                          later queued jobs of at most that size with the
 *                          same mode and algo, up to max_batch_points points
 *                          and max_batch_jobs jobs, and runs them as one
 *                          fused batch (as dbscan_run_batch; results are the
 *                          same as running each job alone). max_job_points
 *                          = 0 turns it off. Defaults: 2^18, 2^24, 4096.
 *                          Returns DBSCAN_ERR_INVALID_ARG unless
 *                          0 <= max_job_points <= max_batch_points < 2^31
 *                          and 1 <= max_batch_jobs <= 2^20.
 *   dbscan_server_hold     hold != 0 pauses admission (queued jobs wait;
 *                          running ones finish), 0 resumes it. Destroy
 *                          resumes it before draining.
 *   dbscan_server_stats    out4[0..3] = jobs completed, jobs run alone,
 *                          fused batches run, jobs run inside them.
 * The paper's method has no serving layer; this is the framework's.
 */
typedef struct dbscan_server dbscan_server;
dbscan_status dbscan_server_create(size_t hbm_budget_bytes, int max_slots, dbscan_server** out);
dbscan_status dbscan_server_submit(dbscan_server* srv, const float* points, int64_t n, int dim, float eps,
                                   int min_pts, int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                                   uint64_t* job_id_out);
dbscan_status dbscan_server_poll(dbscan_server* srv, uint64_t job_id, int* done_out, double* latency_s_out);
dbscan_status dbscan_server_wait(dbscan_server* srv, uint64_t job_id);
dbscan_status dbscan_server_release(dbscan_server* srv, uint64_t job_id);
dbscan_status dbscan_server_destroy(dbscan_server* srv);
dbscan_status dbscan_server_set_batching(dbscan_server* srv, int64_t max_job_points, int64_t max_batch_points,
                                         int max_batch_jobs);
dbscan_status dbscan_server_hold(dbscan_server* srv, int hold);
dbscan_status dbscan_server_stats(dbscan_server* srv, int64_t* out4);

/* Status of the work enqueued by this library on `stream` since the last
 * status was taken: waits for the stream, then returns DBSCAN_ERR_NONFINITE if
 * a run met a NaN or infinite coordinate, DBSCAN_ERR_DEVICE_TIMEOUT if a
 * bounded device-side wait gave up (a run that met either wrote no labels),
 * else DBSCAN_OK; clears the recorded errors. */
dbscan_status dbscan_stream_status(dbscan_stream stream);

/* Frees every cached device workspace (waits for their streams first). */
dbscan_status dbscan_release_workspaces(void);

/* Message of the last error returned on this host thread ("" if none). */
const char* dbscan_last_error(void);

/*
 * Tuning knobs (process-wide): traversal block size in threads (a multiple of
 * 32 up to 1024) and the DenseBox cell-side factor f in (0, 1] (cell side
 * f*eps/sqrt(dim); Sec. 4.2 uses f = 1). Results do not depend on them.
 * 0 = autotune (the default for both): the first dbscan_run,
 * dbscan_run_sync, dbscan_run_host or dbscan_run_batch call of each kind --
 * dimension, ceil(log2 n), minPts, algorithm and mode (and ceil(log2 count)
 * for batches) -- measures block sizes {64, 128, 256} x factors
 * {1, 0.75, 0.5} (FDbscan: block sizes only; a fixed knob keeps its value)
 * on the caller's own data, a few runs each, keeps the fastest in a table
 * and uses it for every later call of that kind. That first call waits for
 * the stream (like workspace growth) and returns device-side errors at once;
 * later calls do not wait. The server, dbscan_run_multi and
 * dbscan_run_slabs use the table's entry when there is one, else block 128
 * and f = 1, and never measure.
 */
dbscan_status dbscan_set_tuning(int block_size, float cell_factor);

/*
 * The autotuner's entry for a kind of call (batch = 0: dbscan_run with dim,
 * n, min_pts; batch = 1: dbscan_run_batch with n = total points, min_pts =
 * the largest, count instances): block size, cell factor and the measured
 * milliseconds per call (ms_out may be NULL). DBSCAN_ERR_NOT_FOUND when that
 * kind has not been tuned. dbscan_tuning_clear() empties the table.
 */
dbscan_status dbscan_tuning_lookup(int batch, int dim, int64_t n, int min_pts, int mode, int algo, int64_t count,
                                   int* block_out, float* cell_factor_out, float* ms_out);
dbscan_status dbscan_tuning_clear(void);

/*
 * How border points join a cluster in DBSCAN mode (Sec. 3.2, Algorithm 3:
 * a core point x within eps of a non-core point y claims y, CAS(labels[y], y,
 * find(x))). Process-wide; set it before enqueueing work.
 *   on = 0: the claims are made in the main traversal as core points find
 *     their non-core neighbours; no per-point neighbour list is stored, so
 *     the memory is O(n) whatever minPts (Sec. 3.2).
 *   on = 1 (default): for 3 <= minPts <= 32, preprocessing keeps each
 *     point's neighbours outside its tile in a list of minPts - 1 entries
 *     (4 (minPts - 1) bytes per point: 604 MB for 2^24 points at minPts 10);
 *     a point that ends non-core then claims its first core neighbour from
 *     the list, and non-core points take no part in the main traversal.
 * Both give a valid border label (one of its core neighbours' clusters) and
 * identical core points, core labels and noise. dbscan_border_lists()
 * returns the current setting.
 */
dbscan_status dbscan_set_border_lists(int on);
int dbscan_border_lists(void);

/*
 * Automatic algorithm choice (DBSCAN_ALGO_AUTO) for data of dimension dim
 * (2 to 8): DenseBox when the estimated share of points in dense cells is at
 * least dense_fraction (in [0, 1]) or the estimated mean cell occupancy is at
 * least occupancy (finite, >= 0), else FDbscan. Defaults: 3D 0.005 and 16
 * (FDbscan's 30-bit Morton grid is coarser than eps there; the same above
 * 3D), 2D 0.3 and 16.
 * Both arguments negative restore the defaults for dim.
 * DBSCAN_ERR_INVALID_ARG otherwise.
 */
dbscan_status dbscan_set_auto_threshold(int dim, float dense_fraction, float occupancy);

/*
 * The algorithm the last clustering call on `stream` used (DBSCAN_ALGO_FDBSCAN
 * or DBSCAN_ALGO_DENSEBOX; -1 before any) and, if it was chosen automatically,
 * the estimates behind the choice in estimates_out[0..1]: the share of points
 * in dense cells and the mean cell occupancy (both -1 otherwise). An
 * automatic choice is made on the device: the call then waits for `stream`
 * to read it.
 */
dbscan_status dbscan_last_choice(dbscan_stream stream, int* algo_out, float* estimates_out);

/* ---------------------------------------------------------------------------
 * Instrumentation (not part of the method; for measurement)
 * ------------------------------------------------------------------------- */

/* Stages of one dbscan_run, in order: bounds, keys, sort, gather, leaves
 * (DenseBox cells / tiles), lbvh (leaf boxes, topology, refit), init,
 * preprocess, main, finalize. */
#define DBSCAN_PROFILE_STAGES 10

/* Process-wide switch: when on, every dbscan_run records a CUDA event pair
 * around each stage on its stream (a few microseconds of overhead per run). */
dbscan_status dbscan_profile_enable(int on);

/* Waits for `stream`, then adds up the recorded stage times since the last
 * collect: ms_out[DBSCAN_PROFILE_STAGES] milliseconds per stage and
 * launches_out[DBSCAN_PROFILE_STAGES] (or NULL) the number of stage
 * executions. Clears the records. */
dbscan_status dbscan_profile_collect(dbscan_stream stream, double* ms_out, int64_t* launches_out);

/* Name of stage i ("" if out of range). */
const char* dbscan_profile_stage_name(int stage);

/* Number of CUDA kernels this library has launched since it was loaded. */
int64_t dbscan_kernel_launches(void);

/* Traversal counters, for measurement (the paper has no counterpart). Only a
 * library built with -DGBD_COUNTERS counts (the product build returns
 * DBSCAN_ERR_NOT_FOUND). Waits for the device, writes out[phase * 4 + kind]
 * summed since the last call and zeroes them: phase 0 = per-leaf index
 * lists, 1 = preprocessing, 2 = main phase (intra-tile and traversal);
 * kind 0 = point-to-point distance tests (per lane), 1 = point- and
 * box-to-box tests (per lane), 2 = node visits and 3 = leaf visits (per
 * warp). cap >= 12. */
dbscan_status dbscan_traversal_counters(uint64_t* out, int cap);

/* Test hooks of the radix sort's bounded look-back wait (the paper has no
 * counterpart; they exist to exercise the timeout path without a fault):
 * every later sort waits at most wait_limit polls (negative: the default,
 * about 2^22 polls), and with stall_first_tile != 0 the first tile of each
 * pass publishes nothing, so that every other tile's wait runs out. The sort
 * then reports DBSCAN_ERR_DEVICE_TIMEOUT, its timed-out tiles write nothing,
 * and no stage after it runs. Process-wide; restore with (-1, 0). */
dbscan_status dbscan_test_sort_hooks(int64_t wait_limit, int stall_first_tile);

/* Statistics of the last dbscan_run on `stream` (waits for it):
 * stats_out[0] = number of BVH leaves m, stats_out[1] = number of dense cells
 * (DenseBox; 0 for FDBSCAN). */
dbscan_status dbscan_last_stats(dbscan_stream stream, int64_t* stats_out);

/* ---------------------------------------------------------------------------
 * Component entry points: the individual stages of the pipeline, exposed so
 * that each can be used and tested on its own. All are asynchronous on
 * `stream` and take device pointers.
 * ------------------------------------------------------------------------- */

/*
 * Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits of
 * the 64-bit keys (9-bit digits, one decoupled look-back pass per digit;
 * the ordering of Morton codes in Sec. 4.1). keys/values are sorted in
 * place; n < 2^30.
 */
dbscan_status dbscan_sort_pairs_u64(uint64_t* keys, uint32_t* values, int64_t n, int key_bits,
                                    dbscan_stream stream);

/*
 * dbscan_sort_pairs_u64 for callers that cannot allocate device memory. Some
 * callers may not call cudaMalloc: a real-time loop, because an allocation
 * can synchronise the device or fail at a moment the loop cannot absorb; an
 * application or framework that hands all of the GPU's memory to its own
 * pool or budget, so that memory taken behind the pool's back is not
 * accounted for and can push the process out of memory. The paper has no
 * counterpart; this is an interface convenience of this library.
 *   Same arguments, results and errors as dbscan_sort_pairs_u64, for
 *   n <= DBSCAN_SORT_NOALLOC_MAX_PAIRS (larger n: DBSCAN_ERR_INVALID_ARG,
 *   nothing enqueued). The caller owns keys and values (device).
 *   Its scratch is a fixed static device array of about 14 MB, held by every
 *   GPU that loads the library until the process exits; the call makes no
 *   cudaMalloc/cudaFree or other allocating call.
 *   All calls share that array and it keeps the last call's contents: each
 *   call clears the parts that must start at zero. Calls that overlap on the
 *   GPU (other streams or host threads) race on it and give wrong results;
 *   the caller must serialise them.
 *   The first call in each CUDA context of a device looks up the array's
 *   address (cudaGetSymbolAddress, with that device current) and keeps it
 *   for that context; make that first call before any stream capture. Like
 *   dbscan_sort_pairs_u64 it waits for the stream at the end to report the
 *   sort's bounded-wait status.
 */
#define DBSCAN_SORT_NOALLOC_MAX_PAIRS (1 << 20)
dbscan_status dbscan_sort_pairs_u64_noalloc(uint64_t* keys, uint32_t* values, int64_t n, int key_bits,
                                            dbscan_stream stream);

/*
 * Morton codes (Sec. 4.1): each coordinate is mapped to an integer cell of a
 * 2^bits-per-axis grid over [lo, hi] of that axis (cell = floor((x-lo) *
 * (2^bits / (hi-lo))) clamped to [0, 2^bits-1]; 0 where hi == lo) and the
 * cell indices are bit-interleaved with axis 0 in the lowest bit.
 * dim*bits <= 64. lo/hi are host arrays of dim floats.
 */
dbscan_status dbscan_morton_codes(const float* points, int64_t n, int dim, const float* lo,
                                  const float* hi, int bits, uint64_t* codes_out, dbscan_stream stream);

/*
 * Karras linear BVH topology (Sec. 4.1) over m >= 2 leaves with sorted keys
 * (equal keys are ordered by leaf index). Internal node i (0 <= i < m-1) gets
 * children_out[2i], children_out[2i+1] (a child c >= m-1 is leaf c-(m-1),
 * otherwise internal node c), and range_out[2i], range_out[2i+1] = the first
 * and last leaf index it covers. Node 0 is the root.
 */
dbscan_status dbscan_lbvh_topology(const uint64_t* leaf_keys, int64_t m, int32_t* children_out,
                                   int32_t* range_out, dbscan_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GBDBSCAN_H */
