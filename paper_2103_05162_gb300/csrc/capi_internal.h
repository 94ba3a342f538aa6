// Host-side internals of the C ABI shared by capi.cu, batch.cu and server.cpp.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "gbdbscan.h"

namespace gbd {

struct Arena {
    void* base = nullptr;
    size_t cap = 0;
};

// One per (device, stream): the pipeline's buffers live in `main`; `aux`
// serves the component entry points and `io` the host-buffer entry point.
struct ProfState;

struct Workspace {
    int device = 0;
    cudaStream_t stream = nullptr;
    Arena main, aux, io;
    uint32_t* ctrl_host = nullptr;  // pinned mirror of the control block
    ProfState* prof = nullptr;      // per-stage event records (profiling on)
    // batches: the stream their CUDA graph runs on, and the events that fork
    // it from and join it back to the caller's stream
    cudaStream_t gstream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // the algorithm the last run on this stream used (-1 before any; -2:
    // chosen on the device, read from the control block on request)
    int last_algo = -1;
};

struct Tuning {
    int block;             // traversal block size (threads); 0: chosen by the autotuner
    float cell_factor;     // DenseBox cell side factor f in (0, 1]; 0: chosen by the autotuner
    // border claims (DBSCAN mode): 1 = from preprocessing's per-point
    // neighbour lists, 0 = by core points during the main traversal (no
    // per-point list; Algorithm 3 as written)
    int border_lists;
    // DBSCAN_ALGO_AUTO, per dimension (index 2, 3): DenseBox from this
    // estimated dense-point share up, or from this estimated mean cell
    // occupancy up
    float auto_fraction[9];
    float auto_occupancy[9];
};
// defaults from measurements on GB300: in 3D FDbscan's 10-bit Morton grid is
// coarser than eps and DenseBox wins as soon as a few dense cells exist; in
// 2D FDbscan's 16-bit grid is finer than the DenseBox cells and wins unless
// the data is dense
constexpr float DEFAULT_AUTO_FRACTION_2D = 0.3f, DEFAULT_AUTO_FRACTION_3D = 0.005f;
constexpr float DEFAULT_AUTO_OCCUPANCY = 16.0f;
extern Tuning g_tuning;

// The traversal block size and DenseBox cell factor of the run being
// enqueued on this thread: every entry point sets it (resolve_tuning, or the
// autotuner while it measures) before enqueueing work.
struct RunTuning {
    int block;
    float cell_factor;
};
constexpr RunTuning DEFAULT_RUN_TUNING = {128, 1.0f};
extern thread_local RunTuning t_run;
// Autotuner table keys: one per kind of call (0 dbscan_run, 1 batch), dim
// (0 for batches), ceil(log2 n), minPts (the largest, for batches),
// algorithm, mode and ceil(log2 count) (batches).
struct TuneKey {
    int kind, dim, log2n, min_pts, algo, mode, log2count;
    bool operator<(const TuneKey& o) const;
};
TuneKey tune_key(int kind, int dim, int64_t n, int min_pts, int algo, int mode, int64_t count);
// the fixed knobs, or the table's entry for the key, or the defaults (never measures)
RunTuning resolve_tuning(const TuneKey& k);
bool autotune_on();
bool tuned(const TuneKey& k);
void store_tuning(const TuneKey& k, RunTuning t, float ms);
// the candidates the autotuner measures (fixed knobs restrict them)
int tuning_candidates(int algo, RunTuning* out, int cap);

dbscan_status set_error(dbscan_status st, const char* fmt, ...);
// empties this thread's dbscan_last_error() message (every entry point starts so)
void clear_error();
dbscan_status cuda_error(cudaError_t e, const char* what);
dbscan_status check_run_args(const void* points, int64_t n, int dim, float eps, int min_pts, int mode, int algo,
                             const void* labels_out);
Workspace* get_workspace(cudaStream_t s);
cudaError_t ensure_arena(Arena& a, size_t bytes, cudaStream_t s);
void free_workspace(Workspace* w);
void release_stream_workspace(cudaStream_t s);
// Neighbour lists of preprocessing (DBSCAN mode, 3 <= minPts <= 32, border
// lists switched on): every point keeps up to minPts - 1 of its neighbours
// outside its own tile, which is all of them when it ends non-core; 0 means
// no lists (core points then claim their border neighbours in the main phase).
constexpr int LIST_MAX_MINPTS = 32;
inline int list_cap(int min_pts, int mode)
{
    return (g_tuning.border_lists && mode == DBSCAN_MODE_DBSCAN && min_pts > 2 && min_pts <= LIST_MAX_MINPTS)
               ? min_pts - 1
               : 0;
}
// the list capacity a batch of any minPts may need
inline int list_cap_max() { return g_tuning.border_lists ? LIST_MAX_MINPTS - 1 : 0; }
size_t workspace_bytes(int64_t n, int dim, int algo, int min_pts, int mode);
size_t workspace_bytes_multi(int64_t n, int dim, int algo, int max_min_pts, int mode);
dbscan_status run_pipeline(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int mode,
                           int algo, int32_t* labels_out, uint8_t* core_out, cudaStream_t s);
dbscan_status run_core_flags(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int algo,
                             uint8_t* core_out, int32_t* labels_scratch, cudaStream_t s);
dbscan_status run_with_core(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int mode,
                            int algo, const uint8_t* core_in, int32_t* labels_out, cudaStream_t s);
// host points and outputs, clustered in slabs of at most slab_points points
dbscan_status run_slabs(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int mode,
                        int algo, int32_t* labels, uint8_t* core, int64_t slab_points, cudaStream_t s);
dbscan_status run_multi(Workspace* w, const float* points, int64_t n, int dim, float eps, const int32_t* min_pts,
                        int count, int mode, int algo, int32_t* labels_out, uint8_t* core_out, cudaStream_t s);
// count instances: rows offsets[b]..offsets[b+1]-1 of the concatenation;
// instance b's points, labels and core flags (cores may be null, or an entry
// of it) are separate device buffers
// device bytes run_batch plans for n points in count instances
size_t batch_workspace_bytes(int64_t n, int count, int algo, int lcap);
// waits for s, then returns (and clears) the device error bits of w's arena
dbscan_status workspace_status(Workspace* w, cudaStream_t s);
dbscan_status run_batch(Workspace* w, int32_t count, const int64_t* offsets, const float* const* points,
                        const int32_t* dims, const float* eps, const int32_t* min_pts, int32_t* const* labels,
                        uint8_t* const* cores, int mode, int algo, cudaStream_t s);
void release_batch_graphs(Workspace* w);

}  // namespace gbd
