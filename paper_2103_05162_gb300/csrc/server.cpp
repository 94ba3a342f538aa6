// Serving: a request loop that admits DBSCAN jobs as they arrive, against a
// device-memory budget and a slot limit, and runs the admitted jobs
// concurrently, each on the stream of its slot. A slot keeps its device
// workspace (sorted points, BVH, union-find) between jobs, so device memory
// is allocated once per slot, not per request.
//
// Admission is first-come first-served among the jobs that fit: a slot that
// becomes idle takes the first queued job whose planned workspace, added to
// those of the running jobs, stays within the budget. A job larger than the
// whole budget is rejected at submission.
//
// Continuous batching (the rule is in admission.h): when the job a slot takes
// is small, the slot also takes the later queued small jobs with the same
// mode and algorithm, within the batch limits and the budget, and runs them
// as one fused batch (one sort, one BVH with a subtree per job, one clustering
// pass). Each job's points and outputs stay in the caller's buffers. Jobs
// pulled forward this way only start earlier; none is held back to wait for
// others. If the fused run fails, its jobs are run one by one so that each
// gets its own status.
#include <chrono>
#include <condition_variable>
#include <iterator>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "admission.h"
#include "capi_internal.h"

using namespace gbd;

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id;
    const float* points;
    int64_t n;
    int dim;
    float eps;
    int min_pts;
    int mode;
    int algo;
    int32_t* labels;
    uint8_t* core;
    bool mergeable;  // batches take 2D/3D and an explicit algorithm: other jobs run alone
    size_t bytes;
    Clock::time_point t_submit, t_done;
    bool done = false;
    dbscan_status status = DBSCAN_OK;
};

}  // namespace

struct dbscan_server {
    size_t budget = 0;
    size_t used = 0;
    int device = 0;
    MergeLimits lim;  // continuous batching limits (job_points = 0: off)
    bool hold = false;  // admission paused (queued jobs wait)
    // counters: jobs completed, single runs, fused batches, jobs run in them
    int64_t n_done = 0, n_single = 0, n_batches = 0, n_batched_jobs = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::list<Job*> queue;  // erasing keeps the other iterators valid
    std::map<uint64_t, Job*> jobs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    uint64_t next_id = 1;
    bool stop = false;

    size_t pick_locked(std::vector<Job*>& group)
    {
        return pick_group(queue, group, used, budget, lim, [&](int64_t pts, int count) {
            // list capacity of the largest minPts a batch can have
            return batch_workspace_bytes(pts, count, group[0]->algo, list_cap_max());
        });
    }

    dbscan_status run_single(Workspace* w, Job* j, cudaStream_t s)
    {
        if (!w) return DBSCAN_ERR_CUDA;
        t_run = resolve_tuning(tune_key(0, j->dim, j->n, j->min_pts, j->algo, j->mode, 0));
        dbscan_status st =
            run_pipeline(w, j->points, j->n, j->dim, j->eps, j->min_pts, j->mode, j->algo, j->labels, j->core, s);
        const dbscan_status ds = workspace_status(w, s);
        return st != DBSCAN_OK ? st : ds;
    }

    dbscan_status run_group(Workspace* w, const std::vector<Job*>& g, cudaStream_t s)
    {
        if (!w) return DBSCAN_ERR_CUDA;
        const int count = (int)g.size();
        std::vector<int64_t> offs((size_t)count + 1, 0);
        std::vector<const float*> pts((size_t)count);
        std::vector<int32_t> dims((size_t)count), mps((size_t)count);
        std::vector<float> eps((size_t)count);
        std::vector<int32_t*> labels((size_t)count);
        std::vector<uint8_t*> cores((size_t)count);
        for (int b = 0; b < count; ++b) {
            const Job* j = g[b];
            offs[b + 1] = offs[b] + j->n;
            pts[b] = j->points;
            dims[b] = j->dim;
            eps[b] = j->eps;
            mps[b] = j->min_pts;
            labels[b] = j->labels;
            cores[b] = j->core;
        }
        int max_mp = 1;
        for (int b = 0; b < count; ++b) max_mp = mps[b] > max_mp ? mps[b] : max_mp;
        t_run = resolve_tuning(tune_key(1, 0, offs[count], max_mp, g[0]->algo, g[0]->mode, count));
        dbscan_status st = run_batch(w, count, offs.data(), pts.data(), dims.data(), eps.data(), mps.data(),
                                     labels.data(), cores.data(), g[0]->mode, g[0]->algo, s);
        const dbscan_status ds = workspace_status(w, s);
        return st != DBSCAN_OK ? st : ds;
    }

    void worker(int slot)
    {
        cudaSetDevice(device);
        cudaStream_t s = streams[slot];
        Workspace* w = get_workspace(s);
        std::vector<Job*> group;
        for (;;) {
            size_t bytes = 0;
            group.clear();
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || (!hold && (bytes = pick_locked(group)) != 0); });
                if (group.empty()) return;  // stopping and nothing admissible left
                used += bytes;
            }
            std::vector<dbscan_status> st(group.size(), DBSCAN_OK);
            bool fused = false;
            if (group.size() == 1) {
                st[0] = run_single(w, group[0], s);
            } else {
                const dbscan_status gs = run_group(w, group, s);
                if (gs == DBSCAN_OK) {
                    fused = true;
                } else {
                    for (size_t k = 0; k < group.size(); ++k) st[k] = run_single(w, group[k], s);
                }
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                used -= bytes;
                const Clock::time_point t = Clock::now();
                for (size_t k = 0; k < group.size(); ++k) {
                    group[k]->status = st[k];
                    group[k]->t_done = t;
                    group[k]->done = true;
                }
                n_done += (int64_t)group.size();
                if (fused) {
                    n_batches += 1;
                    n_batched_jobs += (int64_t)group.size();
                } else {
                    n_single += (int64_t)group.size();
                }
            }
            cv.notify_all();
        }
    }
};

extern "C" {

dbscan_status dbscan_server_create(size_t hbm_budget_bytes, int max_slots, dbscan_server** out)
{
    if (!out || max_slots < 1 || max_slots > 256 || hbm_budget_bytes == 0)
        return set_error(DBSCAN_ERR_INVALID_ARG, "need out != NULL, 1 <= max_slots <= 256, budget > 0");
    dbscan_server* srv = new dbscan_server();
    srv->budget = hbm_budget_bytes;
    cudaGetDevice(&srv->device);
    for (int i = 0; i < max_slots; ++i) {
        cudaStream_t s;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t t : srv->streams) cudaStreamDestroy(t);
            delete srv;
            return cuda_error(e, "cudaStreamCreateWithFlags");
        }
        srv->streams.push_back(s);
    }
    for (int i = 0; i < max_slots; ++i) srv->workers.emplace_back(&dbscan_server::worker, srv, i);
    *out = srv;
    return DBSCAN_OK;
}

dbscan_status dbscan_server_set_batching(dbscan_server* srv, int64_t max_job_points, int64_t max_batch_points,
                                         int max_batch_jobs)
{
    if (!srv) return set_error(DBSCAN_ERR_INVALID_ARG, "null server");
    if (max_job_points < 0 || max_batch_points < max_job_points || max_batch_points >= (int64_t(1) << 31) ||
        max_batch_jobs < 1 || max_batch_jobs > (1 << 20))
        return set_error(DBSCAN_ERR_INVALID_ARG,
                         "need 0 <= max_job_points <= max_batch_points < 2^31 and 1 <= max_batch_jobs <= 2^20");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->lim.job_points = max_job_points;
    srv->lim.batch_points = max_batch_points;
    srv->lim.batch_jobs = max_batch_jobs;
    return DBSCAN_OK;
}

dbscan_status dbscan_server_hold(dbscan_server* srv, int hold)
{
    if (!srv) return set_error(DBSCAN_ERR_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->hold = hold != 0;
    }
    srv->cv.notify_all();
    return DBSCAN_OK;
}

dbscan_status dbscan_server_stats(dbscan_server* srv, int64_t* out4)
{
    if (!srv || !out4) return set_error(DBSCAN_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    out4[0] = srv->n_done;
    out4[1] = srv->n_single;
    out4[2] = srv->n_batches;
    out4[3] = srv->n_batched_jobs;
    return DBSCAN_OK;
}

dbscan_status dbscan_server_submit(dbscan_server* srv, const float* points, int64_t n, int dim, float eps,
                                   int min_pts, int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                                   uint64_t* job_id_out)
{
    if (!srv || !job_id_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null server or job id pointer");
    dbscan_status st = check_run_args(points, n, dim, eps, min_pts, mode, algo, labels_out);
    if (st != DBSCAN_OK) return st;
    const size_t bytes = n > 0 ? workspace_bytes(n, dim, algo, min_pts, mode) : 0;
    if (bytes > srv->budget)
        return set_error(DBSCAN_ERR_INVALID_ARG, "job needs %zu bytes of device memory, above the budget of %zu",
                         bytes, srv->budget);
    Job* j = new Job();
    j->points = points;
    j->n = n;
    j->dim = dim;
    j->eps = eps;
    j->min_pts = min_pts;
    j->mode = mode;
    j->algo = algo;
    j->labels = labels_out;
    j->core = core_out;
    j->mergeable = algo != DBSCAN_ALGO_AUTO && dim <= 3;
    j->bytes = bytes;
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) {
            delete j;
            return set_error(DBSCAN_ERR_INVALID_ARG, "server is shutting down");
        }
        j->id = srv->next_id++;
        srv->jobs[j->id] = j;
        if (n == 0) {
            j->done = true;
            j->t_done = j->t_submit;
        } else {
            srv->queue.push_back(j);
        }
        *job_id_out = j->id;
    }
    srv->cv.notify_all();
    return DBSCAN_OK;
}

dbscan_status dbscan_server_poll(dbscan_server* srv, uint64_t job_id, int* done_out, double* latency_s_out)
{
    if (!srv || !done_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return set_error(DBSCAN_ERR_NOT_FOUND, "unknown job %llu", (unsigned long long)job_id);
    Job* j = it->second;
    *done_out = j->done ? 1 : 0;
    if (latency_s_out)
        *latency_s_out = j->done ? std::chrono::duration<double>(j->t_done - j->t_submit).count() : 0.0;
    return j->done ? j->status : DBSCAN_OK;
}

dbscan_status dbscan_server_wait(dbscan_server* srv, uint64_t job_id)
{
    if (!srv) return set_error(DBSCAN_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return set_error(DBSCAN_ERR_NOT_FOUND, "unknown job %llu", (unsigned long long)job_id);
    Job* j = it->second;
    srv->cv.wait(lk, [&] { return j->done; });
    return j->status;
}

dbscan_status dbscan_server_release(dbscan_server* srv, uint64_t job_id)
{
    if (!srv) return set_error(DBSCAN_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return set_error(DBSCAN_ERR_NOT_FOUND, "unknown job %llu", (unsigned long long)job_id);
    if (!it->second->done) return set_error(DBSCAN_ERR_BUSY, "job %llu is still running", (unsigned long long)job_id);
    delete it->second;
    srv->jobs.erase(it);
    return DBSCAN_OK;
}

dbscan_status dbscan_server_destroy(dbscan_server* srv)
{
    if (!srv) return set_error(DBSCAN_ERR_INVALID_ARG, "null server");
    {
        // drain: wait until every queued job has run
        std::unique_lock<std::mutex> lk(srv->mu);
        srv->hold = false;
        srv->cv.notify_all();
        srv->cv.wait(lk, [&] {
            if (!srv->queue.empty()) return false;
            for (auto& kv : srv->jobs)
                if (!kv.second->done) return false;
            return true;
        });
        srv->stop = true;
    }
    srv->cv.notify_all();
    for (auto& t : srv->workers) t.join();
    for (cudaStream_t s : srv->streams) {
        release_stream_workspace(s);
        cudaStreamDestroy(s);
    }
    for (auto& kv : srv->jobs) delete kv.second;
    delete srv;
    return DBSCAN_OK;
}

}  // extern "C"
