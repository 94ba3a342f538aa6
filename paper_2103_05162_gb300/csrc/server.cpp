// Serving: a request loop that admits DBSCAN jobs as they arrive, against a
// device-memory budget and a slot limit, and runs the admitted jobs
// concurrently, each on the stream of its slot. A slot keeps its device
// workspace (sorted points, BVH, union-find) between jobs, so device memory
// is allocated once per slot, not per request.
//
// Admission is first-come first-served among the jobs that fit: a job is
// started when a slot is idle and the sum of the planned workspaces of the
// running jobs plus its own stays within the budget. A job larger than the
// whole budget is rejected at submission.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

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
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;
    std::map<uint64_t, Job*> jobs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    uint64_t next_id = 1;
    bool stop = false;

    // the first queued job that fits the remaining budget, or null
    Job* pick_locked()
    {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            if (used + (*it)->bytes <= budget) {
                Job* j = *it;
                queue.erase(it);
                return j;
            }
        }
        return nullptr;
    }

    void worker(int slot)
    {
        cudaSetDevice(device);
        cudaStream_t s = streams[slot];
        Workspace* w = get_workspace(s);
        for (;;) {
            Job* j = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || (j = pick_locked()) != nullptr; });
                if (!j) return;  // stopping and nothing admissible left
                used += j->bytes;
            }
            dbscan_status st = w ? run_pipeline(w, j->points, j->n, j->dim, j->eps, j->min_pts, j->mode, j->algo,
                                                j->labels, j->core, s)
                                 : DBSCAN_ERR_CUDA;
            cudaError_t e = cudaStreamSynchronize(s);
            if (st == DBSCAN_OK && e != cudaSuccess) st = DBSCAN_ERR_CUDA;
            {
                std::lock_guard<std::mutex> lk(mu);
                used -= j->bytes;
                j->status = st;
                j->t_done = Clock::now();
                j->done = true;
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

dbscan_status dbscan_server_submit(dbscan_server* srv, const float* points, int64_t n, int dim, float eps,
                                   int min_pts, int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                                   uint64_t* job_id_out)
{
    if (!srv || !job_id_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null server or job id pointer");
    dbscan_status st = check_run_args(points, n, dim, eps, min_pts, mode, algo, labels_out);
    if (st != DBSCAN_OK) return st;
    const size_t bytes = n > 0 ? workspace_bytes(n, dim, algo) : 0;
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
