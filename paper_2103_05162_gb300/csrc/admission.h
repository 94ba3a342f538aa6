// Admission rule of the serving loop, host only (no CUDA), so that it can be
// tested without a GPU.
//
// A slot that becomes idle takes the first queued job whose planned device
// bytes, added to those of the running jobs, stay within the budget. If that
// job is small (at most job_points points) it also takes the later queued
// small jobs with the same mode and algorithm, in queue order, while the
// group stays within batch_points points, batch_jobs jobs and the budget
// (with the group's batch workspace in place of the single one). Jobs that
// do not join stay queued in their order.
#pragma once

#include <cstddef>
#include <cstdint>
#include <list>
#include <vector>

namespace gbd {

struct MergeLimits {
    int64_t job_points = int64_t(1) << 18;  // 0: no merging
    int64_t batch_points = int64_t(1) << 24;
    int batch_jobs = 4096;
};

// Job: has n (points), mode, algo, mergeable (false: always runs alone) and
// bytes (planned single-run workspace).
// batch_bytes(points, jobs): planned workspace of a fused batch.
// Moves the chosen jobs from queue to group (in queue order) and returns the
// bytes to reserve for them; returns 0 and leaves both alone if no queued job
// fits.
template <class Job, class BatchBytes>
size_t pick_group(std::list<Job*>& queue, std::vector<Job*>& group, size_t used, size_t budget,
                  const MergeLimits& lim, BatchBytes batch_bytes)
{
    group.clear();
    auto head = queue.end();
    for (auto it = queue.begin(); it != queue.end(); ++it) {
        if (used + (*it)->bytes <= budget) {
            head = it;
            break;
        }
    }
    if (head == queue.end()) return 0;
    Job* h = *head;
    group.push_back(h);
    size_t bytes = h->bytes;
    auto small = [&](const Job* j) { return j->mergeable && lim.job_points > 0 && j->n <= lim.job_points; };
    std::vector<typename std::list<Job*>::iterator> take{head};
    if (small(h)) {
        int64_t pts = h->n;
        for (auto it = std::next(head); it != queue.end() && (int)group.size() < lim.batch_jobs; ++it) {
            Job* j = *it;
            if (!small(j) || j->mode != h->mode || j->algo != h->algo || pts + j->n > lim.batch_points) continue;
            const size_t b = batch_bytes(pts + j->n, (int)group.size() + 1);
            if (used + b > budget) continue;
            group.push_back(j);
            take.push_back(it);
            pts += j->n;
            bytes = b;
        }
    }
    for (auto t : take) queue.erase(t);  // list: the other iterators stay valid
    return bytes;
}

}  // namespace gbd
