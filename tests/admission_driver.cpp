// Drives the serving loop's admission rule (csrc/admission.h) on the host.
// stdin: budget used job_points batch_points batch_jobs per_point per_job
//        njobs, then njobs lines "n mode algo bytes"
// The fused-batch workspace is modelled as per_point * points + per_job * jobs.
// stdout: the bytes reserved, the chosen job indices, the indices left queued.
#include <cstdio>
#include <list>
#include <vector>

#include "admission.h"

struct J {
    int idx;
    long long n;
    int mode, algo;
    bool mergeable;  // algorithm 2 (automatic choice) never merges
    size_t bytes;
};

int main()
{
    unsigned long long budget, used, per_point, per_job;
    long long jp, bp;
    int bj, nj;
    if (scanf("%llu %llu %lld %lld %d %llu %llu %d", &budget, &used, &jp, &bp, &bj, &per_point, &per_job, &nj) != 8)
        return 2;
    std::vector<J> jobs((size_t)nj);
    std::list<J*> queue;
    for (int i = 0; i < nj; ++i) {
        unsigned long long b;
        if (scanf("%lld %d %d %llu", &jobs[i].n, &jobs[i].mode, &jobs[i].algo, &b) != 4) return 2;
        jobs[i].idx = i;
        jobs[i].mergeable = jobs[i].algo != 2;
        jobs[i].bytes = (size_t)b;
        queue.push_back(&jobs[i]);
    }
    gbd::MergeLimits lim;
    lim.job_points = jp;
    lim.batch_points = bp;
    lim.batch_jobs = bj;
    std::vector<J*> group;
    const size_t r = gbd::pick_group(queue, group, (size_t)used, (size_t)budget, lim, [&](long long pts, int count) {
        return (size_t)(per_point * (unsigned long long)pts + per_job * (unsigned long long)count);
    });
    printf("%zu\n", r);
    for (J* j : group) printf("%d ", j->idx);
    printf("\n");
    for (J* j : queue) printf("%d ", j->idx);
    printf("\n");
    return 0;
}
