"""Batched and served clustering: every instance's result must be what the
oracle gives for that instance alone (core and noise sets and core labels
exactly, border labels within their valid sets)."""
import numpy as np
import pytest

import oracle
from tests.parity import assert_matches_oracle
from workloads import batch_instances, blobs

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu

WAIT_S = 300.0  # a job still queued after this long is a failure, not a hang


def _concat(instances):
    flat = np.concatenate([np.ascontiguousarray(x.points, np.float32).ravel() for x in instances]).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum([x.n for x in instances])]).astype(np.int64)
    return flat, offsets


class _Inst:
    def __init__(self, points, eps, min_pts):
        self.points = np.ascontiguousarray(points, np.float32)
        self.eps = float(np.float32(eps))
        self.min_pts = int(min_pts)
        self.n = self.points.shape[0]
        self.dim = self.points.shape[1] if self.points.ndim == 2 else 3


def _mixed_instances(seed):
    rs = np.random.default_rng(seed)
    out = []
    for i in range(60):
        d = int(rs.choice([2, 3]))
        n = int(rs.choice([0, 1, 2, 31, 33, 500, 3000, 20000])) if i % 5 else int(rs.integers(1, 5000))
        eps = float(rs.uniform(0.01, 0.06))
        mp = int(rs.choice([1, 2, 3, 5, 10]))
        pts = blobs(n, d, int(rs.integers(0, 2**31))) if n else np.zeros((0, d), np.float32)
        out.append(_Inst(pts, eps, mp))
    # duplicates and exact ties
    out.append(_Inst(np.full((100, 3), 0.5, np.float32), 1e-3, 10))
    out.append(_Inst(rs.integers(0, 6, size=(400, 2)).astype(np.float32), 1.0, 4))
    return out


def _check_batch(instances, mode, algo, labels, core):
    offs = np.concatenate([[0], np.cumsum([x.n for x in instances])])
    for b, x in enumerate(instances):
        if x.n == 0:
            continue
        lab = labels[offs[b]:offs[b + 1]]
        cor = core[offs[b]:offs[b + 1]].astype(bool)
        assert_matches_oracle(x.points, x.eps, x.min_pts, mode, lab, cor)


@pytest.mark.parametrize("algo", [gb.ALGO_FDBSCAN, gb.ALGO_DENSEBOX])
@pytest.mark.parametrize("mode", [gb.MODE_DBSCAN, gb.MODE_DBSCAN_STAR])
def test_batch_matches_oracle_per_instance(mode, algo):
    inst = _mixed_instances(10 + mode + 2 * algo)
    flat, offs = _concat(inst)
    pts = torch.from_numpy(flat).cuda()
    total = int(offs[-1])
    labels = torch.empty(total, dtype=torch.int32, device="cuda")
    core = torch.empty(total, dtype=torch.uint8, device="cuda")
    gb.dbscan_run_batch(pts, offs, [x.dim for x in inst], [x.eps for x in inst], [x.min_pts for x in inst],
                        mode=mode, algo=algo, labels_out=labels, core_out=core)
    torch.cuda.synchronize()
    gb.stream_status()
    _check_batch(inst, mode, algo, labels.cpu().numpy(), core.cpu().numpy())


def test_batch_replays_with_new_contents():
    """Calls with the same shapes: the first launches directly, the second
    captures a graph, the later ones replay it -- with new points and
    per-instance parameters each time, and new output buffers in the last."""
    for rnd in range(4):
        rs = np.random.default_rng(100 + rnd)
        inst = [_Inst(blobs(3000, 3 if b % 2 else 2, 1000 * rnd + b), rs.uniform(0.01, 0.05),
                      int(rs.choice([2, 5, 10]))) for b in range(40)]
        flat, offs = _concat(inst)
        if rnd == 0:
            pts = torch.from_numpy(flat).cuda()
            labels = torch.empty(int(offs[-1]), dtype=torch.int32, device="cuda")
            core = torch.empty(int(offs[-1]), dtype=torch.uint8, device="cuda")
        else:
            pts.copy_(torch.from_numpy(flat))
        if rnd == 3:
            labels = torch.full((int(offs[-1]),), -7, dtype=torch.int32, device="cuda")
            core = torch.full((int(offs[-1]),), 9, dtype=torch.uint8, device="cuda")
        gb.dbscan_run_batch(pts, offs, [x.dim for x in inst], [x.eps for x in inst], [x.min_pts for x in inst],
                            algo=gb.ALGO_DENSEBOX, labels_out=labels, core_out=core)
        torch.cuda.synchronize()
        _check_batch(inst, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX, labels.cpu().numpy(), core.cpu().numpy())


def test_batch_of_generated_workload_instances():
    inst = batch_instances(48, 3, size_scale=0.1)
    flat, offs = _concat(inst)
    pts = torch.from_numpy(flat).cuda()
    labels, core = gb.dbscan_run_batch(pts, offs, [x.dim for x in inst], [x.eps for x in inst],
                                       [x.min_pts for x in inst], core_out=torch.empty(int(offs[-1]),
                                                                                      dtype=torch.uint8,
                                                                                      device="cuda"))
    torch.cuda.synchronize()
    _check_batch(inst, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX, labels.cpu().numpy(), core.cpu().numpy())


def test_batch_rejects_nonfinite():
    inst = [_Inst(blobs(100, 3, 1), 0.05, 3), _Inst(blobs(100, 2, 2), 0.05, 3)]
    inst[1].points[7, 1] = np.nan
    flat, offs = _concat(inst)
    with pytest.raises(gb.DbscanError) as e:
        gb.dbscan_run_batch(torch.from_numpy(flat).cuda(), offs, [3, 2], [0.05, 0.05], [3, 3])
    assert e.value.name == "NONFINITE"


# --- serving ------------------------------------------------------------------

def _serve_jobs(seed):
    """A mix of small jobs (merged into fused batches), mid-size ones and a
    few that run alone, in both dimensions, both algorithms and modes."""
    rs = np.random.default_rng(seed)
    jobs = []
    for i in range(48):
        d = int(rs.choice([2, 3]))
        n = int(rs.choice([0, 1, 40, 700, 5000, 20000])) if i % 8 else int(rs.choice([300_000, 400_000]))
        eps = float(np.float32(rs.uniform(0.01, 0.05)))
        mp = int(rs.choice([2, 5, 10]))
        mode = int(rs.choice([gb.MODE_DBSCAN, gb.MODE_DBSCAN_STAR]))
        algo = int(rs.choice([gb.ALGO_FDBSCAN, gb.ALGO_DENSEBOX]))
        pts = blobs(n, d, int(rs.integers(0, 2**31))) if n else np.zeros((0, d), np.float32)
        jobs.append((pts, eps, mp, mode, algo))
    return jobs


def _serve(jobs, batching=True, slots=4, budget=8 << 30, hold=True):
    with gb.Server(budget, max_slots=slots) as srv:
        if not batching:
            srv.set_batching(0, 1 << 24, 4096)
        dev = [(torch.from_numpy(p).cuda(), torch.empty(p.shape[0], dtype=torch.uint8, device="cuda"))
               for p, *_ in jobs]
        torch.cuda.synchronize()
        if hold:
            srv.hold(True)  # queue everything first: merging is then certain
        ids = [srv.submit(x, eps, mp, mode=mode, algo=algo, core_out=c)
               for (x, c), (_, eps, mp, mode, algo) in zip(dev, jobs)]
        srv.hold(False)
        out = []
        for jid, (_, c) in zip(ids, dev):
            lab = srv.wait(jid, timeout=WAIT_S)
            done, lat = srv.poll(jid)
            assert done and lat >= 0.0
            out.append((lab.cpu().numpy(), c.cpu().numpy()))
            srv.release(jid)
        stats = srv.stats()
    return out, stats


def test_server_jobs_match_oracle_and_batch():
    jobs = _serve_jobs(7)
    out, stats = _serve(jobs)
    assert stats["done"] == sum(1 for p, *_ in jobs if p.shape[0] > 0)
    assert stats["batches"] >= 1 and stats["batched_jobs"] >= 2, stats
    for (pts, eps, mp, mode, algo), (lab, cor) in zip(jobs, out):
        if 0 < pts.shape[0] <= 20000:
            assert_matches_oracle(pts, eps, mp, mode, lab, cor)
    # the large jobs: same as the same job run alone through dbscan_run
    for (pts, eps, mp, mode, algo), (lab, cor) in zip(jobs, out):
        if pts.shape[0] > 20000:
            x = torch.from_numpy(pts).cuda()
            c = torch.empty(pts.shape[0], dtype=torch.uint8, device="cuda")
            alone = gb.dbscan_run(x, eps, mp, mode=mode, algo=algo, core_out=c)[0].cpu().numpy()
            np.testing.assert_array_equal(cor, c.cpu().numpy())
            np.testing.assert_array_equal(lab[cor.astype(bool)], alone[cor.astype(bool)])
            np.testing.assert_array_equal(lab == -1, alone == -1)


def test_server_result_same_alone_and_in_mix():
    """A job's core set, core labels and noise set do not depend on which
    jobs it was merged with, nor on whether batching is on."""
    jobs = _serve_jobs(11)
    mixed, st_on = _serve(jobs, batching=True, slots=3)
    single, st_off = _serve(jobs, batching=False, slots=2)
    assert st_on["batches"] >= 1 and st_off["batches"] == 0
    for (pts, *_), (la, ca), (lb, cb) in zip(jobs, mixed, single):
        np.testing.assert_array_equal(ca, cb)
        core = ca.astype(bool)
        np.testing.assert_array_equal(la[core], lb[core])
        np.testing.assert_array_equal(la == -1, lb == -1)


def test_server_budget_admission_and_rejection():
    small = [(blobs(4000, 3, s), 0.03, 5, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX) for s in range(6)]
    # a budget that admits about one small job at a time: jobs queue, all finish
    out, stats = _serve(small, budget=3 << 20, slots=4, hold=False)
    assert stats["done"] == len(small)
    for (pts, eps, mp, mode, algo), (lab, cor) in zip(small, out):
        assert_matches_oracle(pts, eps, mp, mode, lab, cor)
    with gb.Server(1 << 20, max_slots=1) as srv:
        x = torch.from_numpy(blobs(200_000, 3, 1)).cuda()
        with pytest.raises(gb.DbscanError):
            srv.submit(x, 0.03, 5)


def test_server_bad_job_does_not_fail_its_batch():
    good = [(blobs(3000, 2, s), 0.03, 5, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX) for s in range(5)]
    bad = blobs(3000, 2, 99)
    bad[17, 0] = np.nan
    jobs = good[:2] + [(bad, 0.03, 5, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX)] + good[2:]
    with gb.Server(8 << 30, max_slots=1) as srv:
        dev = [torch.from_numpy(p).cuda() for p, *_ in jobs]
        torch.cuda.synchronize()
        srv.hold(True)
        ids = [srv.submit(x, eps, mp, mode=mode, algo=algo) for x, (_, eps, mp, mode, algo) in zip(dev, jobs)]
        srv.hold(False)
        for k, jid in enumerate(ids):
            if k == 2:
                with pytest.raises(gb.DbscanError):
                    srv.wait(jid, timeout=WAIT_S)
            else:
                lab = srv.wait(jid, timeout=WAIT_S).cpu().numpy()
                p, eps, mp, mode, _ = jobs[k]
                olab, ocore = oracle.dbscan(p, eps, mp, mode)
                np.testing.assert_array_equal(lab[ocore], olab[ocore])
