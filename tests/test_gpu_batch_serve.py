"""Batched and served clustering: every instance's result must be what the
oracle gives for that instance alone (core and noise sets and core labels
exactly, border labels within their valid sets)."""
import numpy as np
import pytest

from tests.parity import assert_matches_oracle
from workloads import batch_instances, blobs

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu


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
    """The second call with the same buffers and shapes replays the kept
    graph; its per-instance parameters and points are new."""
    for rnd in range(3):
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
