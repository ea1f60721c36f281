"""The merge tree split over ranks (paper_2211_14969_b300.distributed) on the
CPU, as gloo process groups of 2 and 4 ranks on 127.0.0.1.

Every rank condenses the leaves of its own subtree box with the oracle,
merges them to the box root, and the roots' [T | h] go through the real
exchange (torch.distributed gather / scatter of distributed.TorchExchange);
rank 0 merges the grid of boxes and solves it, the boxes' boundary values
are scattered back, and each rank finishes its box.  The numerical steps are
the oracle's (OracleBackend below), so what is under test is the partition,
the packing of the root maps and the exchange: the distributed solution
must equal the oracle's single-rank hps_upward / hps_downward over the whole
grid to 1e-12 on every leaf.
"""

import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2211_14969_b300 import distributed as D  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def workload(nx=4, ny=4, p=8):
    from paper_2211_14969_b300 import workloads as WL
    w = WL.bumps(p=p, nx=nx, ny=ny, kappa=15.0, seed=3, m=1)
    w.dirichlet = "planewave"
    return w


def oracle_leaf(w, l):
    import oracle.hps_oracle as O
    p = int(w.p[l])
    box = w.boxes()[l]
    x, y = O.leaf_nodes(p, box)
    return O.condense_leaf(p, box, w.coefficients(x, y), w.kappa, w.body_load(x, y).reshape(p * p, -1))


def outer_data(w):
    import oracle.hps_oracle as O
    p = int(w.p[0])
    keys = O.outer_boundary_keys(p, w.nx, w.ny)
    return keys, np.array([[w.dirichlet_data(*O.key_coords(p, k, w.nx, w.ny))] for k in keys])


class OracleBackend:
    """The split's numerical steps done by the oracle (merge_two and the
    level recursions of hps_upward / hps_downward) on host arrays."""

    host = True

    def __init__(self, w, part, rank):
        self.w, self.part, self.rank = w, part, rank
        self.p = int(w.p[0])
        self.leaves = [oracle_leaf(w, int(l)) for l in part.leaves(rank)]

    def local_merge(self, m):
        import oracle.hps_oracle as O
        import torch
        wx0, wy0 = self.part.wx0, self.part.wy0
        self.levels = O.hps_upward(self.p, wx0, wy0, self.leaves)
        root = self.levels[-1][(0, 0)] if self.levels else self.leaves[0]
        return torch.from_numpy(np.hstack([root["T"], root["h"]]))

    def top_merge(self, Th, part, m):
        import oracle.hps_oracle as O
        T, h = Th
        boxes = {}
        for b in range(part.world):
            ix0, iy0 = part.box_origin(b)
            boxes[(ix0, iy0)] = {"T": np.asarray(T[b]), "h": np.asarray(h[b]),
                                 "keys": O.box_keys(self.p, ix0, iy0, part.wx0, part.wy0)}
        sizes = D.merge_sizes(part.nx, part.ny)
        wx, wy = part.wx0, part.wy0
        self.top_levels = []
        for nwx, nwy in sizes[sizes.index((wx, wy)) + 1:]:
            along_x = nwx != wx
            new = {}
            for (ix0, iy0) in sorted(boxes):
                if along_x and (ix0 // wx) % 2 == 0:
                    a, b = boxes[(ix0, iy0)], boxes[(ix0 + wx, iy0)]
                elif not along_x and (iy0 // wy) % 2 == 0:
                    a, b = boxes[(ix0, iy0)], boxes[(ix0, iy0 + wy)]
                else:
                    continue
                kpar = O.box_keys(self.p, ix0, iy0, nwx, nwy)
                rec = O.merge_two(a["keys"], a["T"], a["h"], b["keys"], b["T"], b["h"], kpar)
                rec["keys"] = kpar
                new[(ix0, iy0)] = rec
            boxes, wx, wy = new, nwx, nwy
            self.top_levels.append(new)

    def top_solve(self, g, part, m):
        import oracle.hps_oracle as O
        keys, _ = outer_data(self.w)
        vals = {k: np.asarray(g)[i] for i, k in enumerate(keys)}
        for lev in reversed(self.top_levels):
            for rec in lev.values():
                u3 = rec["S3"] @ np.array([vals[k] for k in rec["k12"]]) + rec["w3"]
                vals.update(zip(rec["k3"], u3))
        out = []
        for b in range(part.world):
            ix0, iy0 = part.box_origin(b)
            out.append(np.array([vals[k] for k in O.box_keys(self.p, ix0, iy0, part.wx0, part.wy0)]))
        return out

    def local_solve(self, ub, m):
        import oracle.hps_oracle as O
        ub = np.asarray(ub).reshape(-1, m)
        keys = O.box_keys(self.p, 0, 0, self.part.wx0, self.part.wy0)
        return O.hps_downward(self.p, self.part.wx0, self.part.wy0, self.levels, self.leaves,
                              dict(zip(keys, ub)))


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = workload()
        part = D.Partition(w.nx, w.ny, world)
        be = OracleBackend(w, part, rank)
        exch = D.TorchExchange(rank, world)
        q_nodes = int(w.p[0]) - 2
        D.split_merge(be, exch, part, rank, q_nodes, 1)
        _, g = outer_data(w)
        sol = D.split_solve(be, exch, part, rank, q_nodes, g if rank == 0 else None, 1)
        q.put((rank, [int(l) for l in part.leaves(rank)],
               [(s["u_b"].copy(), s["u_i"].copy()) for s in sol]))
    finally:
        dist.destroy_process_group()


def reference():
    import oracle.hps_oracle as O
    w = workload()
    p = int(w.p[0])
    leaves = [oracle_leaf(w, l) for l in range(w.n_leaves)]
    levels = O.hps_upward(p, w.nx, w.ny, leaves)
    keys, g = outer_data(w)
    return O.hps_downward(p, w.nx, w.ny, levels, leaves, dict(zip(keys, g)))


def test_partition_boxes_follow_the_merge_schedule():
    # 4 x 4 leaves: (1,1) (2,1) (2,2) (4,2) (4,4)
    assert D.merge_sizes(4, 4) == [(1, 1), (2, 1), (2, 2), (4, 2), (4, 4)]
    p2 = D.Partition(4, 4, 2)
    assert (p2.wx0, p2.wy0, p2.bx, p2.by) == (4, 2, 1, 2)
    assert list(p2.leaves(1)) == [2, 3, 6, 7, 10, 11, 14, 15]
    p4 = D.Partition(4, 4, 4)
    assert (p4.wx0, p4.wy0, p4.bx, p4.by) == (2, 2, 2, 2)
    assert p4.box_origin(3) == (2, 2) and list(p4.leaves(2)) == [8, 9, 12, 13]
    # 64 x 64N leaves (the benchmark's weak-scaling grid): 64 x 64 rank boxes
    for n in (2, 4, 8):
        pn = D.Partition(64, 64 * n, n)
        assert (pn.wx0, pn.wy0, pn.bx, pn.by) == (64, 64, 1, n)
    every = np.sort(np.concatenate([p4.leaves(r) for r in range(4)]))
    assert list(every) == list(range(16))
    with pytest.raises(ValueError):
        D.Partition(4, 4, 3)


@pytest.mark.parametrize("world", [2, 4])
def test_split_merge_and_solve_equal_the_single_rank_tree(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = {}
    for _ in range(world):
        rank, leaves, sol = q.get(timeout=240)
        for l, s in zip(leaves, sol):
            got[l] = s
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    ref = reference()
    assert sorted(got) == list(range(len(ref)))
    worst = 0.0
    for l, r in enumerate(ref):
        ub, ui = got[l]
        for a, b in ((ub, r["u_b"]), (ui, r["u_i"])):
            worst = max(worst, float(np.linalg.norm(a - b) / np.linalg.norm(b)))
    assert worst < 1e-12, worst


def test_bench_rank_view_is_the_rank_box():
    """bench.py's multi-rank workload: rank r condenses the 64 x 64 leaves
    of the stacked grid with y in [r, r+1], in its box's local order."""
    import bench
    w = bench.make_workload("bumps_p20")
    for ws, rank in ((2, 1), (4, 2), (8, 7)):
        v, part = bench.rank_view(w, ws, rank)
        b = v.boxes()
        assert v.n_leaves == 4096 and len(b) == 4096 and (part.wx0, part.wy0) == (64, 64)
        assert np.allclose(b[:, 1].min(), rank) and np.allclose(b[:, 1].max() + b[:, 3].max(), rank + 1)
        assert np.allclose(b[:, :2] - [0.0, rank], w.boxes()[:, :2])     # the single-GPU tiling, shifted
    v0, _ = bench.rank_view(w, 4, 0)
    assert np.array_equal(v0.boxes(), w.boxes())
