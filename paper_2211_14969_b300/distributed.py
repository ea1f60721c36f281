"""The HPS merge tree split over ranks: one subtree of leaves per GPU.

Leaf condensation needs no communication (Section 2: the leaf operations
are independent per leaf).  The leaf grid is partitioned into the boxes of
one level of its merge tree, one box (a subtree of leaves) per rank; every
rank condenses its box's leaves and merges them up to the box's root,
including the root's own DtN map and flux [T | h].  The one exchange step:

  1. gather   the boxes' root [T | h] on rank 0;
  2. rank 0   merges the grid of boxes (the tree's top levels) and solves it
              for every box's boundary values from the outer Dirichlet data;
  3. scatter  each box's boundary values back to its rank;
  4. every rank finishes the downward pass and the leaf recovery in its box.

The numerical steps belong to a backend (LibraryBackend: the CUDA library's
hps_merge_boxes / hps_solve_boxes / hps_solve); this module holds the
partition, the packing and the exchange, so the same code runs with NCCL on
GPUs and with gloo on CPUs.  The merge schedule is the library's: x first,
then alternating, a direction continuing alone once the other spans the
grid (power-of-two grids).
"""

import numpy as np


def merge_sizes(nx, ny):
    """Box sizes (wx, wy) in leaves after 0, 1, ... merge levels of an
    nx x ny leaf grid, ending with (nx, ny)."""
    for n in (nx, ny):
        if n < 1 or (n & (n - 1)):
            raise ValueError("the merge tree needs power-of-two leaf counts")
    wx, wy, out = 1, 1, [(1, 1)]
    while wx < nx or wy < ny:
        if wx < nx and (wx <= wy or wy == ny):
            wx *= 2
        else:
            wy *= 2
        out.append((wx, wy))
    return out


class Partition:
    """The rank boxes of an nx x ny leaf grid over `world` ranks (a power of
    two): the boxes of the merge tree log2(world) levels below its root,
    box b = bx * by_count + by, rank r owns box r."""

    def __init__(self, nx, ny, world):
        if world < 1 or (world & (world - 1)):
            raise ValueError("world size must be a power of two")
        sizes = merge_sizes(nx, ny)
        k = world.bit_length() - 1
        if k > len(sizes) - 1:
            raise ValueError(f"{world} ranks exceed the {nx * ny} leaves")
        self.nx, self.ny, self.world = nx, ny, world
        self.wx0, self.wy0 = sizes[len(sizes) - 1 - k]
        self.bx, self.by = nx // self.wx0, ny // self.wy0
        assert self.bx * self.by == world

    def box_origin(self, rank):
        """(ix0, iy0) of rank's box, in leaves."""
        b, c = divmod(rank, self.by)
        return b * self.wx0, c * self.wy0

    def leaves(self, rank):
        """Global leaf indices (ix * ny + iy) of rank's box in its local order
        (local leaf jx * wy0 + jy)."""
        ix0, iy0 = self.box_origin(rank)
        jx, jy = np.meshgrid(np.arange(self.wx0), np.arange(self.wy0), indexing="ij")
        return ((ix0 + jx) * self.ny + (iy0 + jy)).ravel()

    def box_nodes(self, q):
        """Boundary nodes of a rank box (q edge nodes per leaf side)."""
        return 2 * (self.wx0 + self.wy0) * q

    def root_nodes(self, q):
        return 2 * (self.nx + self.ny) * q


class TorchExchange:
    """gather / scatter over a torch.distributed process group (NCCL with
    device tensors, gloo with host tensors); rank 0 is the root."""

    def __init__(self, rank, world, device=None):
        self.rank, self.world, self.device = rank, world, device

    def _t(self, a):
        import torch
        t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
        return t.to(self.device) if self.device is not None else t

    def gather(self, a):
        """Every rank's array (same shape) as a list on rank 0; None elsewhere."""
        import torch
        import torch.distributed as dist
        t = self._t(a).contiguous()
        lst = [torch.empty_like(t) for _ in range(self.world)] if self.rank == 0 else None
        dist.gather(t, lst, dst=0)
        return lst

    def scatter(self, parts, like):
        """Rank 0's list of arrays, one per rank (each shaped like `like`)."""
        import torch
        import torch.distributed as dist
        out = torch.empty_like(self._t(like)).contiguous()
        lst = [self._t(p).contiguous() for p in parts] if self.rank == 0 else None
        dist.scatter(out, lst, src=0)
        return out


def split_merge(backend, exch, part, rank, q, m):
    """Steps 1-2 upward: the rank's subtree merged to its root [T | h],
    gathered on rank 0, which merges the grid of boxes.  Returns the
    rank's root [T | h] (kept for diagnostics)."""
    th = backend.local_merge(m)
    lst = exch.gather(th)
    if rank == 0:
        backend.top_merge(unpack_roots(lst, part.box_nodes(q), m), part, m)
    return th


def split_solve(backend, exch, part, rank, q, g, m):
    """Steps 2-4 downward: rank 0 solves the top levels for the boxes'
    boundary values from the outer Dirichlet data g ([W, E, S, N] order of
    the whole grid, n_root x m), scatters them, and every rank solves its
    box.  Returns the rank's solution from backend.local_solve."""
    nb = part.box_nodes(q)
    parts = backend.top_solve(g, part, m) if rank == 0 else None
    like = np.zeros((nb, m)) if backend.host else backend.zeros((nb, m))
    ub = exch.scatter(parts, like)
    return backend.local_solve(ub, m)


def unpack_roots(ths, nb, m):
    """Stacked root maps and fluxes of the boxes (box order) from their
    [T | h] blocks (nb x (nb + m) each): (T [boxes][nb][nb], h [boxes][nb][m])."""
    T = [th.reshape(nb, nb + m)[:, :nb] for th in ths]
    h = [th.reshape(nb, nb + m)[:, nb:] for th in ths]
    return T, h


class LibraryBackend:
    """The numerical steps on the GPU through the CUDA library: the rank's
    leaf plan (hps_condense, hps_merge_boxes with the root map, hps_solve)
    and, on rank 0, a plan for the grid of boxes (hps_merge_boxes,
    hps_solve_boxes)."""

    host = False

    def __init__(self, p, kappa, part, rank, boxes, plan=None, out=None):
        from . import hps
        self.hps = hps
        self.part, self.rank, self.p, self.kappa = part, rank, int(p), float(kappa)
        self.boxes = np.asarray(boxes, dtype=np.float64)           # the rank's leaf boxes, local order
        self.own = plan is None
        self.plan = plan if plan is not None else hps.Plan(np.full(len(self.boxes), self.p, dtype=np.int32),
                                                             self.boxes, kappa)
        self.top = None
        self.out = out      # the leaves' condensed S, T, h, W (set by condense, or given)

    def zeros(self, shape):
        import torch
        return torch.zeros(shape, dtype=torch.float64, device="cuda")

    def condense(self, coef, f, m, prec="fp64", tol=1e-12, kmax=6, out=None):
        self.out = self.plan.condense(coef, f, m=m, prec=prec, tol=tol, kmax=kmax, out=out)
        return self.out

    def local_merge(self, m):
        return self.plan.merge_boxes(self.part.wx0, self.part.wy0, 1, 1, self.out["T"], self.out.get("h"), m,
                                     root=True)

    def top_merge(self, Th, part, m):
        import torch
        T, h = Th
        if self.top is None:
            hx = part.wx0 * self.boxes[0, 2]
            hy = part.wy0 * self.boxes[0, 3]
            geo = np.array([[b // part.by * hx, b % part.by * hy, hx, hy] for b in range(part.world)])
            self.top = self.hps.Plan(np.full(part.world, self.p, dtype=np.int32), geo, self.kappa)
        self.Tb = torch.stack([t.contiguous() for t in T]).contiguous().view(-1)
        self.hb = torch.stack([x.contiguous() for x in h]).contiguous().view(-1)
        self.top.merge_boxes(part.bx, part.by, part.wx0, part.wy0, self.Tb, self.hb, m)

    def top_solve(self, g, part, m):
        import torch
        g = g if isinstance(g, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(g)).cuda()
        ub = self.top.solve_boxes(g.contiguous().view(-1), m)
        nb = part.box_nodes(self.p - 2)
        return list(ub.view(part.world, nb, m))

    def local_solve(self, ub, m):
        return self.plan.solve(ub.contiguous().view(-1), self.out["S"], self.out.get("W"), m)

    def close(self):
        if self.own:
            self.plan.close()
        if self.top is not None:
            self.top.close()


def run_in_process(backends, part, q, g, m):
    """The split with every rank in this process (one GPU, or none): the
    same steps in the same order as split_merge / split_solve, the exchange
    replaced by passing the arrays; returns each rank's local_solve result.
    (Ranks whose kernels wait on each other never share a GPU: there are no
    such waits here, every step completes before the next starts.)"""
    ths = [b.local_merge(m) for b in backends]
    backends[0].top_merge(unpack_roots(ths, part.box_nodes(q), m), part, m)
    parts = backends[0].top_solve(g, part, m)
    return [b.local_solve(parts[r], m) for r, b in enumerate(backends)]
