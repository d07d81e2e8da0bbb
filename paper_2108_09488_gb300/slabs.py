"""Slab decomposition of one plume over ranks (one process per GPU): the exchange steps of a
multi-GPU predictor-corrector step (Eq. 8-9), as host logic over ``torch.distributed``.

Rank r owns the particles whose x coordinate lies in [r L/W, (r + 1) L/W) of the periodic box
(ownership is fixed at the start of a step).  Eq. 4 at an owned particle needs its neighbours
within H, so before each of the step's two evaluations every rank sends its two neighbours the
owned particles within ``reach`` of their common face (positions and the concentrations of that
evaluation) and evaluates the rate on owned + received particles.  After the corrector, particles
that drifted into another slab move to their new owner.  Global diagnostics (sum m C, min, max)
are FP64 all-reduces.  No other exchange is needed: each particle's update uses only its own rate.

The rate itself is a callable ``rate_fn(x, C, n_own) -> dC/dt of the first n_own particles`` over
the local set (owned first, then received), so the same logic drives the FP64 oracle on CPU ranks
(the tests) or the GPU library on one GPU per rank (``ade_dispersion_rate`` on the local set).
Messages are variable-length: a count, then the payload, tagged per direction so that a world of
two (both neighbours the same rank) stays unambiguous.
"""
from __future__ import annotations

import numpy as np


class SlabDecomposition:
    """Ownership and exchanges of x-slabs of width L/W; ``reach`` = H plus any drift between the
    ownership test and an evaluation (here: half a step of the fastest particle)."""

    TAG_LEFT, TAG_RIGHT, TAG_MIGRATE_LEFT, TAG_MIGRATE_RIGHT = 11, 12, 13, 14

    def __init__(self, box, reach, world, rank):
        self.box = np.asarray(box, dtype=np.float64)
        self.L = float(self.box[0])
        self.world, self.rank = int(world), int(rank)
        self.width = self.L / self.world
        self.reach = float(reach)
        if self.world > 1 and not self.reach < self.width:
            raise ValueError("slabs must be wider than the exchange reach")
        if self.world == 2 and not 2.0 * self.reach < self.width:
            # both faces border the same rank: a particle within reach of both would arrive twice
            raise ValueError("with two ranks the slabs must be wider than twice the exchange reach")
        self.lo = self.rank * self.width
        self.left = (self.rank - 1) % self.world
        self.right = (self.rank + 1) % self.world

    # ---- ownership ---------------------------------------------------------------------------
    def owner(self, x):
        """Owning rank of positions x [n][dim] (x wrapped into [0, L))."""
        u = np.mod(np.asarray(x, dtype=np.float64)[:, 0], self.L)
        return np.minimum((u / self.width).astype(np.int64), self.world - 1)

    def _face_distances(self, x):
        """Signed distances of x to this slab's left and right faces (positive inside), from the
        minimum-image offset to the slab's centre (unambiguous while particles stay within half a
        box of it, which the one-slab drift limit guarantees)."""
        u = np.asarray(x, dtype=np.float64)[:, 0]
        d = np.mod(u - (self.lo + 0.5 * self.width) + 0.5 * self.L, self.L) - 0.5 * self.L
        return d + 0.5 * self.width, 0.5 * self.width - d

    # ---- messages ----------------------------------------------------------------------------
    def _exchange(self, send_left, send_right, tag_l, tag_r):
        """Send float64 blocks [k][m] to the left and right neighbours and receive theirs; returns
        (from_left, from_right)."""
        import torch
        import torch.distributed as dist

        def t(a):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))

        m = send_left.shape[1]
        nl = torch.tensor([send_left.shape[0]], dtype=torch.int64)
        nr = torch.tensor([send_right.shape[0]], dtype=torch.int64)
        cl = torch.zeros(1, dtype=torch.int64)
        cr = torch.zeros(1, dtype=torch.int64)
        # counts: what goes left arrives at the left neighbour as "from its right" (tag_r there)
        reqs = [dist.irecv(cl, self.left, tag=tag_r), dist.irecv(cr, self.right, tag=tag_l),
                dist.isend(nl, self.left, tag=tag_l), dist.isend(nr, self.right, tag=tag_r)]
        for q in reqs:
            q.wait()
        bl = torch.empty((int(cl.item()), m), dtype=torch.float64)
        br = torch.empty((int(cr.item()), m), dtype=torch.float64)
        reqs = []
        if bl.shape[0]:
            reqs.append(dist.irecv(bl, self.left, tag=tag_r + 100))
        if br.shape[0]:
            reqs.append(dist.irecv(br, self.right, tag=tag_l + 100))
        if send_left.shape[0]:
            reqs.append(dist.isend(t(send_left), self.left, tag=tag_l + 100))
        if send_right.shape[0]:
            reqs.append(dist.isend(t(send_right), self.right, tag=tag_r + 100))
        for q in reqs:
            q.wait()
        return bl.numpy(), br.numpy()

    def halo(self, x, C):
        """Positions and concentrations of the neighbours' particles within reach of this slab
        (received), for one evaluation."""
        if self.world == 1:
            return np.zeros((0, x.shape[1])), np.zeros(0)
        dl, dr = self._face_distances(x)
        rec = np.concatenate([x, C[:, None]], axis=1)
        fl, fr = self._exchange(rec[dl < self.reach], rec[dr < self.reach], self.TAG_LEFT, self.TAG_RIGHT)
        got = np.concatenate([fl, fr], axis=0)
        return got[:, :-1], got[:, -1]

    def migrate(self, ids, x, C):
        """Hand particles that left the slab to their new owners (neighbours: the drift per step is
        below the slab width); returns the rank's particles (ids, x, C) sorted by id."""
        if self.world == 1:
            return ids, x, C
        own = self.owner(x)
        keep = own == self.rank
        rec = np.concatenate([ids[:, None].astype(np.float64), x, C[:, None]], axis=1)
        to_left = rec[(~keep) & (own == self.left)]
        to_right = rec[(~keep) & (own == self.right) & (own != self.left)]
        if np.any((~keep) & (own != self.left) & (own != self.right)):
            raise RuntimeError("a particle moved farther than one slab in one step")
        fl, fr = self._exchange(to_left, to_right, self.TAG_MIGRATE_LEFT, self.TAG_MIGRATE_RIGHT)
        allr = np.concatenate([rec[keep], fl, fr], axis=0)
        order = np.argsort(allr[:, 0], kind="stable")
        allr = allr[order]
        return allr[:, 0].astype(np.int64), allr[:, 1:-1], allr[:, -1]


def distributed_step(dec, rate_fn, ids, x, v, C, dt):
    """One predictor-corrector step (Eq. 8-9) of the rank's particles: halo exchange + rate,
    predictor, halo exchange at the half step + rate, corrector, migration.  v: uniform velocity
    [dim].  Returns the rank's new (ids, x, C)."""
    n = x.shape[0]
    hx, hC = dec.halo(x, C)
    r0 = rate_fn(np.concatenate([x, hx]), np.concatenate([C, hC]), n)
    Ch = C + 0.5 * dt * r0
    xh = np.mod(x + 0.5 * dt * v[None, :], dec.box[None, : x.shape[1]])
    hx, hC = dec.halo(xh, Ch)
    r1 = rate_fn(np.concatenate([xh, hx]), np.concatenate([Ch, hC]), n)
    C1 = C + dt * r1
    x1 = np.mod(x + dt * v[None, :], dec.box[None, : x.shape[1]])
    return dec.migrate(ids, x1, C1)


def global_stats(C, mass):
    """FP64 sum m C, min C, max C over all ranks."""
    import torch
    import torch.distributed as dist
    s = torch.tensor([float(np.sum(C) * mass)], dtype=torch.float64)
    lo = torch.tensor([float(np.min(C)) if C.size else np.inf], dtype=torch.float64)
    hi = torch.tensor([float(np.max(C)) if C.size else -np.inf], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(lo, op=dist.ReduceOp.MIN)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX)
    return float(s.item()), float(lo.item()), float(hi.item())
