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
the local set (owned first, then received).  ``SlabDecomposition`` works on FP64 positions (numpy,
host messages); ``FixedSlabs`` / ``fixed_step`` work on the library's own state -- uint32
fixed-point position words and float32 C as torch tensors on the rank's device, exchanged as int32
records with point-to-point sends (NCCL between GPUs, gloo between CPU ranks) -- and
``LibraryRate`` evaluates a rank's owned + received set with ``ade_dispersion_rate``.
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


# ---- the library's fixed-point state: device buffers, point-to-point exchange ---------------------
# The same decomposition over the state the library keeps on the GPU: positions as uint32
# fixed-point words (int32 tensors [dim][n], x = word * L / 2^32) and C as float32.  A halo or
# migration record is one int32 row: (for migration the particle id,) the dim position words and
# the bits of C -- the library's own format, so a rank's owned + received set goes to
# ``ade_dispersion_rate`` without conversion.  Records travel as tensors on the rank's device with
# torch.distributed point-to-point (NCCL between GPUs; gloo between CPU ranks, where the tests run);
# no collective is used on the data path.

_TWO32 = 1 << 32
_MASK32 = _TWO32 - 1


def fixed_increment(v, dt, L):
    """Fixed-point drift of one axis over dt: v dt / L * 2^32 rounded to nearest (ties to even),
    modulo 2^32 (the library's rounding of its drift words)."""
    return int(round(v * dt / L * float(_TWO32))) % _TWO32


def drift(xq, inc):
    """xq + inc per axis, modulo 2^32 (int32 tensor [dim][n]; inc: one word per axis)."""
    import torch
    w = (xq.to(torch.int64) & _MASK32) + torch.tensor(list(inc), dtype=torch.int64, device=xq.device)[:, None]
    w = w & _MASK32
    return torch.where(w >= (1 << 31), w - _TWO32, w).to(torch.int32)


class FixedSlabs:
    """x-slabs of the library's fixed-point box: rank r owns the words u of axis x with
    floor(u W / 2^32) = r.  ``reach`` (a length) = H plus the drift between the ownership test and
    an evaluation; it is rounded up to words with a two-word margin, so the selection is exact
    integer arithmetic."""

    TAG_LEFT, TAG_RIGHT, TAG_MIGRATE_LEFT, TAG_MIGRATE_RIGHT = 21, 22, 23, 24

    def __init__(self, reach, box_x, world, rank, device="cpu"):
        import math
        self.world, self.rank, self.device = int(world), int(rank), device
        self.reach_u = int(math.ceil(reach / float(box_x) * float(_TWO32))) + 2
        width_u = _TWO32 // self.world
        if self.world > 1 and not self.reach_u < width_u:
            raise ValueError("slabs must be wider than the exchange reach")
        if self.world == 2 and not 2 * self.reach_u < width_u:
            raise ValueError("with two ranks the slabs must be wider than twice the exchange reach")
        self.centre = ((2 * self.rank + 1) << 32) // (2 * self.world)
        self.half = _TWO32 // (2 * self.world)
        self.left = (self.rank - 1) % self.world
        self.right = (self.rank + 1) % self.world

    def owner(self, xq):
        """Owning rank of fixed-point positions xq [dim][n]."""
        import torch
        u = xq[0].to(torch.int64) & _MASK32
        return (u * self.world) >> 32

    def _faces(self, xq):
        """Distances in words to this slab's left and right faces (positive inside; within one
        word of the exact faces), from the minimum-image offset to the slab's centre."""
        import torch
        u = xq[0].to(torch.int64) & _MASK32
        d = ((u - self.centre + (1 << 31)) & _MASK32) - (1 << 31)
        return d + self.half, self.half - d

    @staticmethod
    def records(xq, C):
        """int32 records [n][dim + 1]: the position words and the bits of C."""
        import torch
        return torch.cat([xq.t(), C.contiguous().view(torch.int32)[:, None]], dim=1).contiguous()

    def outgoing(self, xq, C):
        """Records of the owned particles within reach of the left and of the right face."""
        dl, dr = self._faces(xq)
        rec = self.records(xq, C)
        return rec[dl < self.reach_u], rec[dr < self.reach_u]

    def exchange(self, send_left, send_right, tag_l, tag_r):
        """Send int32 records to the left and right neighbours and receive theirs (counts first,
        then payloads; tags per direction, so a world of two stays unambiguous)."""
        import torch
        import torch.distributed as dist
        dev = send_left.device
        m = send_left.shape[1]
        nl = torch.tensor([send_left.shape[0]], dtype=torch.int64, device=dev)
        nr = torch.tensor([send_right.shape[0]], dtype=torch.int64, device=dev)
        cl = torch.zeros(1, dtype=torch.int64, device=dev)
        cr = torch.zeros(1, dtype=torch.int64, device=dev)
        reqs = [dist.irecv(cl, self.left, tag=tag_r), dist.irecv(cr, self.right, tag=tag_l),
                dist.isend(nl, self.left, tag=tag_l), dist.isend(nr, self.right, tag=tag_r)]
        for q in reqs:
            q.wait()
        bl = torch.empty((int(cl.item()), m), dtype=torch.int32, device=dev)
        br = torch.empty((int(cr.item()), m), dtype=torch.int32, device=dev)
        reqs = []
        if bl.shape[0]:
            reqs.append(dist.irecv(bl, self.left, tag=tag_r + 100))
        if br.shape[0]:
            reqs.append(dist.irecv(br, self.right, tag=tag_l + 100))
        if send_left.shape[0]:
            reqs.append(dist.isend(send_left, self.left, tag=tag_l + 100))
        if send_right.shape[0]:
            reqs.append(dist.isend(send_right, self.right, tag=tag_r + 100))
        for q in reqs:
            q.wait()
        return bl, br

    @staticmethod
    def unpack(rec):
        """(xq [dim][k], C [k]) of int32 records [k][dim + 1]."""
        import torch
        return rec[:, :-1].t().contiguous(), rec[:, -1].contiguous().view(torch.float32)

    def halo(self, xq, C):
        """The neighbours' particles within reach of this slab (received), for one evaluation."""
        import torch
        if self.world == 1:
            return (torch.zeros((xq.shape[0], 0), dtype=torch.int32, device=xq.device),
                    torch.zeros(0, dtype=torch.float32, device=xq.device))
        fl, fr = self.exchange(*self.outgoing(xq, C), self.TAG_LEFT, self.TAG_RIGHT)
        return self.unpack(torch.cat([fl, fr], dim=0))

    def migrate(self, ids, xq, C):
        """Hand particles that left the slab to their new owners; returns (ids, xq, C) sorted by
        id (ids int32, below 2^31)."""
        import torch
        if self.world == 1:
            return ids, xq, C
        own = self.owner(xq)
        keep = own == self.rank
        rec = torch.cat([ids[:, None].to(torch.int32), self.records(xq, C)], dim=1)
        to_left = rec[(~keep) & (own == self.left)]
        to_right = rec[(~keep) & (own == self.right) & (own != self.left)]
        if bool(((~keep) & (own != self.left) & (own != self.right)).any()):
            raise RuntimeError("a particle moved farther than one slab in one step")
        fl, fr = self.exchange(to_left, to_right, self.TAG_MIGRATE_LEFT, self.TAG_MIGRATE_RIGHT)
        allr = torch.cat([rec[keep], fl, fr], dim=0)
        allr = allr[torch.argsort(allr[:, 0], stable=True)]
        xq1, C1 = self.unpack(allr[:, 1:])
        return allr[:, 0].contiguous(), xq1, C1


def fixed_step(dec, rate_fn, ids, xq, C, inc_half, inc_full, dt):
    """One predictor-corrector step (Eq. 8-9) of the rank's particles in the library's format:
    halo exchange + rate, C^{l+1/2} = C^l + dt/2 r^l and x^{l+1/2} = x^l + the half-step drift,
    halo exchange + rate at the half step, C^{l+1} = C^l + dt r^{l+1/2} and x^{l+1} = x^l + the
    full-step drift, migration.  ``rate_fn(xq, C, n_own)`` returns the float32 rates of the first
    n_own particles of the local set (owned first, then received)."""
    import torch
    n = C.shape[0]
    hx, hC = dec.halo(xq, C)
    r0 = rate_fn(torch.cat([xq, hx], dim=1), torch.cat([C, hC]), n)
    Ch = C + (0.5 * dt) * r0
    xh = drift(xq, inc_half)
    hx, hC = dec.halo(xh, Ch)
    r1 = rate_fn(torch.cat([xh, hx], dim=1), torch.cat([Ch, hC]), n)
    C1 = C + dt * r1
    x1 = drift(xq, inc_full)
    return dec.migrate(ids, x1, C1)


class LibraryRate:
    """``rate_fn`` over the GPU library: Eq. 4 at the local set (owned + received particles, int32
    position words [dim][m] and float32 C on this rank's GPU) by ``ade_dispersion_rate`` with the
    plume's parameters; returns the owned particles' rates on the device.  The local set is a
    subset of the periodic box, so every owned particle meets all its neighbours (the received
    ones cover H across the faces) and the received particles' own rates are discarded."""

    def __init__(self, params):
        self.p = params

    def __call__(self, xq, C, n_own):
        import ctypes
        import torch
        from . import ade
        xq = xq.contiguous()
        C = C.contiguous()
        m = int(C.shape[0])
        nbytes = ade.workspace_bytes(self.p, m)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=C.device)
        ptr = (ws.data_ptr() + 255) // 256 * 256
        out = torch.empty(max(m, 1), dtype=torch.float32, device=C.device)
        stream = ctypes.c_void_p(torch.cuda.current_stream(C.device).cuda_stream)
        ctx = ade.init_particles(self.p, m, xq.data_ptr(), C.data_ptr(), ptr, nbytes)
        try:
            ade.dispersion_rate(ctx, out.data_ptr(), stream)
            torch.cuda.current_stream(C.device).synchronize()
        finally:
            ade.destroy(ctx)
        return out[:n_own]
