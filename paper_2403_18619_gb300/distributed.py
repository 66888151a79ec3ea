"""One graph solved on several GPUs: blocked FW over 2-D block-cyclic tiles.

For a matrix larger than one GPU's memory (int32 dist + pred: n beyond about
150 000 on a GB300), the R x R tiles of the blocked algorithm (Sec. 2.3,
Fig. 2) are spread over a pr x pc grid of ranks: tile (I, J) lives on rank
(I mod pr) * pc + (J mod pc).  Round r then runs, with one exchange:

  1. the owner of tile (r, r) closes it (phase 1, fw_tile_closure) and
     broadcasts it;
  2. the ranks of process row r mod pr update their tiles of tile row r (row
     panel: B = the tile itself, predecessors from its own rows) and the ranks
     of process column r mod pc their tiles of tile column r (column panel: A
     = the tile itself, predecessors from the pivot's rows) -- phases 2 and 3,
     fw_tile_minplus;
  3. every process column receives the row panel of its tile columns from its
     rank in process row r mod pr, every process row the column panel of its
     tile rows from its rank in process column r mod pc (broadcasts on the
     row / column sub-groups);
  4. every rank updates its other tiles: C = min(C, column panel (x) row panel)
     (phase 4, fw_tile_minplus over its whole local block, skipping the panel
     tiles).

The paper runs the blocked algorithm on one shared-memory node and names a
library form as future work (Sec. 5); this is the same schedule with the
tiles of a round spread over GPUs, each exchange a broadcast of one pivot
tile and of bs x (n / pc) and (n / pr) x bs panel strips.

Local blocks are tile-padded: a rank holds its tile rows and tile columns as
one (rows x bs) x (cols x bs) matrix, padding vertices isolated (INF off the
diagonal, 0 on it).  Predecessors are last hops in global vertex ids.

The schedule runs over a list of rank states and a communicator: with
TorchComm (one state, torch.distributed: NCCL on GPUs, gloo on CPU tensors)
each process is one rank; with LocalComm several ranks run in one process, in
lockstep, and a broadcast is a copy -- no kernel ever waits for another
rank's.  Tile operations come from an ops object; CudaTileOps calls the CUDA
library (the only implementation in this package).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fw_block_init_pred, fw_tile_closure, fw_tile_minplus


@dataclass(frozen=True)
class Grid:
    """A pr x pc process grid over the R x R tiles of an n-vertex graph."""
    n: int
    bs: int
    pr: int
    pc: int

    @property
    def R(self) -> int:
        return (self.n + self.bs - 1) // self.bs

    @property
    def world(self) -> int:
        return self.pr * self.pc

    def coords(self, rank: int):
        return rank // self.pc, rank % self.pc

    def owner(self, I: int, J: int) -> int:
        return (I % self.pr) * self.pc + (J % self.pc)

    def tile_rows(self, prow: int):
        return list(range(prow, self.R, self.pr))

    def tile_cols(self, pcol: int):
        return list(range(pcol, self.R, self.pc))

    def local_shape(self, rank: int):
        prow, pcol = self.coords(rank)
        return len(self.tile_rows(prow)) * self.bs, len(self.tile_cols(pcol)) * self.bs

    def global_ids(self, tiles):
        """Global vertex ids of the local rows (or columns) of these tiles."""
        return (np.asarray(tiles, np.int64)[:, None] * self.bs +
                np.arange(self.bs, dtype=np.int64)[None, :]).reshape(-1)


def _inf_of(dtype):
    dtype = np.dtype(dtype)
    if dtype == np.int32:
        return 1 << 29
    if dtype == np.int64:
        return 1 << 61
    return np.inf


def scatter_block(W: np.ndarray, grid: Grid, rank: int) -> np.ndarray:
    """The tile-padded local block of rank `rank` from a host matrix W."""
    prow, pcol = grid.coords(rank)
    ri = grid.global_ids(grid.tile_rows(prow))
    ci = grid.global_ids(grid.tile_cols(pcol))
    out = np.full((len(ri), len(ci)), _inf_of(W.dtype), dtype=W.dtype)
    rin, cin = ri < grid.n, ci < grid.n
    out[np.ix_(rin, cin)] = W[np.ix_(ri[rin], ci[cin])]
    pad = ri[:, None] == ci[None, :]
    out[pad & ~(rin[:, None] & cin[None, :])] = 0
    return out


def gather_blocks(blocks, grid: Grid, fill=-1) -> np.ndarray:
    """The n x n matrix from every rank's local block (host arrays, rank order)."""
    out = np.full((grid.n, grid.n), fill, dtype=np.asarray(blocks[0]).dtype)
    for rank, blk in enumerate(blocks):
        prow, pcol = grid.coords(rank)
        ri = grid.global_ids(grid.tile_rows(prow))
        ci = grid.global_ids(grid.tile_cols(pcol))
        rin, cin = ri < grid.n, ci < grid.n
        out[np.ix_(ri[rin], ci[cin])] = np.asarray(blk)[np.ix_(rin, cin)]
    return out


@dataclass
class RankState:
    """One rank's local block, its predecessors (None: distances only) and the
    exchange buffers of a round (torch tensors on the rank's device)."""
    rank: int
    D: object
    P: object = None
    piv: object = None
    pivP: object = None
    rowbuf: object = None
    rowbufP: object = None
    colbuf: object = None

    @classmethod
    def create(cls, rank: int, grid: Grid, D, P=None) -> "RankState":
        import torch
        bs = grid.bs
        rows, cols = grid.local_shape(rank)
        if tuple(D.shape) != (rows, cols):
            raise ValueError("rank %d needs a %d x %d local block" % (rank, rows, cols))
        kw = dict(dtype=D.dtype, device=D.device)
        pk = dict(dtype=torch.int32, device=D.device)
        st = cls(rank=rank, D=D, P=P)
        st.piv = torch.empty((bs, bs), **kw)
        st.rowbuf = torch.empty((bs, cols), **kw)
        st.colbuf = torch.empty((rows, bs), **kw)
        if P is not None:
            st.pivP = torch.empty((bs, bs), **pk)
            st.rowbufP = torch.empty((bs, cols), **pk)
        return st


class TorchComm:
    """Broadcasts over torch.distributed (this process holds one rank).  The
    row and column sub-groups are created here, by every rank in the same
    order, as torch.distributed requires."""

    def __init__(self, grid: Grid):
        import torch.distributed as dist
        self.dist = dist
        self.grid = grid
        self.row_groups = [dist.new_group([a * grid.pc + c for c in range(grid.pc)])
                           for a in range(grid.pr)]
        self.col_groups = [dist.new_group([a * grid.pc + c for a in range(grid.pr)])
                           for c in range(grid.pc)]

    def bcast_all(self, states, name: str, root: int):
        for st in states:
            t = getattr(st, name)
            if t is not None:
                self.dist.broadcast(t, src=root)

    def bcast_in_cols(self, states, name: str, root_prow: int):
        for st in states:
            t = getattr(st, name)
            if t is None:
                continue
            prow, pcol = self.grid.coords(st.rank)
            self.dist.broadcast(t, src=root_prow * self.grid.pc + pcol,
                                group=self.col_groups[pcol])

    def bcast_in_rows(self, states, name: str, root_pcol: int):
        for st in states:
            t = getattr(st, name)
            if t is None:
                continue
            prow, pcol = self.grid.coords(st.rank)
            self.dist.broadcast(t, src=prow * self.grid.pc + root_pcol,
                                group=self.row_groups[prow])


class LocalComm:
    """Every rank of the grid in this process, run in lockstep: a broadcast
    copies the root's buffer into the other ranks' of the group."""

    def __init__(self, grid: Grid):
        self.grid = grid

    @staticmethod
    def _copy(states, name, root, members):
        src = getattr(states[root], name)
        if src is None:
            return
        for r in members:
            if r != root:
                getattr(states[r], name).copy_(src)

    def bcast_all(self, states, name, root):
        self._copy(states, name, root, range(len(states)))

    def bcast_in_cols(self, states, name, root_prow):
        g = self.grid
        for pcol in range(g.pc):
            self._copy(states, name, root_prow * g.pc + pcol,
                       [a * g.pc + pcol for a in range(g.pr)])

    def bcast_in_rows(self, states, name, root_pcol):
        g = self.grid
        for prow in range(g.pr):
            self._copy(states, name, prow * g.pc + root_pcol,
                       [prow * g.pc + c for c in range(g.pc)])


class CudaTileOps:
    """The tile operations of the schedule, by the CUDA library (a rank with
    no tile rows or columns has empty blocks and nothing to do)."""

    @staticmethod
    def init_pred(D, P, bs, n, rt0, rts, ct0, cts):
        if D.numel():
            fw_block_init_pred(D, P, bs, n, rt0, rts, ct0, cts)

    @staticmethod
    def closure(tile, ptile, bs):
        fw_tile_closure(tile, ptile, bs)

    @staticmethod
    def minplus(C, Pc, A, B, Pb, bs, skip_row=-1, skip_col=-1):
        if C.numel():
            fw_tile_minplus(C, Pc, A, B, Pb, bs, skip_row, skip_col)


def solve_block_cyclic(states, grid: Grid, comm, ops=CudaTileOps) -> None:
    """Blocked FW over the grid: `states` are the RankStates this process
    holds (one under TorchComm, every rank under LocalComm), their D holding
    the weights on entry and the distances on exit, P (if given) receiving
    the last hops."""
    bs, pr, pc = grid.bs, grid.pr, grid.pc
    preds = states[0].P is not None
    if preds:
        for st in states:
            prow, pcol = grid.coords(st.rank)
            ops.init_pred(st.D, st.P, bs, grid.n, prow, pr, pcol, pc)
    for r in range(grid.R):
        rp, rc = r % pr, r % pc
        lr, lc = r // pr, r // pc  # local tile indices of tile row / column r where owned
        owner = grid.owner(r, r)
        # 1. phase 1 on the owner, then the pivot to every rank
        for st in states:
            if st.rank == owner:
                tile = st.D[lr * bs:(lr + 1) * bs, lc * bs:(lc + 1) * bs]
                ptile = st.P[lr * bs:(lr + 1) * bs, lc * bs:(lc + 1) * bs] if preds else None
                ops.closure(tile, ptile, bs)
                st.piv.copy_(tile)
                if preds:
                    st.pivP.copy_(ptile)
        comm.bcast_all(states, "piv", owner)
        comm.bcast_all(states, "pivP", owner)
        # 2. phases 2 and 3 on the panel owners (the pivot tile itself is closed)
        for st in states:
            prow, pcol = grid.coords(st.rank)
            if prow == rp:
                strip = st.D[lr * bs:(lr + 1) * bs, :]
                pstrip = st.P[lr * bs:(lr + 1) * bs, :] if preds else None
                ops.minplus(strip, pstrip, st.piv, strip, pstrip, bs, -1, lc if pcol == rc else -1)
                st.rowbuf.copy_(strip)
                if preds:
                    st.rowbufP.copy_(pstrip)
            if pcol == rc:
                strip = st.D[:, lc * bs:(lc + 1) * bs]
                pstrip = st.P[:, lc * bs:(lc + 1) * bs] if preds else None
                ops.minplus(strip, pstrip, strip, st.piv, st.pivP if preds else None, bs,
                            lr if prow == rp else -1, -1)
                st.colbuf.copy_(strip)
        # 3. the exchange: row panels down the process columns, column panels
        #    across the process rows
        comm.bcast_in_cols(states, "rowbuf", rp)
        comm.bcast_in_cols(states, "rowbufP", rp)
        comm.bcast_in_rows(states, "colbuf", rc)
        # 4. phase 4 on every rank's other tiles
        for st in states:
            prow, pcol = grid.coords(st.rank)
            ops.minplus(st.D, st.P, st.colbuf, st.rowbuf, st.rowbufP if preds else None, bs,
                        lr if prow == rp else -1, lc if pcol == rc else -1)
