"""2D-partitioned BFS over several GPUs: the vertex and edge partition and the
per-level frontier exchange (after Buluc and Madduri, SC 2011).

Not measured on hardware: every run of this project has one GPU, so the
multi-GPU search is a design whose partition and exchange schedule are tested
with CPU processes (gloo) in tests/test_bfs2d.py.  Nothing here computes a
search step: the local expansion of a rank's block is passed in (on GPUs it
would be the library's top-down step over the rank's CSR block; the test
passes a plain one), and this module only decides who holds what and what
moves between ranks at each level.

Layout, on an R x C grid of ranks (rank r = i * C + j for grid row i, column j):

* the n vertices are cut into P = R * C equal pieces; rank (i, j) owns piece
  q = i * C + j: its level and parent entries and its part of every frontier;
* grid row i covers the C pieces i * C .. i * C + C - 1 (the row block),
  grid column j the R pieces k * C + j, k = 0 .. R - 1 (the column block);
* rank (i, j) holds the directed edges u -> v (both directions of every
  undirected edge) with u in column block j and v in row block i, as a CSR
  over the column block's vertices.

One level (top-down; Sec. 2.3.2's level-synchronous step):

1. expand: the frontier bitmaps of the pieces of column block j are gathered
   within grid column j (an all-gather of n / P bits per rank);
2. local step: from those frontier vertices through the rank's edges, the
   smallest-id frontier neighbour of every vertex of row block i (or n if
   none): an int32 array over the row block;
3. fold: within grid row i the arrays are combined by minimum and each rank
   keeps its own piece (a reduce-scatter; gloo has none, so the test's
   exchange is an all-reduce followed by taking the piece -- the same
   result);
4. the owner marks its unvisited vertices with a parent below n: level l + 1,
   that parent, and the next frontier; an all-reduce of the counts ends the
   search when no rank found a vertex.

The minimum in the fold makes every parent the smallest-id neighbour one
level up, the canonical tree of the oracle.  Per level and rank the exchange
moves n / P bits per rank of its grid column (expand) and 4 n / R bytes
(fold); the bitmaps are frontier-sized and never pass through TMA multicast.
"""
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Grid:
    R: int
    C: int
    n: int

    @property
    def P(self):
        return self.R * self.C

    def coords(self, rank):
        return divmod(rank, self.C)

    def piece_range(self, q):
        """Vertices [lo, hi) of piece q."""
        return q * self.n // self.P, (q + 1) * self.n // self.P

    def piece_of(self, v):
        """Piece of each vertex id (array)."""
        v = np.asarray(v, dtype=np.int64)
        # the largest q with lo(q) <= v
        q = (v * self.P) // self.n
        lo = q * self.n // self.P
        q = np.where(lo > v, q - 1, q)
        hi = (q + 1) * self.n // self.P
        return np.where(v >= hi, q + 1, q)

    def row_pieces(self, i):
        return [i * self.C + k for k in range(self.C)]

    def col_pieces(self, j):
        return [k * self.C + j for k in range(self.R)]

    def block_vertices(self, pieces):
        """The vertices of a list of pieces, in piece order."""
        return np.concatenate([np.arange(*self.piece_range(q), dtype=np.int64) for q in pieces])


@dataclass
class LocalBlock:
    """Rank (i, j)'s edges u -> v, u in column block j, v in row block i: a CSR
    over the column block's vertices (local ids) whose entries are local ids
    of the row block."""
    col_vertices: np.ndarray   # global ids of the column block, local id = position
    row_vertices: np.ndarray   # global ids of the row block
    off: np.ndarray            # int64 [len(col_vertices) + 1]
    dst: np.ndarray            # int32 local row-block ids


def partition(edges, grid, rank):
    """The block of `rank` from the undirected tuples edges [2, m] (self-loops
    and duplicates dropped, both directions kept)."""
    i, j = grid.coords(rank)
    cols = grid.block_vertices(grid.col_pieces(j))
    rows = grid.block_vertices(grid.row_pieces(i))
    u = np.concatenate([edges[0], edges[1]]).astype(np.int64)
    v = np.concatenate([edges[1], edges[0]]).astype(np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    col_of = np.full(grid.n, -1, dtype=np.int64)
    col_of[cols] = np.arange(cols.size)
    row_of = np.full(grid.n, -1, dtype=np.int64)
    row_of[rows] = np.arange(rows.size)
    sel = (col_of[u] >= 0) & (row_of[v] >= 0)
    lu, lv = col_of[u[sel]], row_of[v[sel]]
    key = np.unique(lu * max(rows.size, 1) + lv)
    lu, lv = key // max(rows.size, 1), key % max(rows.size, 1)
    off = np.zeros(cols.size + 1, dtype=np.int64)
    np.add.at(off, lu + 1, 1)
    return LocalBlock(cols, rows, np.cumsum(off), lv.astype(np.int32))


class Exchange:
    """The collectives of one rank: its grid-column and grid-row groups."""

    def __init__(self, dist, grid, rank):
        self.dist, self.grid, self.rank = dist, grid, rank
        i, j = grid.coords(rank)
        self.i, self.j = i, j
        self.col_groups = [dist.new_group([k * grid.C + jj for k in range(grid.R)]) for jj in range(grid.C)]
        self.row_groups = [dist.new_group([ii * grid.C + k for k in range(grid.C)]) for ii in range(grid.R)]
        self.col_group = self.col_groups[j]
        self.row_group = self.row_groups[i]

    def expand(self, frontier_piece):
        """All-gather of the frontier bits of the column block's pieces."""
        import torch
        parts = [torch.zeros_like(frontier_piece) for _ in range(self.grid.R)]
        self.dist.all_gather(parts, frontier_piece, group=self.col_group)
        return torch.cat(parts)

    def fold(self, cand_row_block, piece_sizes):
        """Min over the grid row, each rank keeping its own piece."""
        import torch
        t = cand_row_block.clone()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.row_group)
        start = sum(piece_sizes[:self.j])
        return t[start:start + piece_sizes[self.j]]

    def total(self, x):
        import torch
        t = torch.tensor([int(x)], dtype=torch.int64)
        self.dist.all_reduce(t)
        return int(t.item())


def bfs_2d(block, grid, rank, root, ex, local_step):
    """Levels and parents of this rank's piece from `root`.

    local_step(block, frontier_cols) -> int32 array over the row block: for
    each of its vertices the smallest global id of a frontier neighbour
    through this block's edges, or grid.n.  frontier_cols is a bool array
    over the column block."""
    import torch
    q = rank
    lo, hi = grid.piece_range(q)
    size = hi - lo
    level = np.full(size, -1, dtype=np.int32)
    parent = np.full(size, -1, dtype=np.int32)
    frontier = np.zeros(size, dtype=bool)
    if lo <= root < hi:
        level[root - lo] = 0
        parent[root - lo] = root
        frontier[root - lo] = True
    row_sizes = [grid.piece_range(p)[1] - grid.piece_range(p)[0] for p in grid.row_pieces(ex.i)]
    col_sizes = [grid.piece_range(p)[1] - grid.piece_range(p)[0] for p in grid.col_pieces(ex.j)]
    l = 0
    while True:
        fr = torch.from_numpy(frontier.astype(np.uint8))
        # pieces of a grid column may differ by one vertex: gather padded parts
        pad = max(col_sizes)
        fr = torch.nn.functional.pad(fr, (0, pad - fr.numel()))
        parts = ex.expand(fr).numpy().reshape(grid.R, pad)
        fcols = np.concatenate([parts[k, :col_sizes[k]] for k in range(grid.R)]).astype(bool)
        cand = local_step(block, fcols)
        mine = ex.fold(torch.from_numpy(np.ascontiguousarray(cand, dtype=np.int32)), row_sizes).numpy()
        new = (mine < grid.n) & (level < 0)
        level[new] = l + 1
        parent[new] = mine[new]
        frontier = new
        if ex.total(new.sum()) == 0:
            return level, parent
        l += 1
