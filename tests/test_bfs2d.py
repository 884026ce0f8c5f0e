"""The 2D-partitioned BFS design (paper_2012_13548_gb300/bfs2d.py) on CPU
processes: its partition and per-level exchange, with gloo ranks.

Each rank builds its block of a Kronecker graph, runs the level loop with a
plain local step (this test's, not the library's: the multi-GPU search is a
design, unmeasured on hardware), and the pieces gathered from all ranks must
equal the oracle's levels and canonical parents (Sec. 2.3.1): the
minimum in the fold picks the smallest-id parent.  Grids 1 x 2, 2 x 1 and 2 x 2.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def local_step(block, frontier_cols):
    """Smallest global id of a frontier neighbour of every row-block vertex
    through this block's edges (n if none)."""
    n_rows = block.row_vertices.size
    best = np.full(n_rows, np.iinfo(np.int32).max, dtype=np.int64)
    deg = np.diff(block.off)
    src = np.repeat(np.arange(block.col_vertices.size), deg)
    on = frontier_cols[src]
    np.minimum.at(best, block.dst[on].astype(np.int64), block.col_vertices[src[on]])
    return best


def _worker(rank, world, R, C, port, scale, roots, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2012_13548_gb300 import bfs2d
    from paper_2012_13548_gb300 import workloads as W
    spec = W.GraphSpec(scale=scale)
    e = oracle.kron_generate(**spec.kron_args())
    grid = bfs2d.Grid(R, C, spec.n)
    block = bfs2d.partition(e, grid, rank)
    ex = bfs2d.Exchange(dist, grid, rank)

    def step(b, f):
        best = local_step(b, f)
        return np.where(best >= grid.n, grid.n, best).astype(np.int32)

    out = []
    for r in roots:
        level, parent = bfs2d.bfs_2d(block, grid, rank, r, ex, step)
        out.append((level, parent))
    q.put((rank, out, block.dst.size))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("R,C", [(1, 2), (2, 1), (2, 2)])
def test_2d_bfs_pieces_equal_the_oracle(R, C):
    import oracle
    from paper_2012_13548_gb300 import bfs2d
    from paper_2012_13548_gb300 import workloads as W
    scale = 10
    spec = W.GraphSpec(scale=scale)
    e = oracle.kron_generate(**spec.kron_args())
    off, col = oracle.csr_build(e, scale)
    roots = [int(r) for r in W.select_roots(off, 3, spec.seeds()[3])]
    iso = int(np.nonzero(np.diff(off) == 0)[0][0])   # an isolated root reaches itself only
    roots.append(iso)
    world, port = R * C, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, R, C, port, scale, roots, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    grid = bfs2d.Grid(R, C, spec.n)
    # every directed CSR entry sits on exactly one rank
    assert sum(x[2] for x in res) == col.size
    for k, r in enumerate(roots):
        level = np.concatenate([res[q][1][k][0] for q in range(world)])
        parent = np.concatenate([res[q][1][k][1] for q in range(world)])
        p_ref, l_ref = oracle.bfs(off, col, r)
        assert np.array_equal(level, l_ref), (R, C, r)
        assert np.array_equal(parent, p_ref), (R, C, r)


def test_grid_pieces_cover_the_vertices_once():
    from paper_2012_13548_gb300 import bfs2d
    for (R, C, n) in [(2, 2, 1000), (3, 2, 1 << 12), (1, 5, 17)]:
        g = bfs2d.Grid(R, C, n)
        allv = np.concatenate([np.arange(*g.piece_range(q)) for q in range(g.P)])
        assert np.array_equal(allv, np.arange(n))
        v = np.arange(n)
        q = g.piece_of(v)
        lo = np.array([g.piece_range(x)[0] for x in q])
        hi = np.array([g.piece_range(x)[1] for x in q])
        assert ((lo <= v) & (v < hi)).all()
        # each piece lies in exactly one row block and one column block
        for i in range(R):
            for j in range(C):
                assert set(g.row_pieces(i)) & set(g.col_pieces(j)) == {i * C + j}
