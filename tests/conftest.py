import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


import functools  # noqa: E402

import numpy as np  # noqa: E402


@functools.lru_cache(maxsize=None)
def oracle_graph(scale, index=-1):
    """(edges [2, m], off, col) of the oracle for the workload graph of `scale`
    (graph `index` of a batch when index >= 0).  Cached per test session."""
    import oracle
    from paper_2012_13548_gb300 import workloads as W
    spec = W.GraphSpec(scale=scale, index=index)
    e = oracle.kron_generate(**spec.kron_args())
    off, col = oracle.csr_build(e, scale)
    return e, off, col


@functools.lru_cache(maxsize=None)
def oracle_bfs(scale, root, index=-1):
    import oracle
    _, off, col = oracle_graph(scale, index)
    return oracle.bfs(off, col, root)


def roots_for(scale, k, index=-1):
    from paper_2012_13548_gb300 import workloads as W
    _, off, _ = oracle_graph(scale, index)
    return [int(r) for r in W.select_roots(off, k, W.GraphSpec(scale=scale, index=index).seeds()[3])]
