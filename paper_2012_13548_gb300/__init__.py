"""GB300-native Graph500 kernels 1, 2 and 3 (arXiv 2012.13548, Sec. 2).

The compute path is the CUDA library built from ``csrc/`` (sm_103a); this
package only loads it (``binding``) and holds the seeded input recipes
(``workloads``).
"""
from .binding import (GbError, Graph, Server, bfs, bfs_batch, bfs_noalloc, bfs_get_options,  # noqa: F401
                      bfs_last_stats, bfs_validate, bfs_multi_graph, bfs_set_options, debug_fail_allocations,
                      debug_live_allocations, gb_device_status,
                      gb_kernel_launches, graph_build_csr, graph_build_csr_counting,
                      graph_build_csr_weighted, graph_from_csr, graph_generate_csr, kron_generate,
                      kron_weights, lib, sort_portion, sssp, sssp_last_stats, sssp_validate)
