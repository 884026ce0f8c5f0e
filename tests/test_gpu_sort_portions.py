"""The chained (multi-portion) path of the device radix sort, against the oracle.

kron_generate and kernel 1 sort their keys with one radix sort.  A sort of more
keys than one portion (2^28 by default: kernel 1 from SCALE 24 up, the SCALE 26
shuffle) runs portion by portion, each portion's digit counts giving the next
one's output positions.  gb_set_sort_portion makes the portions small, so the
same chained path runs here on graphs the oracle builds in seconds: two, three
and many portions, portion sizes that are not a multiple of the sort's tile,
and a last portion of a single key.  Every output must equal the oracle's bit
for bit (Sec. 2.1 edge list, Sec. 2.2 CSR), as it does with one portion.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2012_13548_gb300 as gb  # noqa: E402
from paper_2012_13548_gb300 import workloads as W  # noqa: E402
from tests.conftest import oracle_bfs, oracle_graph, roots_for  # noqa: E402

pytestmark = pytest.mark.gpu

DEFAULT_PORTION = 1 << 28


@pytest.fixture(autouse=True)
def _restore_portion():
    gb.sort_portion(0)
    gb.bfs_set_options(canonical_parents=0)
    yield
    gb.sort_portion(0)
    gb.bfs_set_options(canonical_parents=0)
    gb.gb_device_status()


def np_(t):
    return t.cpu().numpy()


def portions_for(nkeys):
    """Portion sizes that split a sort of nkeys keys into 2, 3 and many
    portions; sizes off the 8192-key tile, and one leaving a 1-key last portion."""
    return sorted({(nkeys + 1) // 2, (nkeys + 2) // 3, 5000, 8192 + 7, nkeys - 1})


def test_portion_setting_round_trips_and_rejects_bad_sizes():
    assert gb.sort_portion() == DEFAULT_PORTION
    assert gb.sort_portion(12345) == 12345
    assert gb.sort_portion(0) == DEFAULT_PORTION
    for bad in (-1, DEFAULT_PORTION + 1):
        with pytest.raises(gb.GbError, match="INVALID"):
            gb.sort_portion(bad)
    assert gb.sort_portion() == DEFAULT_PORTION


@pytest.mark.parametrize("scale", [12, 16])
def test_generator_with_portions_equals_the_oracle(scale):
    # the generator sorts n vertex hashes (permutation) and m tuple hashes (shuffle)
    spec = W.GraphSpec(scale=scale)
    e_ref, _, _ = oracle_graph(scale)
    for p in portions_for(spec.n) + portions_for(spec.m):
        if p < 2:
            continue
        gb.sort_portion(p)
        e = gb.kron_generate(**spec.kron_args())
        assert np.array_equal(np_(e), e_ref), p


# 12, 16, 20: 8-bit digit passes only; 13 (9, 9, 8), 17 (9, 9, 8, 8) and 18
# (four 9-bit passes) exercise the 512-digit passes and their chained bases.
@pytest.mark.parametrize("scale", [12, 13, 16, 17, 18, 20])
def test_kernel1_with_portions_equals_the_oracle(scale):
    spec = W.GraphSpec(scale=scale)
    e_ref, off_ref, col_ref = oracle_graph(scale)
    e = torch.as_tensor(e_ref).cuda()
    nkeys = 2 * spec.m   # both symmetric keys of every tuple
    sizes = portions_for(nkeys) if scale < 20 else [(nkeys + 2) // 3, 1 << 20]
    for p in sizes:
        gb.sort_portion(p)
        g = gb.graph_build_csr(e, scale)
        off, col = g.csr()
        assert np.array_equal(np_(off), off_ref), p
        assert np.array_equal(np_(col), col_ref), p
        g.free()


@pytest.mark.parametrize("scale", [12, 16])
def test_fused_generate_build_with_portions_equals_the_oracle(scale):
    spec = W.GraphSpec(scale=scale)
    _, off_ref, col_ref = oracle_graph(scale)
    for p in [(2 * spec.m + 1) // 2, (2 * spec.m + 2) // 3, 5000]:
        gb.sort_portion(p)
        g = gb.graph_generate_csr(**spec.kron_args())
        off, col = g.csr()
        assert np.array_equal(np_(off), off_ref), p
        assert np.array_equal(np_(col), col_ref), p
        g.free()


def test_counting_sort_long_rows_with_portions_equal_the_oracle():
    # the counting-sort kernel 1 radix-sorts the entries of rows longer than
    # 4096 together; a hub of 12000 repeated neighbours gives that sort work
    rng = np.random.default_rng(29)
    scale = 13
    n = 1 << scale
    hub = np.stack([np.zeros(12000, dtype=np.int64), rng.integers(1, n, 12000)])
    hub2 = np.stack([rng.integers(0, n, 9000), np.full(9000, 5, dtype=np.int64)])
    rnd = rng.integers(0, n, size=(2, 2 * n))
    e = np.concatenate([hub, hub2, rnd], axis=1).astype(np.int64)
    off_ref, col_ref = oracle.csr_build(e, scale)
    for p in [4099, 10000, 8192 * 3 + 1]:
        gb.sort_portion(p)
        g = gb.graph_build_csr_counting(torch.as_tensor(e).cuda(), scale)
        off, col = g.csr()
        assert np.array_equal(np_(off), off_ref), p
        assert np.array_equal(np_(col), col_ref), p
        g.free()


def test_weighted_kernel1_with_portions_equals_the_oracle():
    # the weighted build sorts every row again by weight (keys with values)
    scale = 12
    spec = W.GraphSpec(scale=scale)
    e_ref, _, _ = oracle_graph(scale)
    w_ref = oracle.kron_weights(e_ref.shape[1], spec.seed_weight())
    off_ref, col_ref, wgt_ref = oracle.csr_build_weighted(e_ref, w_ref, scale)
    e = torch.as_tensor(e_ref).cuda()
    w = torch.as_tensor(w_ref.astype(np.float32)).cuda()   # exact: multiples of 2^-24
    ref_units = np.rint(np.asarray(wgt_ref, dtype=np.float64) * 2.0 ** 24).astype(np.int64)
    r = roots_for(scale, 1)[0]
    for p in [(col_ref.size + 1) // 2, 5000]:
        gb.sort_portion(p)
        g = gb.graph_build_csr_weighted(e, w, scale)
        off, col = g.csr()
        assert np.array_equal(np_(off), off_ref) and np.array_equal(np_(col), col_ref), p
        assert np.array_equal(np_(g.weights()).astype(np.int64), ref_units), p
        # the weight-sorted rows are what the search reads: its distances too
        dist, _ = gb.sssp(g, r)
        d_ref, _ = oracle.sssp(off_ref, col_ref, wgt_ref, r)
        assert np.array_equal(np_(dist), d_ref), p
        g.free()


def test_search_on_a_chained_build_equals_the_oracle():
    scale = 16
    spec = W.GraphSpec(scale=scale)
    gb.sort_portion(3 * 8192 + 5)
    e = gb.kron_generate(**spec.kron_args())
    g = gb.graph_build_csr(e, scale)
    gb.bfs_set_options(canonical_parents=1)
    for r in roots_for(scale, 3):
        parent, level = gb.bfs(g, r)
        p_ref, l_ref = oracle_bfs(scale, r)
        assert np.array_equal(np_(level), l_ref) and np.array_equal(np_(parent), p_ref)
    g.free()
