"""CUDA path vs the CPU oracle, element by element (integer work: bit-exact).

Every call goes through the C ABI (libflash.so) via the thin binding.  Sizes
span several tiles / warps / row groups with ragged tails; edge cases cover
empty rows, single non-zeros, repeated and unsorted columns, the sparse/dense
insertion switch, bin counts that are not multiples of 4 or 32, the largest
bin count, heavy buckets (m >> R), k beyond the candidates and the block-level
query path.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1709_01190_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_01190_gb300 as fl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fl.build()
    assert fl.flash_device_error() == 0


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def csr_of(rows, dim):
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, dtype=np.int32) for r in rows]) if rp[-1] else np.zeros(0, np.int32)
    return synth.CSR(rp, col, None, dim)


def params_of(w):
    p = w.params
    return fl.FlashParams(p.K, p.L, p.R, p.range_bits, p.seed)


def adversarial_rows(rng, B, dim, n=300):
    rows = [[], [0], [dim - 1], [5, 5, 5], [dim - 1, 0, 7, 7, 3]]
    for m in (B // 2 - 1, B // 2, B // 2 + 1, B, 2 * B, 31, 32, 33, 1, 2, 3, 4, 5):
        if m >= 0:
            rows.append(list(rng.integers(0, dim, max(m, 0))))
    while len(rows) < n:
        m = int(rng.choice([0, 1, 2, 3, 17, B // 2, B // 2 + 1, int(rng.integers(0, 3 * B + 5))]))
        r = list(rng.integers(0, dim, m))
        if rng.random() < 0.3 and r:
            r = r + r[: len(r) // 3]  # repeats
        rng.shuffle(r)
        rows.append(r)
    return rows


HASH_SHAPES = [(1, 1), (3, 5), (4, 16), (2, 33), (4, 64), (3, 128), (4, 256), (8, 512)]


@pytest.mark.parametrize("K,L", HASH_SHAPES)
def test_doph_hashes_adversarial(K, L):
    B = K * L
    rng = np.random.default_rng(B)
    dim = 1 << 24
    c = csr_of(adversarial_rows(rng, B, dim), dim)
    p = fl.FlashParams(K, L, 4, 10, 0xABCDEF + B)
    got = u32(fl.hash_rows(p, fl.DeviceCSR.from_host(c)))
    exp = oracle.doph(c.row_ptr, c.col, K, L, p.seed)
    assert np.array_equal(got, exp)
    assert fl.flash_device_error() == 0


@pytest.mark.parametrize("order", [0, 1])
def test_doph_long_rows_every_length_class(order):
    """Rows of every length class next to each other (empty, sparse, the sparse/dense switch,
    one partial group, exact groups, many groups), in index order and longest first."""
    from paper_1709_01190_gb300 import tuning
    rng = np.random.default_rng(77)
    dim = 1 << 20
    lens = rng.choice([0, 1, 100, 129, 130, 511, 512, 513, 2047, 2048, 2049, 5000, 20000], 400)
    rows = [list(rng.integers(0, dim, int(m))) for m in lens]
    c = csr_of(rows, dim)
    p = fl.FlashParams(4, 64, 4, 12, 0x1234)
    tuning.set_tuning(tuning.Tuning(doph_order=order))
    try:
        got = u32(fl.hash_rows(p, fl.DeviceCSR.from_host(c)))
        keys = fl.row_keys(p, fl.DeviceCSR.from_host(c)).cpu().numpy().view(np.uint32)
    finally:
        tuning.set_tuning(None)
    assert np.array_equal(got, oracle.doph(c.row_ptr, c.col, p.K, p.L, p.seed))
    ek = oracle.keys(c.row_ptr, c.col, p.K, p.L, p.range_bits, p.seed)
    ek[:, np.diff(c.row_ptr) == 0] = 1 << p.range_bits
    assert np.array_equal(keys, ek)
    assert fl.flash_device_error() == 0


@pytest.mark.parametrize("lens", [
    [600] * 300 + [30_000] * 6,       # the long rows last in index order
    [10] * 800 + [5_000] * 200,       # a fifth of the rows long
    [200_000] + [10] * 7,             # one long row first, the rest tiny
])
def test_doph_long_rows_hashed_first(lens):
    """With rows of 512 or more non-zeros on average, the rows of at least 4x the average length
    (rounded up to a power of two) are hashed first and then skipped in index order: keys and
    hashes equal the oracle's wherever the long rows sit."""
    rng = np.random.default_rng(len(lens))
    dim = 1 << 22
    rows = [list(rng.integers(0, dim, m)) for m in lens]
    c = csr_of(rows, dim)
    assert c.row_ptr[-1] >= 512 * len(lens)
    p = fl.FlashParams(4, 64, 4, 14, 0x51ED)
    dev = fl.DeviceCSR.from_host(c)
    got_k = u32(fl.row_keys(p, dev))
    got_h = u32(fl.hash_rows(p, dev))
    assert np.array_equal(got_k, oracle.keys(c.row_ptr, c.col, p.K, p.L, p.range_bits, p.seed))
    assert np.array_equal(got_h, oracle.doph(c.row_ptr, c.col, p.K, p.L, p.seed))
    assert fl.flash_device_error() == 0


# ---------------------------------------------- optimal densification ([36])


@pytest.mark.parametrize("K,L", [(1, 1), (3, 5), (4, 16), (2, 33), (4, 256), (8, 512)])
def test_doph_optimal_densification_adversarial(K, L):
    B = K * L
    rng = np.random.default_rng(B + 5)
    dim = 1 << 24
    c = csr_of(adversarial_rows(rng, B, dim), dim)
    p = fl.FlashParams(K, L, 4, 10, 0xABCDEF + B, densify=1)
    got = u32(fl.hash_rows(p, fl.DeviceCSR.from_host(c)))
    assert np.array_equal(got, oracle.doph(c.row_ptr, c.col, K, L, p.seed, densify=1))
    assert fl.flash_device_error() == 0


@pytest.mark.parametrize("name,n", [("kdd12_like", 20_000), ("url_like_batched", 4_000), ("tiny_plain", 3_000)])
def test_doph_optimal_densification_workloads(name, n):
    """Sparse rows (kdd12-like: about 12 non-zeros in 1,024 bins) densify most bins."""
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p0 = params_of(w)
    p = fl.FlashParams(p0.K, p0.L, p0.R, p0.range_bits, p0.seed, densify=1)
    dev = fl.DeviceCSR.from_host(c)
    got = u32(fl.hash_rows(p, dev))
    assert np.array_equal(got, oracle.doph(c.row_ptr, c.col, p.K, p.L, p.seed, densify=1))
    keys = fl.row_keys(p, dev).cpu().numpy().view(np.uint32)
    ek = oracle.keys(c.row_ptr, c.col, p.K, p.L, p.range_bits, p.seed, densify=1)
    ek[:, np.diff(c.row_ptr) == 0] = 1 << p.range_bits
    assert np.array_equal(keys, ek)


@pytest.mark.parametrize("name,n,over", [("kdd12_like", 15_000, dict(range_bits=13, L=64)),
                                         ("tiny_plain", 6_000, None)])
def test_knn_graph_optimal_densification(name, n, over):
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p0 = _params_override(w, over)
    p = fl.FlashParams(p0.K, p0.L, p0.R, p0.range_bits, p0.seed, densify=1)
    ids, cnt = fl.knn_graph(p, fl.DeviceCSR.from_host(c), w.k)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, w.k, densify=1)
    assert np.array_equal(ids.cpu().numpy(), ei)
    assert np.array_equal(cnt.cpu().numpy(), en)


def test_doph_column_array_not_16_byte_aligned():
    """A column array starting 4, 8 or 12 bytes past a 16-byte boundary (a slice): the
    kernels find each row's 16-byte body from the actual address; a pointer that is not
    even 4-byte aligned is rejected on the host."""
    w = synth.WORKLOADS["webspam_like"].scaled(600)
    c = synth.generate(w.data.replace(with_val=False))
    p = fl.FlashParams(4, 64, 8, 12, 7)
    exp = oracle.doph(c.row_ptr, c.col, p.K, p.L, p.seed)
    for shift in (1, 2, 3):
        big = torch.zeros(c.nnz + 8, dtype=torch.int32, device="cuda")
        big[shift:shift + c.nnz] = torch.from_numpy(c.col).cuda()
        dev = fl.DeviceCSR(torch.from_numpy(c.row_ptr).cuda(), big[shift:shift + c.nnz], c.dim)
        assert dev.col.data_ptr() % 16 == 4 * shift
        got = fl.hash_rows(p, dev).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, exp), shift
    assert fl.flash_device_error() == 0
    raw = torch.zeros(c.nnz + 4, dtype=torch.int32, device="cuda")
    x = fl._lib.Csr(torch.from_numpy(c.row_ptr).cuda().data_ptr(), raw.data_ptr() + 2, None, c.n_rows, int(c.nnz),
                    int(c.dim))
    out = torch.empty((c.n_rows, p.K * p.L), dtype=torch.int32, device="cuda")
    rc = fl._lib.lib().flash_hash(ctypes.byref(p.c()), ctypes.byref(x), out.data_ptr(), None)
    assert rc == 1  # FLASH_EINVAL


def test_doph_hashes_unaligned_output_and_tail():
    K, L = 4, 16
    c = synth.generate(synth.WORKLOADS["tiny_plain"].data.replace(n_rows=777, n_clusters=10))
    p = fl.FlashParams(K, L, 4, 10, 99)
    buf = torch.empty(c.n_rows * K * L + 1, dtype=torch.int32, device="cuda")
    view = buf[1:]  # 4-byte aligned, not 16-byte aligned: scalar store path
    fl.flash_hash(p, fl.DeviceCSR.from_host(c), view)
    assert np.array_equal(u32(view).reshape(c.n_rows, K * L), oracle.doph(c.row_ptr, c.col, K, L, 99))


@pytest.mark.parametrize("name,n", [("tiny_plain", 10_000), ("webspam_like", 1500), ("url_like_batched", 20_000),
                                    ("kdd12_like", 30_000)])
def test_doph_hashes_workloads(name, n):
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = params_of(w)
    got = u32(fl.hash_rows(p, fl.DeviceCSR.from_host(c)))
    assert np.array_equal(got, oracle.doph(c.row_ptr, c.col, p.K, p.L, p.seed))


@pytest.mark.parametrize("name,n", [("tiny_plain", 10_000), ("webspam_like", 1200), ("url_like_batched", 15_000),
                                    ("kdd12_like", 20_000)])
def test_keys_workloads(name, n):
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = params_of(w)
    got = u32(fl.row_keys(p, fl.DeviceCSR.from_host(c)))
    exp = oracle.keys(c.row_ptr, c.col, p.K, p.L, p.range_bits, p.seed)
    empty = np.diff(c.row_ptr) == 0
    exp[:, empty] = 1 << p.range_bits
    assert np.array_equal(got, exp)


def test_keys_adversarial():
    K, L, rb = 3, 40, 7
    rng = np.random.default_rng(3)
    c = csr_of(adversarial_rows(rng, K * L, 1 << 20, n=500), 1 << 20)
    p = fl.FlashParams(K, L, 4, rb, 1234)
    got = u32(fl.row_keys(p, fl.DeviceCSR.from_host(c)))
    exp = oracle.keys(c.row_ptr, c.col, K, L, rb, 1234)
    exp[:, np.diff(c.row_ptr) == 0] = 1 << rb
    assert np.array_equal(got, exp)


# The sort partitions each table by the address bits above the low 10, in
# passes of at most 8 bits, then sorts every segment of 2^10 buckets by one warp.
BUILD_CASES = [
    ("tiny_plain", 10_000, None),
    ("tiny_plain", 3_001, dict(range_bits=6, R=3)),       # many heavy buckets
    ("tiny_plain", 2_500, dict(range_bits=3, R=1)),       # R = 1, every bucket heavy
    ("tiny_plain", 4_000, dict(range_bits=9, R=200, L=4)),  # R above every occupancy
    ("url_like_batched", 30_000, dict(range_bits=12)),   # Zipf heavy buckets, R = 128
    ("kdd12_like", 40_000, dict(range_bits=13, L=32)),
    ("kdd12_like", 30_000, dict(range_bits=20, L=4, R=2)),          # 10 high bits: two passes
    ("url_like_batched", 20_000, dict(range_bits=21, L=2, R=4, K=2)),  # 11 high bits: two passes
    ("url_like_batched", 20_000, dict(range_bits=19, L=2, R=4)),    # 9 high bits: two passes
    ("tiny_plain", 20_000, dict(range_bits=24, L=1, R=2)),          # 14 high bits, segments mostly empty
    ("webspam_like", 5_000, dict(range_bits=18, L=8)),              # 8 high bits: one pass
    ("tiny_plain", 5_000, dict(range_bits=10, R=4)),                # no high bits: one segment per table
    ("tiny_plain", 100_000, dict(range_bits=10, L=2, R=8)),         # one warp places 100,000 points
    ("tiny_plain", 5_000, dict(range_bits=1, R=64, L=3)),            # two buckets: m >> R everywhere
]


def _params_override(w, over):
    p = params_of(w)
    if over:
        p = fl.FlashParams(over.get("K", p.K), over.get("L", p.L), over.get("R", p.R),
                           over.get("range_bits", p.range_bits), p.seed)
    return p


@pytest.mark.parametrize("name,n,over", BUILD_CASES)
def test_build_tables(name, n, over):
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = _params_override(w, over)
    ix = fl.flash_build(p, fl.DeviceCSR.from_host(c))
    tables, counts = ix.export()
    et, ec = oracle.build_tables(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed)
    assert np.array_equal(u32(counts).reshape(ec.shape), ec)
    assert np.array_equal(tables.cpu().numpy(), et)
    ix.free()


def test_build_with_empty_rows_and_edge_columns():
    rng = np.random.default_rng(11)
    dim = 5000
    c = csr_of(adversarial_rows(rng, 24, dim, n=2000), dim)
    p = fl.FlashParams(3, 8, 5, 5, 77)
    ix = fl.flash_build(p, fl.DeviceCSR.from_host(c))
    tables, counts = ix.export()
    et, ec = oracle.build_tables(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed)
    assert np.array_equal(u32(counts).reshape(ec.shape), ec)
    assert np.array_equal(tables.cpu().numpy(), et)


QUERY_CASES = [
    ("tiny_plain", 10_000, None, 10, 0),
    ("tiny_plain", 6_000, dict(range_bits=7, R=16), 25, 0),
    ("url_like_batched", 20_000, dict(range_bits=12), 64, 0),
    ("url_like_batched", 20_000, dict(range_bits=12), 64, 64),   # warp table too small: block path
    ("kdd12_like", 30_000, dict(range_bits=14), 32, 0),
    ("tiny_plain", 3_000, dict(range_bits=5, R=8), 1, 0),
    ("tiny_plain", 3_000, dict(range_bits=5, R=8), 300, 0),      # k > 256: block path only
    # block path, second tier: most reservoirs full (M near L*R = 16384 > the 64 KB table's 10922)
    ("url_like_batched", 20_000, dict(range_bits=6, K=1), 64, 0),
    # both block tiers mixed (M spread around 10922), k = 200 written at their ranks by the block
    ("url_like_batched", 20_000, dict(range_bits=8, K=1), 200, 64),
    # k > 256 with second-tier queries: every query on the block path, block bitonic sort
    ("url_like_batched", 20_000, dict(range_bits=7, K=1), 300, 0),
    # block path with fewer distinct candidates than k (every candidate is output, then padding)
    ("tiny_plain", 3_000, dict(range_bits=9, R=8), 100, 64),
]


@pytest.mark.parametrize("name,n,over,k,wt", QUERY_CASES)
def test_query_sampled_rows_with_exclusion(name, n, over, k, wt):
    from paper_1709_01190_gb300 import tuning
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = _params_override(w, over)
    dev = fl.DeviceCSR.from_host(c)
    ix = fl.flash_build(p, dev)
    qids = synth.sample_rows(c.n_rows, min(400, c.n_rows), seed=5)
    sub = c.rows(qids)
    excl = torch.from_numpy(qids.astype(np.int32)).cuda()
    if wt:  # a warp table this small sends most queries to the block path
        tuning.set_tuning(tuning.Tuning(query_warp_table=wt))
    try:
        ids, cnt = fl.query(ix, fl.DeviceCSR.from_host(sub), k, excl)
    finally:
        tuning.set_tuning(None)
    et, ec = oracle.build_tables(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed)
    ei, en = oracle.query(et, ec, p.K, p.L, p.R, p.range_bits, p.seed, sub.row_ptr, sub.col, k,
                          exclude=qids.astype(np.int32))
    assert fl.flash_device_error() == 0
    assert np.array_equal(ids.cpu().numpy(), ei)
    assert np.array_equal(cnt.cpu().numpy(), en)


def test_query_fresh_rows_no_exclusion():
    w = synth.WORKLOADS["url_like_batched"].scaled(25_000, n_queries=3_000)
    c = synth.generate(w.data)
    qc = synth.generate(w.query_data)
    p = _params_override(w, dict(range_bits=13))
    ix = fl.flash_build(p, fl.DeviceCSR.from_host(c))
    ids, cnt = fl.query(ix, fl.DeviceCSR.from_host(qc), w.k)
    et, ec = oracle.build_tables(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed)
    ei, en = oracle.query(et, ec, p.K, p.L, p.R, p.range_bits, p.seed, qc.row_ptr, qc.col, w.k)
    assert np.array_equal(ids.cpu().numpy(), ei) and np.array_equal(cnt.cpu().numpy(), en)


@pytest.mark.parametrize("name,n,over", [("tiny_plain", 10_000, None), ("webspam_like", 2_000, dict(range_bits=12)),
                                         ("kdd12_like", 25_000, dict(range_bits=13)),
                                         ("url_like_batched", 12_000, dict(range_bits=11))])
def test_knn_graph(name, n, over):
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = _params_override(w, over)
    ids, cnt = fl.knn_graph(p, fl.DeviceCSR.from_host(c), w.k)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, w.k)
    assert np.array_equal(ids.cpu().numpy(), ei)
    assert np.array_equal(cnt.cpu().numpy(), en)


def test_knn_graph_host_buffers_match_device():
    w = synth.WORKLOADS["tiny_plain"].scaled(5_000)
    c = synth.generate(w.data)
    p = params_of(w)
    ids, cnt = fl.knn_graph(p, fl.DeviceCSR.from_host(c), w.k)
    hi = np.empty((c.n_rows, w.k), np.int32)
    hc = np.empty((c.n_rows, w.k), np.int32)
    fl.flash_knn_graph_host(p, c.row_ptr, c.col, c.dim, w.k, hi, hc)  # pageable: copied first
    assert np.array_equal(hi, ids.cpu().numpy()) and np.array_equal(hc, cnt.cpu().numpy())
    # pinned inputs and outputs: the CSR is read in place by the hashing kernel
    rp = torch.from_numpy(c.row_ptr).pin_memory()
    col = torch.from_numpy(c.col).pin_memory()
    pi = torch.empty((c.n_rows, w.k), dtype=torch.int32).pin_memory()
    pc = torch.empty_like(pi).pin_memory()
    fl.flash_knn_graph_host(p, rp.numpy(), col.numpy(), c.dim, w.k, pi.numpy(), pc.numpy())
    assert np.array_equal(pi.numpy(), ids.cpu().numpy()) and np.array_equal(pc.numpy(), cnt.cpu().numpy())


def test_graph_is_deterministic_across_runs():
    w = synth.WORKLOADS["kdd12_like"].scaled(20_000)
    c = synth.generate(w.data)
    p = params_of(w)
    dev = fl.DeviceCSR.from_host(c)
    a = fl.knn_graph(p, dev, w.k)
    b = fl.knn_graph(p, dev, w.k)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


# ------------------------------------------------------------------ errors

def test_invalid_parameters_are_rejected_on_the_host():
    c = fl.DeviceCSR.from_host(csr_of([[1, 2], [3]], 10))
    out = torch.empty((2, 4), dtype=torch.int32, device="cuda")
    for bad in (fl.FlashParams(0, 4, 4, 8, 1), fl.FlashParams(4, 0, 4, 8, 1), fl.FlashParams(4, 4, 0, 8, 1),
                fl.FlashParams(4, 4, 4, 0, 1), fl.FlashParams(4, 4, 4, 31, 1), fl.FlashParams(64, 128, 1, 8, 1),
                fl.FlashParams(1, 300, 2, 8, 1), fl.FlashParams(4, 4, 4, 8, 1, densify=2)):
        with pytest.raises(fl.FlashError) as e:
            fl.flash_knn_graph(bad, c, 4, out, out.clone())
        assert e.value.code == 1
    with pytest.raises(fl.FlashError):
        fl.flash_knn_graph(fl.FlashParams(2, 2, 4, 8, 1), c, 0, out, out.clone())


def test_bad_columns_and_row_pointers_raise_the_device_flag():
    p = fl.FlashParams(2, 4, 4, 6, 5)
    rp = torch.tensor([0, 2, 4], dtype=torch.int64, device="cuda")
    col = torch.tensor([1, 50, -3, 2], dtype=torch.int32, device="cuda")
    x = fl.DeviceCSR(rp, col, dim=10)
    fl.hash_rows(p, x)
    assert fl.flash_device_error() & fl.DEVERR_COL_RANGE
    assert fl.flash_device_error() == 0
    rp2 = torch.tensor([0, 3, 2, 9], dtype=torch.int64, device="cuda")
    x2 = fl.DeviceCSR(rp2, col, dim=10, nnz=4)
    h = fl.hash_rows(p, x2)
    assert fl.flash_device_error() & fl.DEVERR_ROW_PTR
    assert np.all(u32(h)[1:] == 0xFFFFFFFF)  # rows 1 and 2 treated as empty


def test_scratch_budget_below_need_returns_enomem_and_nothing_is_launched():
    """Host-side allocation-failure injection: a scratch budget below what a call needs makes
    flash_knn_graph and flash_query fail with FLASH_ENOMEM before any launch; the library stays
    usable, and the same calls succeed (and match the oracle) once the budget is restored."""
    w = synth.WORKLOADS["tiny_plain"].scaled(2_000)
    c = synth.generate(w.data)
    p = params_of(w)
    dev = fl.DeviceCSR.from_host(c)
    need_graph = fl.flash_knn_graph_scratch_bytes(p, c.n_rows)
    need_query = fl.flash_query_scratch_bytes(p, c.n_rows)
    assert need_graph > 0 and need_query > 0
    ix = fl.flash_build(p, dev)
    ids = torch.full((c.n_rows, w.k), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full_like(ids, -7)
    old = fl.flash_set_scratch_budget(need_graph - 1)
    try:
        with pytest.raises(fl.FlashError) as e:
            fl.flash_knn_graph(p, dev, w.k, ids, cnt)
        assert e.value.code == 2  # FLASH_ENOMEM
        assert fl.flash_last_launch_count() == 0
        fl.flash_set_scratch_budget(need_query - 1)
        with pytest.raises(fl.FlashError) as e:
            fl.flash_query(ix, dev, w.k, None, ids, cnt)
        assert e.value.code == 2
        assert fl.flash_last_launch_count() == 0
        torch.cuda.synchronize()
        assert int((ids != -7).sum()) == 0  # nothing was written
        fl.flash_set_scratch_budget(need_query)  # exactly enough
        fl.flash_query(ix, dev, w.k, torch.arange(c.n_rows, dtype=torch.int32, device="cuda"), ids, cnt)
    finally:
        fl.flash_set_scratch_budget(old)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, w.k)
    assert np.array_equal(ids.cpu().numpy(), ei) and np.array_equal(cnt.cpu().numpy(), en)
    gi, gc = fl.knn_graph(p, dev, w.k)
    assert np.array_equal(gi.cpu().numpy(), ei) and np.array_equal(gc.cpu().numpy(), en)
    ix.free()


# ------------------------------------------------ the plain, unbatched path

PLAIN_CASES = [
    ("tiny_plain", 10_000, None, 0),
    ("tiny_plain", 2_500, dict(range_bits=3, R=1), 0),       # every bucket heavy, R = 1
    ("tiny_plain", 4_000, dict(range_bits=5, R=8), 1),       # optimal densification
    ("webspam_like", 2_000, dict(range_bits=12), 0),
    ("url_like_batched", 12_000, dict(range_bits=11), 0),    # thousands of candidates per query
    ("kdd12_like", 25_000, dict(range_bits=13), 0),          # B = 1024, most bins densified
]


@pytest.mark.parametrize("name,n,over,densify", PLAIN_CASES)
def test_knn_graph_plain_path(name, n, over, densify):
    """flash_knn_graph_plain (the baseline) gives the oracle's graph, element by element."""
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p0 = _params_override(w, over)
    p = fl.FlashParams(p0.K, p0.L, p0.R, p0.range_bits, p0.seed, densify=densify)
    ids, cnt = fl.knn_graph_plain(p, fl.DeviceCSR.from_host(c), w.k)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, w.k, densify=densify)
    assert fl.flash_device_error() == 0
    assert np.array_equal(ids.cpu().numpy(), ei)
    assert np.array_equal(cnt.cpu().numpy(), en)


def test_knn_graph_plain_path_with_empty_rows_and_edge_columns():
    rng = np.random.default_rng(12)
    dim = 5000
    c = csr_of(adversarial_rows(rng, 24, dim, n=1500), dim)
    p = fl.FlashParams(3, 8, 5, 5, 77)
    ids, cnt = fl.knn_graph_plain(p, fl.DeviceCSR.from_host(c), 7)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, 7)
    assert np.array_equal(ids.cpu().numpy(), ei) and np.array_equal(cnt.cpu().numpy(), en)


# ------------------------------------------ ADD continued (Algorithm 2 as a stream)

ADD_CASES = [
    ("tiny_plain", 6_000, dict(range_bits=6, R=3), [2_000, 1_500, 2_500]),   # every bucket overflows
    ("tiny_plain", 4_000, dict(range_bits=3, R=1), [1, 3_000, 999]),        # R = 1, one-row batch
    ("tiny_plain", 5_000, None, [4_000, 1_000]),
    ("url_like_batched", 16_000, dict(range_bits=12), [9_000, 7_000]),       # Zipf heavy buckets, R = 128
    ("kdd12_like", 20_000, dict(range_bits=13, L=32), [12_000, 8_000]),
    ("webspam_like", 3_000, dict(range_bits=10, L=8), [1_000, 2_000]),
]


@pytest.mark.parametrize("name,n,over,parts", ADD_CASES)
def test_add_continues_every_bucket_like_one_build(name, n, over, parts):
    """flash_build on the first rows, then flash_add of the rest in batches: the tables equal the
    oracle's build over all rows slot for slot (counts included), and queries agree with the oracle."""
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = _params_override(w, over)
    assert sum(parts) == c.n_rows
    r0 = parts[0]
    ix = fl.flash_build(p, fl.DeviceCSR.from_host(c.slice(0, r0)))
    for sz in parts[1:]:
        fl.flash_add(ix, fl.DeviceCSR.from_host(c.slice(r0, r0 + sz)))
        r0 += sz
    assert ix.n_rows == c.n_rows and ix.info()["n_rows"] == c.n_rows
    tables, counts = ix.export()
    et, ec = oracle.build_tables(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed)
    assert np.array_equal(u32(counts).reshape(ec.shape), ec)
    assert np.array_equal(tables.cpu().numpy(), et)
    # the same tables through the oracle's own ADD on the same batches
    ot, oc = oracle.build_tables(c.row_ptr[:parts[0] + 1], c.col[:int(c.row_ptr[parts[0]])], p.K, p.L, p.R,
                                 p.range_bits, p.seed)
    r0 = parts[0]
    for sz in parts[1:]:
        sub = c.slice(r0, r0 + sz)
        oracle.add_rows(ot, oc, sub.row_ptr, sub.col, r0, p.K, p.L, p.R, p.range_bits, p.seed)
        r0 += sz
    assert np.array_equal(ot, et) and np.array_equal(oc, ec)
    qids = synth.sample_rows(c.n_rows, min(300, c.n_rows), seed=9)
    sub = c.rows(qids)
    ids, cnt = fl.query(ix, fl.DeviceCSR.from_host(sub), w.k, torch.from_numpy(qids.astype(np.int32)).cuda())
    ei, en = oracle.query(et, ec, p.K, p.L, p.R, p.range_bits, p.seed, sub.row_ptr, sub.col, w.k,
                          exclude=qids.astype(np.int32))
    assert np.array_equal(ids.cpu().numpy(), ei) and np.array_equal(cnt.cpu().numpy(), en)
    assert fl.flash_device_error() == 0
    ix.free()


def test_add_rows_with_empty_rows_and_an_empty_batch():
    rng = np.random.default_rng(21)
    dim = 3000
    c = csr_of(adversarial_rows(rng, 15, dim, n=1200), dim)
    p = fl.FlashParams(3, 5, 2, 4, 99)
    ix = fl.flash_build(p, fl.DeviceCSR.from_host(c.slice(0, 500)))
    fl.flash_add(ix, fl.DeviceCSR.from_host(c.slice(500, 500)))  # no rows: nothing changes
    fl.flash_add(ix, fl.DeviceCSR.from_host(c.slice(500, 1200)))
    tables, counts = ix.export()
    et, ec = oracle.build_tables(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed)
    assert np.array_equal(u32(counts).reshape(ec.shape), ec)
    assert np.array_equal(tables.cpu().numpy(), et)
    ix.free()


# ------------------------------------------------ reservoir sharing (Section 3.5)

SHARE_CASES = [
    ("tiny_plain", 5_000, dict(range_bits=9, R=8), 700, 0),          # F ~ 0.09: shared reservoirs overflow
    ("tiny_plain", 3_000, dict(range_bits=6, R=4, L=6), 1, 0),        # one reservoir for every bucket
    ("tiny_plain", 4_000, None, 150_000, 1),                         # optimal densification, F ~ 0.29
    ("url_like_batched", 12_000, dict(range_bits=11), 80_000, 0),    # thousands of candidates per query
    ("kdd12_like", 20_000, dict(range_bits=13, L=32), 70_000, 0),    # F ~ 0.27
    ("kdd12_like", 8_000, dict(range_bits=12, L=16), 1_000_000, 0),  # a pool larger than the range (F ~ 15)
]


@pytest.mark.parametrize("name,n,over,P,densify", SHARE_CASES)
def test_reservoir_sharing_tables_queries_and_graph(name, n, over, P, densify):
    """Build, export, query and k-NN graph with one shared pool of P reservoirs, each against the
    oracle's shared index, element by element."""
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p0 = _params_override(w, over)
    p = fl.FlashParams(p0.K, p0.L, p0.R, p0.range_bits, p0.seed, densify=densify, share_pool=P)
    dev = fl.DeviceCSR.from_host(c)
    ix = fl.flash_build(p, dev)
    tables, counts = ix.export()
    et, ec = oracle.build_tables_shared(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, P, densify=densify)
    assert np.array_equal(u32(counts), ec)
    assert np.array_equal(tables.cpu().numpy(), et)
    qids = synth.sample_rows(c.n_rows, min(300, c.n_rows), seed=17)
    sub = c.rows(qids)
    ids, cnt = fl.query(ix, fl.DeviceCSR.from_host(sub), w.k, torch.from_numpy(qids.astype(np.int32)).cuda())
    ei, en = oracle.query_shared(et, ec, p.K, p.L, p.R, p.range_bits, p.seed, P, sub.row_ptr, sub.col, w.k,
                                 exclude=qids.astype(np.int32), densify=densify)
    assert np.array_equal(ids.cpu().numpy(), ei) and np.array_equal(cnt.cpu().numpy(), en)
    gi, gc = fl.knn_graph(p, dev, w.k)
    gei, gec = oracle.knn_graph_shared(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, w.k, P,
                                       densify=densify)
    assert np.array_equal(gi.cpu().numpy(), gei) and np.array_equal(gc.cpu().numpy(), gec)
    assert fl.flash_device_error() == 0
    ix.free()


def test_reservoir_sharing_is_rejected_where_unsupported():
    c = synth.generate(synth.WORKLOADS["tiny_plain"].data.replace(n_rows=500, n_clusters=10))
    p = fl.FlashParams(2, 4, 4, 8, 3, share_pool=100)
    dev = fl.DeviceCSR.from_host(c)
    ix = fl.flash_build(p, dev)
    with pytest.raises(fl.FlashError) as e:
        fl.flash_add(ix, dev)
    assert e.value.code == 1
    with pytest.raises(fl.FlashError) as e:
        fl.knn_graph_plain(p, dev, 5)
    assert e.value.code == 1
    with pytest.raises(fl.FlashError) as e:
        fl.flash_build(fl.FlashParams(2, 4, 4, 8, 3, share_pool=(1 << 30) + 1), dev)
    assert e.value.code == 1
    ix.free()


# ------------------------------------- quality measures of Section 4.3 (GPU evaluator)

@pytest.mark.parametrize("name,n,over", [("tiny_plain", 6_000, None), ("kdd12_like", 40_000, dict(range_bits=14)),
                                         ("url_like_batched", 15_000, dict(range_bits=12))])
def test_quality_evaluator_matches_brute_force_cosines(name, n, over):
    """flash_eval_quality: each query's nearest neighbour (exact, ties to the smaller id) equals the
    oracle's, its cosine and the mean cosine of the reported ids agree to 1e-12, and R@k / S@k follow."""
    from oracle import quality
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = _params_override(w, over)
    dev = fl.DeviceCSR.from_host(c)
    ids, _ = fl.knn_graph(p, dev, w.k)
    qs = synth.sample_rows(c.n_rows, 150, seed=31)
    q_t = torch.from_numpy(qs.astype(np.int32)).cuda()
    rep = ids[q_t.long()].contiguous()
    got = fl.quality(dev, q_t, rep)
    sim = quality.cosine_to_all(c.row_ptr, c.col, c.dim, qs)
    nn = quality.nearest_neighbours_of_sets(c.row_ptr, c.col, c.dim, qs)
    rep_np = rep.cpu().numpy()
    assert np.array_equal(got["nn"].cpu().numpy(), nn)
    assert np.allclose(got["nn_sim"].cpu().numpy(), sim[np.arange(len(qs)), nn], rtol=0, atol=1e-12)
    per_q = np.array([sim[i, rep_np[i][rep_np[i] >= 0]].mean() if (rep_np[i] >= 0).any() else 0.0
                      for i in range(len(qs))])
    assert np.allclose(got["sim_at_k"].cpu().numpy(), per_q, rtol=0, atol=1e-12)
    assert abs(got["R@k"] - quality.recall_at_k(rep_np, nn)) <= 1e-12
    assert abs(got["S@k"] - quality.similarity_at_k(rep_np, sim)) <= 1e-12
