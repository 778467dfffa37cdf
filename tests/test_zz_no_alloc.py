"""flash_query_noalloc: the query entry point that allocates no device memory.

It serves callers that must not allocate device memory (a latency-critical
serving thread, where cudaMalloc can block, synchronize the device or fail
under memory pressure; or a program whose device memory belongs entirely to
its own pool).  Its scratch is one fixed library-owned device array shared by
all calls, so this test calls it twice in a row through the C ABI and checks
each result element by element against flash_query (integer results: exact).
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1709_01190_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_01190_gb300 as fl  # noqa: E402
from paper_1709_01190_gb300._lib import Csr, lib  # noqa: E402


@pytest.fixture(scope="module")
def index_and_queries():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fl.build()
    w = synth.WORKLOADS["url_like_batched"].scaled(20_000, n_queries=2_500)
    c = synth.generate(w.data)
    p = w.params
    params = fl.FlashParams(p.K, p.L, p.R, 12, p.seed)
    ix = fl.flash_build(params, fl.DeviceCSR.from_host(c))
    qa = fl.DeviceCSR.from_host(synth.generate(w.query_data))
    qb = fl.DeviceCSR.from_host(c.rows(synth.sample_rows(c.n_rows, 1_700, seed=3)))
    yield ix, qa, qb, w.k
    ix.free()


def _noalloc(ix, q, k, exclude=None):
    ids = torch.full((q.n_rows, k), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((q.n_rows, k), -7, dtype=torch.int32, device="cuda")
    c = q.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().flash_query_noalloc(ix.handle, ctypes.byref(c), k,
                                   None if exclude is None else ctypes.c_void_p(exclude.data_ptr()),
                                   ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(cnt.data_ptr()), stream)
    assert rc == 0, fl.flash_strerror(rc)
    torch.cuda.synchronize()
    return ids, cnt


def test_noalloc_query_matches_flash_query_twice_in_a_row(index_and_queries):
    ix, qa, qb, k = index_and_queries
    excl_b = torch.arange(qb.n_rows, dtype=torch.int32, device="cuda") * 3
    ra = _noalloc(ix, qa, k)
    rb = _noalloc(ix, qb, k, excl_b)
    ea = fl.query(ix, qa, k)
    eb = fl.query(ix, qb, k, excl_b)
    torch.cuda.synchronize()
    assert torch.equal(ra[0], ea[0]) and torch.equal(ra[1], ea[1])
    assert torch.equal(rb[0], eb[0]) and torch.equal(rb[1], eb[1])
    # the shared scratch keeps the previous call's contents: a repeat must still agree
    ra2 = _noalloc(ix, qa, k)
    assert torch.equal(ra2[0], ea[0]) and torch.equal(ra2[1], ea[1])


def test_noalloc_query_rejects_batches_beyond_its_scratch(index_and_queries):
    ix, qa, _, k = index_and_queries
    big = Csr(qa.row_ptr.data_ptr(), qa.col.data_ptr(), None, 10_000_000, int(qa.nnz), int(qa.dim))
    out = torch.empty(8, dtype=torch.int32, device="cuda")
    rc = lib().flash_query_noalloc(ix.handle, ctypes.byref(big), k, None, ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1  # FLASH_EINVAL, nothing launched
    assert fl.flash_device_error() == 0


def test_noalloc_query_keeps_the_index_densification():
    """An index built with optimal densification hashes its queries the same way."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    fl.build()
    w = synth.WORKLOADS["kdd12_like"].scaled(8_000)
    c = synth.generate(w.data)
    p = w.params
    params = fl.FlashParams(p.K, 32, p.R, 12, p.seed, densify=1)
    ix = fl.flash_build(params, fl.DeviceCSR.from_host(c))
    q = c.rows(synth.sample_rows(c.n_rows, 500, seed=4))
    dq = fl.DeviceCSR.from_host(q)
    got = _noalloc(ix, dq, w.k)
    exp = fl.query(ix, dq, w.k)
    torch.cuda.synchronize()
    assert torch.equal(got[0], exp[0]) and torch.equal(got[1], exp[1])
    et, ec = oracle.build_tables(c.row_ptr, c.col, params.K, params.L, params.R, params.range_bits, params.seed,
                                 densify=1)
    ei, en = oracle.query(et, ec, params.K, params.L, params.R, params.range_bits, params.seed, q.row_ptr, q.col,
                          w.k, densify=1)
    assert np.array_equal(got[0].cpu().numpy(), ei) and np.array_equal(got[1].cpu().numpy(), en)
    ix.free()


def test_noalloc_query_needs_no_scratch_budget(index_and_queries):
    """The entry point allocates nothing: under a one-byte scratch budget it still runs and
    matches flash_query, while flash_query itself (which allocates its scratch) is refused."""
    ix, qa, _, k = index_and_queries
    exp = fl.query(ix, qa, k)
    torch.cuda.synchronize()
    old = lib().flash_set_scratch_budget(1)
    try:
        got = _noalloc(ix, qa, k)  # asserts a zero status
        ids = torch.empty((qa.n_rows, k), dtype=torch.int32, device="cuda")
        cnt = torch.empty_like(ids)
        c = qa.c()
        rc = lib().flash_query(ix.handle, ctypes.byref(c), k, None, ctypes.c_void_p(ids.data_ptr()),
                               ctypes.c_void_p(cnt.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 2  # FLASH_ENOMEM: flash_query's scratch does not fit the budget
    finally:
        lib().flash_set_scratch_budget(old)
    assert torch.equal(got[0], exp[0]) and torch.equal(got[1], exp[1])
    assert lib().flash_last_launch_count() == 0  # the refused call launched nothing
