// plain.cu -- the plain, unbatched GPU path: a baseline for the optimised
// kernels, computing the same k-NN graph (bit-identical) the straightforward
// way, one launch per stage, with no persistent work claims, no row order,
// no CUDA graph and no tuned launch knobs.
//
//   hash    : one block per row; bins in shared memory (atomicMin per
//             non-zero), each empty bin densified by its own scan (rotation)
//             or probe walk (optimal densification), then the L addresses
//             (Section 2.3, Section 2.2);
//   group   : one library radix sort (CUB) of the L*n (table, address) keys
//             with the point ids as values; the sort is stable, so every
//             bucket's points stay in arrival (id) order (Algorithm 2);
//             bucket starts from the boundaries of the sorted keys;
//   reservoir: one thread per bucket runs Algorithm 1 over its arrivals;
//   query   : the paper's own GPU design (Section 3.4.1) done plainly, in
//             chunks of queries: one block per query gathers its L
//             reservoirs into global memory, a library segmented sort
//             orders every query's candidates, one block per query turns
//             each run of equal ids into a (count, id) key, a second
//             segmented sort orders those keys, and one block per query
//             writes the first k.
// The index it builds has the layout of flash_build's (ids [L][n] grouped by
// bucket, starts [L][2^rb + 1]), so both paths share the counter-based
// reservoir draw of common.cuh.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_segmented_sort.cuh>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kPlainThreads = 256;
constexpr uint32_t kNoKey = 0xFFFFFFFFu;  // sorts after every (count, id) key

// ---------------------------------------------------------------- hash
// One block per row r (blockIdx.x + row0).  Shared memory: B bins and B
// "filled" flags, then the B densified hashes.
__global__ void __launch_bounds__(kPlainThreads) plain_keys_kernel(PlainHashLaunch a, int64_t row0) {
  extern __shared__ uint32_t sm[];
  uint32_t *bins = sm;
  uint32_t *h = bins + a.B;
  unsigned char *filled = reinterpret_cast<unsigned char *>(h + a.B);
  __shared__ int any;
  const int64_t r = row0 + blockIdx.x;
  if (r >= a.n_rows) return;
  const uint32_t T = 1u << a.range_bits;
  if (threadIdx.x == 0) any = 0;
  for (uint32_t j = threadIdx.x; j < a.B; j += blockDim.x) {
    bins[j] = 0xFFFFFFFFu;
    filled[j] = 0;
  }
  __syncthreads();
  int64_t start = a.row_ptr[r], end = a.row_ptr[r + 1];
  if (start < 0 || end < start || end > a.nnz) {
    if (threadIdx.x == 0) raise_error(a.err, FLASH_DEVERR_ROW_PTR);
    start = end = 0;
  }
  for (int64_t e = start + threadIdx.x; e < end; e += blockDim.x) {
    const uint32_t c = static_cast<uint32_t>(a.col[e]);
    if (static_cast<int64_t>(c) >= a.dim || a.col[e] < 0) {
      raise_error(a.err, FLASH_DEVERR_COL_RANGE);
      continue;
    }
    const uint64_t x = a.seeds.a1 * static_cast<uint64_t>(c) + a.seeds.b1;
    const uint64_t p = (x >> 32) * static_cast<uint64_t>(a.B);
    const uint32_t bin = static_cast<uint32_t>(p >> 32);
    atomicMin(&bins[bin], static_cast<uint32_t>(p));
    filled[bin] = 1;
    any = 1;
  }
  __syncthreads();
  if (!any) {  // no entry in range: never inserted, reports nothing
    for (uint32_t t = threadIdx.x; t < a.L; t += blockDim.x) {
      a.comp[static_cast<int64_t>(t) * a.n_rows + r] = t * (T + 1u) + T;
      a.keys_rm[r * a.L + t] = T;
    }
    return;
  }
  for (uint32_t j = threadIdx.x; j < a.B; j += blockDim.x) {
    if (filled[j]) {
      h[j] = bins[j];
    } else if (a.densify == 0) {  // rotation: the first filled bin to the right, plus distance * C
      uint32_t t = 1, src = j + 1 < a.B ? j + 1 : 0;
      while (!filled[src]) {
        ++t;
        src = src + 1 < a.B ? src + 1 : 0;
      }
      h[j] = bins[src] + t * kRotStep;
    } else {  // optimal densification: the first filled bin of the bin's probe sequence
      uint32_t src = kNoKey;
      for (uint32_t i = 1; i <= 8u * a.B; ++i) {
        const uint64_t u = sm64_finalize(a.seeds.d ^ ((static_cast<uint64_t>(j) << 32) | i));
        const uint32_t pr = static_cast<uint32_t>(((u >> 32) * a.B) >> 32);
        if (filled[pr]) {
          src = pr;
          break;
        }
      }
      if (src == kNoKey) {
        src = j + 1 < a.B ? j + 1 : 0;
        while (!filled[src]) src = src + 1 < a.B ? src + 1 : 0;
      }
      h[j] = bins[src];
    }
  }
  __syncthreads();
  const int sh = 64 - static_cast<int>(a.range_bits);
  for (uint32_t t = threadIdx.x; t < a.L; t += blockDim.x) {
    uint64_t x = 0;
    for (uint32_t i = 0; i < a.K; ++i) x = x * a.seeds.a2 + h[t + i * a.L];
    const uint32_t key = static_cast<uint32_t>((a.seeds.a2 * x + a.seeds.b2) >> sh);
    a.comp[static_cast<int64_t>(t) * a.n_rows + r] = t * (T + 1u) + key;
    a.keys_rm[r * a.L + t] = key;
  }
}

// values of the sort: point id p at every (t, p)
__global__ void plain_iota_kernel(int32_t *ids, int64_t n, int64_t total) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    ids[i] = static_cast<int32_t>(i % n);
}

// starts[v] for every composite value v = t*(T+1) + b: the position of the
// first key >= v inside table t's segment of the sorted keys.  Thread i
// writes the values in (key[i-1], key[i]].
__global__ void plain_starts_kernel(const uint32_t *sorted, int64_t n, uint32_t L, uint32_t T, uint32_t *starts) {
  const int64_t total = static_cast<int64_t>(L) * n;
  const int64_t nv = static_cast<int64_t>(L) * (static_cast<int64_t>(T) + 1);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i <= total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t prev = i > 0 ? static_cast<int64_t>(sorted[i - 1]) : -1;
    const int64_t cur = i < total ? static_cast<int64_t>(sorted[i]) : nv;
    for (int64_t v = prev + 1; v <= cur && v < nv; ++v) {
      const int64_t t = v / (static_cast<int64_t>(T) + 1);
      starts[v] = static_cast<uint32_t>(i - t * n);
    }
  }
}

// Algorithm 1 over the arrivals of one bucket, one thread per bucket: slots
// 0..R-1 hold arrivals 0..R-1; arrival i >= R replaces slot j = RANDOM([0, i])
// when j < R.  Reads positions >= R, writes positions < R, in arrival order.
__global__ void plain_reservoir_kernel(int32_t *ids, const uint32_t *starts, int64_t n, uint32_t L, uint32_t T,
                                       uint32_t R, uint64_t rkey) {
  const int64_t total = static_cast<int64_t>(L) * T;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t t = static_cast<uint32_t>(g / T), b = static_cast<uint32_t>(g % T);
    const uint32_t *st = starts + static_cast<int64_t>(t) * (T + 1);
    const uint32_t s = st[b], m = st[b + 1] - s;
    if (m <= R) continue;
    int32_t *seg = ids + static_cast<int64_t>(t) * n + s;
    const uint64_t bk = reservoir_bucket_key(rkey, t, b);
    for (uint32_t i = R; i < m; ++i) {
      const uint32_t j = reservoir_draw(bk, i);
      if (j < R) seg[j] = seg[i];
    }
  }
}

// ---------------------------------------------------------------- query
// One block per query q0 + blockIdx.x: the reservoirs of its L buckets,
// table after table, into cand[blockIdx.x * LR ...]; the segment end.
__global__ void __launch_bounds__(kPlainThreads) plain_gather_kernel(PlainQueryLaunch a, int64_t q0, int64_t nq) {
  __shared__ uint32_t pre[257];
  const int64_t slot = blockIdx.x, q = q0 + slot;
  if (q >= nq) return;
  const uint32_t T = 1u << a.range_bits;
  const uint32_t t = threadIdx.x;  // blockDim >= L
  uint32_t s = 0, m = 0;
  if (t < a.L) {
    const uint32_t key = a.keys_rm[q * a.L + t];
    if (key < T) {
      const uint32_t *st = a.starts + static_cast<int64_t>(t) * (T + 1);
      s = st[key];
      m = min(st[key + 1] - s, a.R);
    }
    pre[t + 1] = m;
  }
  if (t == 0) pre[0] = 0;
  __syncthreads();
  if (t == 0)
    for (uint32_t i = 1; i <= a.L; ++i) pre[i] += pre[i - 1];
  __syncthreads();
  const int64_t base = slot * static_cast<int64_t>(a.L) * a.R;
  if (t < a.L) {
    const int32_t *src = a.ids + static_cast<int64_t>(t) * a.n + s;
    for (uint32_t j = 0; j < m; ++j) a.cand[base + pre[t] + j] = static_cast<uint32_t>(src[j]);
  }
  if (t == 0) {
    a.seg_begin[slot] = base;
    a.seg_end[slot] = base + pre[a.L];
  }
}

// COUNTFREQUENCY over a sorted segment: the head of each run of equal ids
// gets the key (256 - count) << 24 | id (ascending = count descending, then
// id ascending); every other position, and the excluded id, gets kNoKey.
__global__ void __launch_bounds__(kPlainThreads) plain_count_kernel(PlainQueryLaunch a, int64_t q0, int64_t nq) {
  const int64_t slot = blockIdx.x, q = q0 + slot;
  if (q >= nq) return;
  const int64_t b = a.seg_begin[slot], e = a.seg_end[slot];
  const int32_t excl = a.exclude_self ? static_cast<int32_t>(q) : (a.exclude ? a.exclude[q] : -1);
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const uint32_t id = a.sorted[i];
    uint32_t key = kNoKey;
    if (i == b || a.sorted[i - 1] != id) {
      int64_t j = i + 1;
      while (j < e && a.sorted[j] == id) ++j;
      if (static_cast<int32_t>(id) != excl) key = ((256u - static_cast<uint32_t>(j - i)) << 24) | id;
    }
    a.cand[i] = key;
  }
}

// The first k keys of the sorted segment, decoded; (-1, 0) past the end.
__global__ void __launch_bounds__(kPlainThreads) plain_write_kernel(PlainQueryLaunch a, int64_t q0, int64_t nq) {
  const int64_t slot = blockIdx.x, q = q0 + slot;
  if (q >= nq) return;
  const int64_t b = a.seg_begin[slot], e = a.seg_end[slot];
  for (int32_t j = threadIdx.x; j < a.k; j += blockDim.x) {
    const uint32_t key = b + j < e ? a.sorted[b + j] : kNoKey;
    a.out_ids[q * a.k + j] = key == kNoKey ? -1 : static_cast<int32_t>(key & 0xFFFFFFu);
    a.out_counts[q * a.k + j] = key == kNoKey ? 0 : static_cast<int32_t>(256u - (key >> 24));
  }
}

int ok(cudaError_t e) { return e == cudaSuccess ? 0 : FLASH_ECUDA; }

int end_bit_of(uint64_t max_value) {
  int b = 1;
  while (b < 32 && (max_value >> b) != 0) ++b;
  return b;
}

}  // namespace

int64_t plain_query_chunk(uint32_t L, uint32_t R, int64_t nq) {
  // candidates of a chunk: 2 x 4 bytes per slot of L*R, about 2 GiB in all
  int64_t c = (1LL << 31) / (8LL * L * R);
  if (c < 1) c = 1;
  return c < nq ? c : nq;
}

size_t plain_sort_temp_bytes(int64_t n, uint32_t L, uint32_t range_bits) {
  size_t bytes = 0;
  const int64_t total = static_cast<int64_t>(L) * n;
  const uint64_t nv = static_cast<uint64_t>(L) * ((1ull << range_bits) + 1);
  cub::DeviceRadixSort::SortPairs(nullptr, bytes, static_cast<const uint32_t *>(nullptr),
                                  static_cast<uint32_t *>(nullptr), static_cast<const int32_t *>(nullptr),
                                  static_cast<int32_t *>(nullptr), total, 0, end_bit_of(nv));
  return bytes;
}

size_t plain_segsort_temp_bytes(int64_t chunk, uint32_t L, uint32_t R) {
  size_t bytes = 0;
  cub::DeviceSegmentedSort::SortKeys(nullptr, bytes, static_cast<const uint32_t *>(nullptr),
                                     static_cast<uint32_t *>(nullptr), chunk * static_cast<int64_t>(L) * R, chunk,
                                     static_cast<const int64_t *>(nullptr), static_cast<const int64_t *>(nullptr));
  return bytes;
}

int launch_plain_keys(const PlainHashLaunch &a, cudaStream_t stream) {
  const size_t smem = sizeof(uint32_t) * 2 * a.B + a.B;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(plain_keys_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
          cudaSuccess)
    return FLASH_ECUDA;
  for (int64_t r0 = 0; r0 < a.n_rows; r0 += (1LL << 30)) {
    const int64_t rows = a.n_rows - r0 < (1LL << 30) ? a.n_rows - r0 : (1LL << 30);
    plain_keys_kernel<<<static_cast<unsigned>(rows), kPlainThreads, smem, stream>>>(a, r0);
    count_launches(1);
  }
  return ok(cudaGetLastError());
}

int launch_plain_group(const PlainGroupLaunch &g, cudaStream_t stream) {
  const int64_t total = static_cast<int64_t>(g.L) * g.n;
  const uint32_t T = 1u << g.range_bits;
  const uint64_t nv = static_cast<uint64_t>(g.L) * (static_cast<uint64_t>(T) + 1);
  const int blocks = 8 * num_sms();
  plain_iota_kernel<<<blocks, 256, 0, stream>>>(g.ids_in, g.n, total);
  count_launches(1);
  size_t bytes = g.temp_bytes;
  if (int rc = ok(cub::DeviceRadixSort::SortPairs(g.temp, bytes, g.comp_in, g.comp_out, g.ids_in, g.ids_out, total, 0,
                                                  end_bit_of(nv), stream)))
    return rc;
  count_launches(1);
  plain_starts_kernel<<<blocks, 256, 0, stream>>>(g.comp_out, g.n, g.L, T, g.starts);
  plain_reservoir_kernel<<<blocks, 256, 0, stream>>>(g.ids_out, g.starts, g.n, g.L, T, g.R, g.rkey);
  count_launches(2);
  return ok(cudaGetLastError());
}

int launch_plain_query(const PlainQueryLaunch &a, int64_t nq, cudaStream_t stream) {
  const int64_t chunk = plain_query_chunk(a.L, a.R, nq);
  PlainQueryLaunch b = a;
  for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
    const int64_t c = nq - q0 < chunk ? nq - q0 : chunk;
    const unsigned grid = static_cast<unsigned>(c);
    b.sorted = a.cand2;
    plain_gather_kernel<<<grid, kPlainThreads, 0, stream>>>(b, q0, nq);
    size_t bytes = a.temp_bytes;
    if (int rc = ok(cub::DeviceSegmentedSort::SortKeys(a.temp, bytes, a.cand, a.cand2, c * static_cast<int64_t>(a.L) * a.R,
                                                        c, a.seg_begin, a.seg_end, stream)))
      return rc;
    plain_count_kernel<<<grid, kPlainThreads, 0, stream>>>(b, q0, nq);
    bytes = a.temp_bytes;
    if (int rc = ok(cub::DeviceSegmentedSort::SortKeys(a.temp, bytes, a.cand, a.cand2, c * static_cast<int64_t>(a.L) * a.R,
                                                        c, a.seg_begin, a.seg_end, stream)))
      return rc;
    plain_write_kernel<<<grid, kPlainThreads, 0, stream>>>(b, q0, nq);
    count_launches(5);
  }
  return ok(cudaGetLastError());
}

}  // namespace flash
