// eval.cu -- the quality measures of Section 4.3 (R@k and S@k) by brute
// force on the GPU, against the gold standard of cosine similarity over all
// rows for a sample of query rows.
//
// Reading (the rows FLASH hashes are sets, Section 2.1): the similarity of
// two rows is the cosine of their column sets, c / sqrt(|A| |B|) with c the
// number of columns they share (rows hold distinct column ids); a row
// without entries has similarity 0 with every row.  The nearest neighbour of
// query row q is the other row of highest cosine, ties to the smaller id;
// R@k is the share of queries whose nearest neighbour is among their k
// reported ids, S@k the mean over queries of the mean cosine of the reported
// ids (-1 entries left out; 0 for a query with none).
//
// Queries go in batches of 32.  A batch marks every column of its queries in
// a word per column (bit j = query j of the batch); one pass over all rows
// (a warp per row) then counts, for each row, the columns it shares with
// each query of the batch.  The nearest neighbour is decided exactly: cos^2
// ordered as c^2 / |B| is compared by 128-bit cross multiplication.  A first
// pass keeps each query's largest c^2 / |B| as a double (atomicMax on its bits,
// which order like the values for non-negative doubles); a second pass lists
// the rows within rounding of it; a last kernel picks the exact maximum of
// that short list, ties to the smaller id.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kEvalWarps = 8;
constexpr unsigned kFullMask = 0xFFFFFFFFu;

struct EvalArgs {
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t n, dim;
  const int32_t *queries;  // [nq] row ids
  int64_t q0, nb;          // this batch: queries q0 .. q0 + nb - 1 (nb <= 32)
  uint32_t *mask;          // [dim] bit j: column of batch query j
  unsigned long long *best;  // [32] bits of the largest c^2 / |B| (double)
  uint32_t *cand;          // [32][kCand] (row, c) pairs within rounding of best
  uint32_t *ncand;         // [32]
  uint32_t *overflow;      // set when a list overflows
};

constexpr uint32_t kCand = 512;  // rows within rounding of a query's best (ties)

__device__ __forceinline__ int64_t row_len(const EvalArgs &a, int64_t r) { return a.row_ptr[r + 1] - a.row_ptr[r]; }

__global__ void mark_kernel(EvalArgs a, uint32_t value_set) {
  // one block per batch query: set (value_set = 1) or clear (0) its columns' bits
  const int64_t j = blockIdx.x;
  if (j >= a.nb) return;
  const int64_t q = a.queries[a.q0 + j];
  for (int64_t e = a.row_ptr[q] + threadIdx.x; e < a.row_ptr[q + 1]; e += blockDim.x) {
    const uint32_t c = static_cast<uint32_t>(a.col[e]);
    if (c >= static_cast<uint64_t>(a.dim)) continue;
    if (value_set)
      atomicOr(&a.mask[c], 1u << j);
    else
      a.mask[c] = 0u;
  }
}

// The counts c_j(r) of row r against the batch: lane-strided columns, the bits
// of their mask words summed per query with warp ballots (32 bits per word).
// Calls f(j, c) for every query j of the batch with c > 0 (lane j calls it).
template <class F>
__device__ __forceinline__ void row_counts(const EvalArgs &a, int64_t r, F &&f) {
  const int lane = threadIdx.x & 31;
  const int64_t s = a.row_ptr[r], e = a.row_ptr[r + 1];
  uint32_t cnt = 0;  // lane j: the count of query j
  for (int64_t base = s; base < e; base += 32) {
    const int64_t i = base + lane;
    uint32_t m = 0;
    if (i < e) {
      const uint32_t c = static_cast<uint32_t>(a.col[i]);
      if (c < static_cast<uint64_t>(a.dim)) m = __ldg(a.mask + c);
    }
    uint32_t any = __ballot_sync(kFullMask, m != 0u);
    while (any) {  // the few lanes whose column belongs to some query of the batch
      const int src = __ffs(any) - 1;
      any &= any - 1;
      const uint32_t mm = __shfl_sync(kFullMask, m, src);
      cnt += (mm >> lane) & 1u;
    }
  }
  if (cnt) f(lane, cnt);
}

__device__ __forceinline__ double key_of(uint32_t c, int64_t len) {
  return static_cast<double>(c) * static_cast<double>(c) / static_cast<double>(len);
}

__global__ void __launch_bounds__(kEvalWarps * 32) nn_pass1_kernel(EvalArgs a) {
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kEvalWarps;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * kEvalWarps + (threadIdx.x >> 5); r < a.n; r += nw) {
    row_counts(a, r, [&](int j, uint32_t c) {
      if (j < a.nb && a.queries[a.q0 + j] != r)
        atomicMax(&a.best[j], static_cast<unsigned long long>(__double_as_longlong(key_of(c, row_len(a, r)))));
    });
  }
}

__global__ void __launch_bounds__(kEvalWarps * 32) nn_pass2_kernel(EvalArgs a) {
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kEvalWarps;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * kEvalWarps + (threadIdx.x >> 5); r < a.n; r += nw) {
    row_counts(a, r, [&](int j, uint32_t c) {
      if (j >= a.nb || a.queries[a.q0 + j] == r) return;
      const double b = __longlong_as_double(static_cast<long long>(a.best[j]));
      if (key_of(c, row_len(a, r)) >= b * (1.0 - 1e-12)) {
        const uint32_t pos = atomicAdd(&a.ncand[j], 1u);
        if (pos < kCand) {
          a.cand[(j * kCand + pos) * 2] = static_cast<uint32_t>(r);
          a.cand[(j * kCand + pos) * 2 + 1] = c;
        } else {
          *a.overflow = 1u;
        }
      }
    });
  }
}

// One thread per batch query: the exact maximum of c^2 / |B| over its list
// (c1^2 |B2| against c2^2 |B1| in 128 bits), ties to the smaller row; with no
// shared column anywhere, the smallest other row (every cosine is 0).
__global__ void nn_resolve_kernel(EvalArgs a, int32_t *nn, double *nn_sim) {
  const int j = threadIdx.x;
  if (j >= a.nb) return;
  const int64_t q = a.queries[a.q0 + j];
  const uint32_t m = min(a.ncand[j], kCand);
  int64_t best_r = -1;
  uint32_t best_c = 0;
  for (uint32_t i = 0; i < m; ++i) {
    const int64_t r = a.cand[(j * kCand + i) * 2];
    const uint32_t c = a.cand[(j * kCand + i) * 2 + 1];
    if (best_r < 0) {
      best_r = r;
      best_c = c;
      continue;
    }
    const unsigned __int128 lhs = static_cast<unsigned __int128>(static_cast<uint64_t>(c) * c) *
                                  static_cast<uint64_t>(row_len(a, best_r));
    const unsigned __int128 rhs = static_cast<unsigned __int128>(static_cast<uint64_t>(best_c) * best_c) *
                                  static_cast<uint64_t>(row_len(a, r));
    if (lhs > rhs || (lhs == rhs && r < best_r)) {
      best_r = r;
      best_c = c;
    }
  }
  const int64_t lq = row_len(a, q);
  if (best_r < 0) {  // every cosine is 0: the smallest row other than q
    nn[a.q0 + j] = q == 0 ? (a.n > 1 ? 1 : -1) : 0;
    nn_sim[a.q0 + j] = 0.0;
  } else {
    nn[a.q0 + j] = static_cast<int32_t>(best_r);
    nn_sim[a.q0 + j] = lq > 0 ? best_c / sqrt(static_cast<double>(lq) * static_cast<double>(row_len(a, best_r)))
                              : 0.0;
  }
}

// S@k: one warp per (batch query, reported slot); the shared columns of the
// reported row counted through the mask; the mean in slot order per query.
__global__ void __launch_bounds__(kEvalWarps * 32) sim_kernel(EvalArgs a, const int32_t *reported, int32_t k,
                                                              double *cos_slot /* [32][k] */) {
  const int lane = threadIdx.x & 31;
  const int64_t total = a.nb * static_cast<int64_t>(k);
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kEvalWarps;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * kEvalWarps + (threadIdx.x >> 5); g < total; g += nw) {
    const int64_t j = g / k, slot = g - j * k;
    const int64_t q = a.queries[a.q0 + j];
    const int32_t r = reported[(a.q0 + j) * k + slot];
    double v = -1.0;  // no id in this slot
    if (r >= 0 && r < a.n) {
      uint32_t cnt = 0;
      const int64_t s = a.row_ptr[r], e = a.row_ptr[r + 1];
      for (int64_t i = s + lane; i < e; i += 32) {
        const uint32_t c = static_cast<uint32_t>(a.col[i]);
        if (c < static_cast<uint64_t>(a.dim)) cnt += (__ldg(a.mask + c) >> j) & 1u;
      }
      cnt = __reduce_add_sync(kFullMask, cnt);
      const int64_t lq = row_len(a, q), lr = e - s;
      v = (lq > 0 && lr > 0) ? cnt / sqrt(static_cast<double>(lq) * static_cast<double>(lr)) : 0.0;
    }
    if (lane == 0) cos_slot[j * k + slot] = v;
  }
}

__global__ void sim_mean_kernel(EvalArgs a, int32_t k, const double *cos_slot, double *sim_at_k) {
  const int j = threadIdx.x;
  if (j >= a.nb) return;
  double sum = 0.0;
  int m = 0;
  for (int i = 0; i < k; ++i) {
    const double v = cos_slot[j * k + i];
    if (v >= 0.0) {
      sum += v;
      ++m;
    }
  }
  sim_at_k[a.q0 + j] = m ? sum / m : 0.0;
}

}  // namespace

uint32_t eval_candidate_capacity() { return kCand; }

int launch_eval(const EvalLaunch &l, cudaStream_t stream) {
  EvalArgs a{};
  a.row_ptr = l.row_ptr;
  a.col = l.col;
  a.n = l.n;
  a.dim = l.dim;
  a.queries = l.queries;
  a.mask = l.mask;
  a.best = l.best;
  a.cand = l.cand;
  a.ncand = l.ncand;
  a.overflow = l.overflow;
  if (cudaMemsetAsync(l.mask, 0, sizeof(uint32_t) * static_cast<size_t>(l.dim), stream) != cudaSuccess ||
      cudaMemsetAsync(l.overflow, 0, sizeof(uint32_t), stream) != cudaSuccess)
    return FLASH_ECUDA;
  const int64_t rows_blocks = (l.n + kEvalWarps - 1) / kEvalWarps;
  const unsigned grid = static_cast<unsigned>(rows_blocks < 16LL * num_sms() ? rows_blocks : 16LL * num_sms());
  for (int64_t q0 = 0; q0 < l.nq; q0 += 32) {
    a.q0 = q0;
    a.nb = l.nq - q0 < 32 ? l.nq - q0 : 32;
    if (cudaMemsetAsync(l.best, 0, 32 * sizeof(unsigned long long), stream) != cudaSuccess ||
        cudaMemsetAsync(l.ncand, 0, 32 * sizeof(uint32_t), stream) != cudaSuccess)
      return FLASH_ECUDA;
    mark_kernel<<<static_cast<unsigned>(a.nb), 256, 0, stream>>>(a, 1u);
    nn_pass1_kernel<<<grid, kEvalWarps * 32, 0, stream>>>(a);
    nn_pass2_kernel<<<grid, kEvalWarps * 32, 0, stream>>>(a);
    nn_resolve_kernel<<<1, 32, 0, stream>>>(a, l.nn, l.nn_sim);
    const int64_t pairs_blocks = (a.nb * l.k + kEvalWarps - 1) / kEvalWarps;
    sim_kernel<<<static_cast<unsigned>(pairs_blocks), kEvalWarps * 32, 0, stream>>>(a, l.reported, l.k, l.cos_slot);
    sim_mean_kernel<<<1, 32, 0, stream>>>(a, l.k, l.cos_slot, l.sim_at_k);
    mark_kernel<<<static_cast<unsigned>(a.nb), 256, 0, stream>>>(a, 0u);
    count_launches(7);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
