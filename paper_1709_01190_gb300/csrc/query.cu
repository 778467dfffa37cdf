// query.cu -- K4: the Querying phase (Algorithm 3) with count-based
// k-selection (Section 3.2, Section 3.3.2).
//
// For query q with bucket addresses key_t(q):
//   gather : the reservoir of bucket key_t(q) in table t is the first
//            min(m, R) ids of its segment in the grouped table;
//   count  : each id's number of occurrences over the L reservoirs goes into
//            a shared-memory open-addressing table; an entry packs
//            (id + 1) << 8 | (count - 1) (id < 2^24 - 1, count <= L <= 256),
//            inserted with atomicCAS and incremented with atomicAdd; each new
//            entry's slot is appended to a list, so the distinct candidates
//            need no scan of the table afterwards;
//   select : the k largest sort keys (count - 1) << 24 | (2^24 - 1 - id),
//            i.e. count descending then id ascending, found by a radix select
//            over 8-bit digits (histogram, suffix sum, threshold), collected
//            and bitonic-sorted.  The excluded id is never inserted.
// This replaces the paper's segmented sort + CountReduce on the GPU
// (Section 3.4.1) by one pass through shared memory; the result is the
// unique top-k of the (count desc, id asc) order, identical to sorting.
//
// Two launch shapes share the code through a Group (warp or block):
//   query_warp_kernel : one warp per query, software-pipelined over the
//                       queries of the warp: the next query's bucket ranges
//                       are loaded while the current one is counted, and its
//                       first candidate ids while the current one is
//                       selected; queries whose candidates do not fit the
//                       warp's table are appended to an overflow list;
//   query_block_kernel: one block per overflow query, a table sized for L*R.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kQWarps = 8;  // warps per block, warp kernel
constexpr int kQBlockThreads = 256;
constexpr int kBatch = 8;   // candidate ids a thread loads before counting them

struct QArgs {
  const uint32_t *qkeys;
  int64_t q_ld, nq;
  bool q_rm;
  const int32_t *ids;
  const uint32_t *starts;
  int64_t n;
  uint32_t L, R, T;
  int32_t k;
  uint32_t kp;  // next power of two >= k
  const int32_t *exclude;
  bool exclude_self;
  int32_t *out_ids, *out_counts;
  unsigned long long *q_counter;
  unsigned long long *over_count;
  int64_t *overflow;
  uint32_t table_words;   // capacity of the group's count table (power of two)
  uint32_t region_words;  // shared words per group
};

struct WarpGroup {
  static constexpr bool kIsWarp = true;
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ int size() const { return 32; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ bool leader_warp() const { return true; }
};

struct BlockGroup {
  static constexpr bool kIsWarp = false;
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ int size() const { return blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool leader_warp() const { return threadIdx.x < 32; }
};

// Shared layout of one group:
//   [tab S][lst S/2][pre 2x(L+1)][sb 2xL][hist 256][sel kp][misc 40]
// pre/sb are double-buffered: the pipelined warp kernel builds the next
// query's bucket ranges while the current query still uses its own.
struct Region {
  uint32_t *tab, *lst, *pre[2], *sb[2], *hist, *sel, *misc;
};

__device__ __forceinline__ Region carve(uint32_t *base, const QArgs &a) {
  Region r;
  const uint32_t lp = (a.L + 1 + 3) & ~3u;
  r.tab = base;
  r.lst = r.tab + a.table_words;
  r.pre[0] = r.lst + a.table_words / 2;
  r.pre[1] = r.pre[0] + lp;
  r.sb[0] = r.pre[1] + lp;
  r.sb[1] = r.sb[0] + lp;
  r.hist = r.sb[1] + lp;
  r.sel = r.hist + 256;
  r.misc = r.sel + a.kp;
  return r;
}

uint32_t region_words(const QArgs &a) {
  const uint32_t lp = (a.L + 1 + 3) & ~3u;
  return a.table_words + a.table_words / 2 + 4 * lp + 256 + a.kp + 40;
}

__device__ __forceinline__ uint32_t sort_key(uint32_t e) {
  // e = (id + 1) << 8 | (count - 1)  ->  (count - 1) << 24 | (2^24 - 1 - id)
  return ((e & 0xFFu) << 24) | (0xFFFFFFu - ((e >> 8) - 1u));
}

__device__ __forceinline__ uint32_t ilog2_pow2(uint32_t x) { return 31u - __clz(x); }

// Bucket address of table t for query q.
__device__ __forceinline__ uint32_t query_key(const QArgs &a, int64_t q, uint32_t t) {
  return a.q_rm ? __ldcs(a.qkeys + q * a.L + t) : a.qkeys[static_cast<int64_t>(t) * a.q_ld + q];
}

// Addresses of the tables rank, rank + size, ... (TPL per thread); 2^rb past the end.
template <int TPL, class G>
__device__ __forceinline__ void load_query_keys(const G &g, const QArgs &a, int64_t q, uint32_t (&keys)[TPL]) {
#pragma unroll
  for (int i = 0; i < TPL; ++i) {
    const uint32_t t = g.rank() + i * g.size();
    keys[i] = (q >= 0 && q < a.nq && t < a.L) ? query_key(a, q, t) : a.T;
  }
}

// Bucket segment (start, end) of each of the thread's tables.
template <int TPL, class G>
__device__ __forceinline__ void load_ranges(const G &g, const QArgs &a, const uint32_t (&keys)[TPL],
                                            uint32_t (&s)[TPL], uint32_t (&e)[TPL]) {
  const uint64_t keep = l2_policy_keep();
#pragma unroll
  for (int i = 0; i < TPL; ++i) {
    const uint32_t t = g.rank() + i * g.size();
    s[i] = 0;
    e[i] = 0;
    if (t < a.L && keys[i] < a.T) {
      const uint32_t *st = a.starts + static_cast<int64_t>(t) * (static_cast<int64_t>(a.T) + 1);
      s[i] = ld_l2(st + keys[i], keep);
      e[i] = ld_l2(st + keys[i] + 1, keep);
    }
  }
}

// sb[t] = segment start, pre[t] = exclusive prefix of min(m_t, R); returns M = pre[L].
template <int TPL, class G>
__device__ uint32_t build_ranges(const G &g, const QArgs &a, uint32_t *pre, uint32_t *sb,
                                 const uint32_t (&s)[TPL], const uint32_t (&e)[TPL]) {
#pragma unroll
  for (int i = 0; i < TPL; ++i) {
    const uint32_t t = g.rank() + i * g.size();
    if (t < a.L) {
      const uint32_t m = e[i] - s[i];
      sb[t] = s[i];
      pre[t] = m < a.R ? m : a.R;
    }
  }
  g.sync();
  if (g.leader_warp()) {
    const int lane = threadIdx.x & 31;
    const uint32_t per = (a.L + 31) / 32;
    const uint32_t lo = lane * per;
    uint32_t sum = 0;
    for (uint32_t i = 0; i < per; ++i)
      if (lo + i < a.L) sum += pre[lo + i];
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += x;
    }
    uint32_t run = inc - sum;
    for (uint32_t i = 0; i < per; ++i) {
      if (lo + i < a.L) {
        const uint32_t c = pre[lo + i];
        pre[lo + i] = run;
        run += c;
      }
    }
    if (lane == 31) pre[a.L] = inc;
  }
  g.sync();
  return pre[a.L];
}

// Candidate ids base + j*size + rank (j < kBatch) of the ranges (pre, sb); -1 past M.
// A thread's candidate index only grows, so `cursor` walks the tables forward.
template <class G>
__device__ __forceinline__ void load_ids(const G &g, const QArgs &a, const uint32_t *pre, const uint32_t *sb,
                                         uint32_t M, uint32_t base, uint32_t &cursor, int32_t (&idv)[kBatch]) {
  const uint64_t keep = l2_policy_keep();
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    const uint32_t idx = base + j * g.size() + g.rank();
    idv[j] = -1;
    if (idx < M) {
      while (pre[cursor + 1] <= idx) ++cursor;
      idv[j] = ld_l2(a.ids + static_cast<int64_t>(cursor) * a.n + sb[cursor] + (idx - pre[cursor]), keep);
    }
  }
}

template <class G>
__device__ void write_empty(const G &g, const QArgs &a, int64_t q) {
  for (int j = g.rank(); j < a.k; j += g.size()) {
    __stcs(a.out_ids + q * a.k + j, -1);
    __stcs(a.out_counts + q * a.k + j, 0);
  }
}

__device__ __forceinline__ uint32_t table_size(uint32_t M) {
  uint32_t S = 64;
  while (S < 2 * M) S <<= 1;
  return S;
}

// COUNTFREQUENCY into tab (S >= 2M slots).  The first batch of ids is given
// (loaded ahead by the caller); later batches are loaded here with a cursor
// of their own.  The slot of every new entry goes to lst; misc[4] = E.
template <class G>
__device__ void count_phase(const G &g, const QArgs &a, const Region &r, const uint32_t *pre, const uint32_t *sb,
                            int64_t q, uint32_t M, const int32_t (&first)[kBatch]) {
  const uint32_t S = table_size(M);
  const uint32_t lg = ilog2_pow2(S);
  for (uint32_t i = g.rank(); i < S; i += g.size()) r.tab[i] = 0;
  if (g.rank() == 0) r.misc[4] = 0;
  g.sync();
  const int32_t excl = a.exclude_self ? static_cast<int32_t>(q) : (a.exclude ? a.exclude[q] : -1);
  uint32_t cursor = 0;
  int32_t idv[kBatch];
#pragma unroll
  for (int j = 0; j < kBatch; ++j) idv[j] = first[j];
  for (uint32_t base = 0;;) {
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const int32_t id = idv[j];
      if (id < 0 || id == excl) continue;
      const uint32_t tag = (static_cast<uint32_t>(id) + 1u) << 8;
      uint32_t h = (static_cast<uint32_t>(id) * 0x9E3779B1u) >> (32 - lg);
      for (;;) {
        uint32_t cur = r.tab[h];
        if (cur == 0) {
          cur = atomicCAS(&r.tab[h], 0u, tag);
          if (cur == 0) {
            r.lst[atomicAdd(&r.misc[4], 1u)] = h;
            break;
          }
        }
        if ((cur & ~0xFFu) == tag) {
          atomicAdd(&r.tab[h], 1u);
          break;
        }
        h = (h + 1) & (S - 1);
      }
    }
    base += kBatch * g.size();
    if (base >= M) break;
    load_ids(g, a, pre, sb, M, base, cursor, idv);
  }
  g.sync();
}

// Warp bitonic sort, descending, of 32*V keys held V per lane (lane l holds
// positions l*V .. l*V+V-1).
template <int V>
__device__ __forceinline__ void warp_bitonic_desc(uint32_t (&v)[V]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32 * V; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < V) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
          const int jp = j ^ stride;
          if (jp > j) {
            const int i = lane * V + j;
            const bool desc = (i & size) == 0;
            const uint32_t x = v[j], y = v[jp];
            if ((x < y) == desc) {
              v[j] = y;
              v[jp] = x;
            }
          }
        }
      } else {
        const int lstride = stride / V;
        const bool lower = (lane & lstride) == 0;
#pragma unroll
        for (int j = 0; j < V; ++j) {
          const uint32_t other = __shfl_xor_sync(kFull, v[j], lstride);
          const int lo_i = (lower ? lane : (lane ^ lstride)) * V + j;
          const bool desc = (lo_i & size) == 0;
          const uint32_t hi = max(v[j], other), lo = min(v[j], other);
          v[j] = (lower == desc) ? hi : lo;
        }
      }
    }
  }
}

template <int V>
__device__ __forceinline__ void warp_sort_and_write(const QArgs &a, const uint32_t *sel, uint32_t nsel, int64_t q) {
  const int lane = threadIdx.x & 31;
  uint32_t v[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const uint32_t i = lane * V + j;
    v[j] = i < nsel ? sel[i] : 0u;
  }
  warp_bitonic_desc<V>(v);
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = lane * V + j;
    if (i < a.k) {
      const uint32_t key = v[j];
      __stcs(a.out_ids + q * a.k + i, key ? static_cast<int32_t>(0xFFFFFFu - (key & 0xFFFFFFu)) : -1);
      __stcs(a.out_counts + q * a.k + i, key ? static_cast<int32_t>((key >> 24) + 1u) : 0);
    }
  }
  for (int i = 32 * V + lane; i < a.k; i += 32) {  // fewer winners than k: pad
    __stcs(a.out_ids + q * a.k + i, -1);
    __stcs(a.out_counts + q * a.k + i, 0);
  }
}

// Sort keys of the E distinct candidates (in lst), radix select of the k-th
// largest, collection and sorted output (SORTBYVALUE, then the first k).
template <class G>
__device__ void select_phase(const G &g, const QArgs &a, const Region &r, int64_t q) {
  uint32_t *misc = r.misc;  // [0]=prefix [1]=pmask [2]=need [3]=done [4]=E [5]=nsel
  const uint32_t E = misc[4];
  uint32_t *keys = r.lst;
  for (uint32_t i = g.rank(); i < E; i += g.size()) keys[i] = sort_key(r.tab[keys[i]]);
  g.sync();

  uint32_t thr = 1;  // E <= k: every key is selected
  if (E > static_cast<uint32_t>(a.k)) {
    if (g.rank() == 0) {
      misc[0] = 0;
      misc[1] = 0;
      misc[2] = static_cast<uint32_t>(a.k);
      misc[3] = 0;
    }
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      for (uint32_t i = g.rank(); i < 256; i += g.size()) r.hist[i] = 0;
      g.sync();
      const uint32_t prefix = misc[0], pmask = misc[1];
      for (uint32_t i = g.rank(); i < E; i += g.size()) {
        const uint32_t key = keys[i];
        if ((key & pmask) == prefix) atomicAdd(&r.hist[(key >> shift) & 0xFFu], 1u);
      }
      g.sync();
      if (g.leader_warp()) {
        const int lane = threadIdx.x & 31;
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += r.hist[lane * 8 + i];
        uint32_t suf = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t x = __shfl_down_sync(kFull, suf, o);
          if (lane + o < 32) suf += x;
        }
        const uint32_t need = misc[2];
        const uint32_t ball = __ballot_sync(kFull, suf >= need);
        const int ln = 31 - __clz(ball);
        if (lane == ln) {
          uint32_t cum = suf - s;
          int d = lane * 8;
          uint32_t c = 0;
          for (int i = 7; i >= 0; --i) {
            c = r.hist[lane * 8 + i];
            if (cum + c >= need) {
              d = lane * 8 + i;
              break;
            }
            cum += c;
          }
          misc[2] = need - cum;
          misc[0] = prefix | (static_cast<uint32_t>(d) << shift);
          misc[1] = pmask | (0xFFu << shift);
          if (c == need - cum) misc[3] = 1;  // the whole digit bucket is taken: lower digits do not matter
        }
      }
      g.sync();
      if (misc[3]) break;
    }
    thr = misc[0];
  }

  // ---- collect the winners (exactly min(k, E) keys are >= thr)
  if (g.rank() == 0) misc[5] = 0;
  g.sync();
  for (uint32_t i = g.rank(); i < E; i += g.size()) {
    const uint32_t key = keys[i];
    if (key >= thr) {
      const uint32_t pos = atomicAdd(&misc[5], 1u);
      if (pos < a.kp) r.sel[pos] = key;
    }
  }
  g.sync();
  const uint32_t nsel = misc[5] < a.kp ? misc[5] : a.kp;
  if constexpr (G::kIsWarp) {
    if (nsel <= 32) warp_sort_and_write<1>(a, r.sel, nsel, q);
    else if (nsel <= 64) warp_sort_and_write<2>(a, r.sel, nsel, q);
    else if (nsel <= 128) warp_sort_and_write<4>(a, r.sel, nsel, q);
    else warp_sort_and_write<8>(a, r.sel, nsel, q);
    g.sync();
  } else {
    for (uint32_t i = nsel + g.rank(); i < a.kp; i += g.size()) r.sel[i] = 0;
    g.sync();
    for (uint32_t size = 2; size <= a.kp; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = g.rank(); i < a.kp / 2; i += g.size()) {
          const uint32_t lo = (i / stride) * stride * 2 + (i % stride), hi = lo + stride;
          const bool desc = (lo & size) == 0;
          const uint32_t x = r.sel[lo], y = r.sel[hi];
          if ((x < y) == desc) {
            r.sel[lo] = y;
            r.sel[hi] = x;
          }
        }
        g.sync();
      }
    }
    for (int j = g.rank(); j < a.k; j += g.size()) {
      const uint32_t key = r.sel[j];
      __stcs(a.out_ids + q * a.k + j, key ? static_cast<int32_t>(0xFFFFFFu - (key & 0xFFFFFFu)) : -1);
      __stcs(a.out_counts + q * a.k + j, key ? static_cast<int32_t>((key >> 24) + 1u) : 0);
    }
    g.sync();
  }
}

__device__ __forceinline__ unsigned long long claim_query(const QArgs &a) {
  unsigned long long q = 0;
  if ((threadIdx.x & 31) == 0) q = atomicAdd(a.q_counter, 1ULL);
  return __shfl_sync(kFull, q, 0);
}

// TPL = tables per lane = ceil(L / 32).
template <int TPL>
__global__ void __launch_bounds__(kQWarps * 32, 3) query_warp_kernel(QArgs a) {
  extern __shared__ uint32_t smem[];
  const WarpGroup g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Region r = carve(smem + static_cast<size_t>(warp) * a.region_words, a);
  const unsigned long long nq = static_cast<unsigned long long>(a.nq);

  // prologue: query q staged (ranges in buffer 0, first ids in registers),
  // the addresses of query qn in flight
  unsigned long long q = claim_query(a);
  uint32_t keys[TPL], s[TPL], e[TPL];
  load_query_keys<TPL>(g, a, static_cast<int64_t>(q), keys);
  unsigned long long qn = claim_query(a);
  uint32_t keys_n[TPL];
  load_query_keys<TPL>(g, a, static_cast<int64_t>(qn), keys_n);
  load_ranges<TPL>(g, a, keys, s, e);
  uint32_t *pre_c = r.pre[0], *sb_c = r.sb[0], *pre_n = r.pre[1], *sb_n = r.sb[1];
  uint32_t M = build_ranges<TPL>(g, a, pre_c, sb_c, s, e);
  int32_t ids[kBatch];
  uint32_t cur0 = 0;
  load_ids(g, a, pre_c, sb_c, 2 * M <= a.table_words ? M : 0, 0, cur0, ids);

  while (q < nq) {
    // the next query's bucket ranges are in flight while this one is counted
    uint32_t sn[TPL], en[TPL];
    load_ranges<TPL>(g, a, keys_n, sn, en);
    const bool fits = 2 * M <= a.table_words;
    if (M > 0 && fits) count_phase(g, a, r, pre_c, sb_c, static_cast<int64_t>(q), M, ids);

    // stage the next query: its ranges into the other buffer, its first ids in flight
    const unsigned long long qn2 = claim_query(a);
    uint32_t keys_n2[TPL];
    load_query_keys<TPL>(g, a, static_cast<int64_t>(qn2), keys_n2);
    const uint32_t Mn = build_ranges<TPL>(g, a, pre_n, sb_n, sn, en);
    uint32_t curn = 0;
    load_ids(g, a, pre_n, sb_n, 2 * Mn <= a.table_words ? Mn : 0, 0, curn, ids);

    if (M == 0) {
      write_empty(g, a, static_cast<int64_t>(q));
    } else if (!fits) {
      if (lane == 0) a.overflow[atomicAdd(a.over_count, 1ULL)] = static_cast<int64_t>(q);
    } else {
      select_phase(g, a, r, static_cast<int64_t>(q));
    }
    __syncwarp();

    q = qn;
    qn = qn2;
    M = Mn;
    uint32_t *tp = pre_c;
    pre_c = pre_n;
    pre_n = tp;
    tp = sb_c;
    sb_c = sb_n;
    sb_n = tp;
#pragma unroll
    for (int i = 0; i < TPL; ++i) keys_n[i] = keys_n2[i];
  }
}

__global__ void __launch_bounds__(kQBlockThreads) query_block_kernel(QArgs a, int all_queries) {
  extern __shared__ uint32_t smem[];
  const BlockGroup g;
  const Region r = carve(smem, a);
  const int64_t count = all_queries ? a.nq : static_cast<int64_t>(*a.over_count);
  for (int64_t h = blockIdx.x; h < count; h += gridDim.x) {
    const int64_t q = all_queries ? h : a.overflow[h];
    uint32_t keys[1], s[1], e[1];
    load_query_keys<1>(g, a, q, keys);  // blockDim >= L: one table per thread
    load_ranges<1>(g, a, keys, s, e);
    const uint32_t M = build_ranges<1>(g, a, r.pre[0], r.sb[0], s, e);
    if (M == 0) {
      write_empty(g, a, q);
      g.sync();
    } else {
      int32_t ids[kBatch];
      uint32_t cur = 0;
      load_ids(g, a, r.pre[0], r.sb[0], M, 0, cur, ids);
      count_phase(g, a, r, r.pre[0], r.sb[0], q, M, ids);
      select_phase(g, a, r, q);
    }
  }
}

uint32_t next_pow2(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

template <int TPL>
int launch_warp(const QArgs &a, int64_t nq, cudaStream_t stream) {
  const size_t smem = static_cast<size_t>(kQWarps) * a.region_words * sizeof(uint32_t);
  if (cudaFuncSetAttribute(query_warp_kernel<TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return FLASH_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, query_warp_kernel<TPL>, kQWarps * 32, smem) !=
      cudaSuccess)
    return FLASH_ECUDA;
  if (per_sm < 1) return FLASH_EINVAL;
  int64_t blocks = static_cast<int64_t>(per_sm) * num_sms();
  const int64_t useful = (nq + kQWarps - 1) / kQWarps;
  if (blocks > useful) blocks = useful;
  query_warp_kernel<TPL><<<static_cast<unsigned>(blocks), kQWarps * 32, smem, stream>>>(a);
  count_launches(1);
  return 0;
}

}  // namespace

int launch_query(const QueryLaunch &l, cudaStream_t stream) {
  if (l.nq == 0) return 0;
  QArgs a{};
  a.qkeys = l.qkeys;
  a.q_ld = l.q_ld;
  a.nq = l.nq;
  a.q_rm = l.qkeys_rowmajor;
  a.ids = l.ids;
  a.starts = l.starts;
  a.n = l.n;
  a.L = l.L;
  a.R = l.R;
  a.T = 1u << l.range_bits;
  a.k = l.k;
  a.kp = next_pow2(static_cast<uint32_t>(l.k) < 2 ? 2 : static_cast<uint32_t>(l.k));
  a.exclude = l.exclude;
  a.exclude_self = l.exclude_self;
  a.out_ids = l.out_ids;
  a.out_counts = l.out_counts;
  a.q_counter = l.counters;
  a.over_count = l.counters + 1;
  a.overflow = l.overflow;
  if (cudaMemsetAsync(l.counters, 0, 2 * sizeof(unsigned long long), stream) != cudaSuccess) return FLASH_ECUDA;

  const uint32_t full_table = next_pow2(2 * l.L * l.R) < 64 ? 64 : next_pow2(2 * l.L * l.R);
  const bool warp_ok = l.k <= 256;
  int all = 1;
  if (warp_ok) {
    uint32_t tw = l.warp_table ? l.warp_table : 512u;
    if (tw > full_table) tw = full_table;
    a.table_words = tw;
    a.region_words = region_words(a);
    const uint32_t tpl = (l.L + 31) / 32;
    int rc;
    if (tpl <= 1) rc = launch_warp<1>(a, l.nq, stream);
    else if (tpl <= 2) rc = launch_warp<2>(a, l.nq, stream);
    else if (tpl <= 4) rc = launch_warp<4>(a, l.nq, stream);
    else rc = launch_warp<8>(a, l.nq, stream);
    if (rc) return rc;
    all = 0;
  }
  a.table_words = full_table;
  a.region_words = region_words(a);
  const size_t smem_b = static_cast<size_t>(a.region_words) * sizeof(uint32_t);
  if (cudaFuncSetAttribute(query_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem_b)) != cudaSuccess)
    return FLASH_ECUDA;
  int per_sm_b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, query_block_kernel, kQBlockThreads, smem_b) !=
      cudaSuccess)
    return FLASH_ECUDA;
  if (per_sm_b < 1) return FLASH_EINVAL;
  const int64_t blocks_b = static_cast<int64_t>(per_sm_b) * num_sms();
  query_block_kernel<<<static_cast<unsigned>(blocks_b), kQBlockThreads, smem_b, stream>>>(a, all);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
