// query.cu -- K4: the Querying phase (Algorithm 3) with count-based
// k-selection (Section 3.2, Section 3.3.2).
//
// For query q with bucket addresses key_t(q):
//   gather : the reservoir of bucket key_t(q) in table t is the first
//            min(m, R) ids of its segment in the grouped table;
//   count  : each id's number of occurrences over the L reservoirs goes into
//            a shared-memory open-addressing table (linear probing).
//            Warp path (a few hundred candidates): an entry packs
//            (id + 1) << 8 | (count - 1) (id < 2^24 - 1, count <= L <= 256),
//            inserted with atomicCAS and incremented with atomicAdd; each new
//            entry's slot is appended to a list.  Block path (thousands of
//            candidates, nearly all distinct): tags id + 1 in one array,
//            16-bit counts in a parallel one (added with red).  A query whose
//            warps' candidate streams take one or two batches places its tags
//            by atomicCAS; with more batches returning shared atomics cost
//            more than barrier-separated rounds: a read step probes to the
//            id's slot or to the first empty one, a write step stores the tag
//            into that empty slot (blind; the last writer wins) and the next
//            read step finds whether this id won (on the empty table of the
//            first batch every id goes straight to its home slot); the few
//            ids still unplaced after the last round use atomicCAS;
//   select : the k largest sort keys (count - 1) << 24 | (2^24 - 1 - id),
//            i.e. count descending then id ascending, found by a radix select
//            over 8-bit digits (histogram, suffix sum, threshold) and
//            collected; the warp path bitonic-sorts them, the block path
//            writes each at its rank (the number of larger keys).  The
//            excluded id is never inserted.
// This replaces the paper's segmented sort + CountReduce on the GPU
// (Section 3.4.1) by one pass through shared memory; the result is the
// unique top-k of the (count desc, id asc) order, identical to sorting.
//
// Two launch shapes share the code through a Group (warp or block):
//   query_warp_kernel: one warp per query, software-pipelined over the
//                      queries of the warp: the next query's bucket ranges
//                      are loaded while the current one is counted, and its
//                      first candidate ids while the current one is
//                      selected; queries whose candidates do not fit the
//                      warp's table are appended to an overflow list;
//   query_big_kernel : one block per overflow query (all queries when k is
//                      too large for the warp path), in two tiers: a 64 KB
//                      table first (several blocks per SM), then a table
//                      sized for L*R for the few queries that do not fit it.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kQWarps = 8;  // warps per block, warp kernel
constexpr int kBigThreads = 512;
constexpr int kBigWarps = kBigThreads / 32;
constexpr int kMaxTabPerWarp = 256 / kBigWarps;  // L <= 256
constexpr uint32_t kListCap = 2048;  // keys a block-path selection may gather before its last passes
constexpr uint32_t kBigTable = 16384;  // slots of the first big tier's table (64 KB)
constexpr int kBatch = 8;   // candidate ids a thread loads before counting them

struct QArgs {
  const uint32_t *qkeys;
  int64_t q_ld, nq;
  bool q_rm;
  const int32_t *ids;
  const uint32_t *starts;
  int64_t n;
  int64_t st_stride, id_stride;  // table t's starts at t * st_stride, its ids at t * id_stride (0: one shared pool)
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
//   [tab S][aux S/2][pre 2x(L+1)][sb 2xL][hist 256][sel kp][misc 40]
// aux is the list of new entries' slots (warp path) or the 16-bit counts
// (block path).
// pre/sb are double-buffered: the pipelined warp kernel builds the next
// query's bucket ranges while the current query still uses its own.
struct Region {
  uint32_t *tab, *aux, *pre[2], *sb[2], *hist, *sel, *misc;
  // block path only: per-table reservoir sizes and segment starts, each
  // warp's candidate stream (table starts in the stream, element offsets),
  // the list of keys gathered by the selection, and the bitmap of slots whose
  // id arrived more than once (one bit per table slot)
  uint32_t *mt, *sbk, *wpre, *lst, *dup;
  long long *off;
};

// Each pre buffer is followed by its cell index (pre_words covers both).
__host__ __device__ __forceinline__ uint32_t pre_prefix_words(uint32_t L) { return (L + 1 + 3) & ~3u; }
__host__ __device__ __forceinline__ uint32_t cell_words(uint32_t table_words) { return ((table_words / 8) + 3) & ~3u; }

__device__ __forceinline__ Region carve(uint32_t *base, const QArgs &a) {
  Region r;
  const uint32_t lp = pre_prefix_words(a.L);
  const uint32_t pw = lp + cell_words(a.table_words);
  r.tab = base;
  r.aux = r.tab + a.table_words;
  r.pre[0] = r.aux + a.table_words / 2;
  r.pre[1] = r.pre[0] + pw;
  r.sb[0] = r.pre[1] + pw;
  r.sb[1] = r.sb[0] + lp;
  r.hist = r.sb[1] + lp;
  r.sel = r.hist + 256;
  r.misc = r.sel + a.kp;
  return r;
}

// Block path: [tab S][aux S/2][mt 256][sbk 256][wpre 16x17 (+pad)][off 16x16 x2][lst 2048][dup S/32]
//             [hist 256][sel kp][misc 40]
constexpr uint32_t kWpreWords = (kBigWarps * (kMaxTabPerWarp + 1) + 3) & ~3u;

__device__ __forceinline__ Region carve_big(uint32_t *base, const QArgs &a) {
  Region r{};
  r.tab = base;
  r.aux = r.tab + a.table_words;
  r.mt = r.aux + a.table_words / 2;
  r.sbk = r.mt + 256;
  r.wpre = r.sbk + 256;
  r.off = reinterpret_cast<long long *>(r.wpre + kWpreWords);
  r.lst = reinterpret_cast<uint32_t *>(r.off + kBigWarps * kMaxTabPerWarp);
  r.dup = r.lst + kListCap;
  r.hist = r.dup + (a.table_words + 31) / 32;
  r.sel = r.hist + 256;
  r.misc = r.sel + a.kp;
  return r;
}

uint32_t big_region_words(const QArgs &a) {
  const uint32_t w = a.table_words + a.table_words / 2 + 512 + kWpreWords + 2 * kBigWarps * kMaxTabPerWarp + kListCap +
                     (a.table_words + 31) / 32 + 256 + a.kp + 40;
  return (w + 3) & ~3u;
}

uint32_t region_words(const QArgs &a) {
  const uint32_t lp = pre_prefix_words(a.L);
  const uint32_t w = a.table_words + a.table_words / 2 + 4 * lp + 2 * cell_words(a.table_words) + 256 + a.kp + 40;
  return (w + 3) & ~3u;  // every group's table starts on 16 bytes (uint4 reads)
}

// Tag id + 1 and count c >= 1  ->  (c - 1) << 24 | (2^24 - 1 - id).
__device__ __forceinline__ uint32_t sort_key(uint32_t tag, uint32_t c) {
  return ((c - 1u) << 24) | (0xFFFFFFu - (tag - 1u));
}

// Packed entry (id + 1) << 8 | (count - 1)  ->  the same sort key.
__device__ __forceinline__ uint32_t sort_key_packed(uint32_t e) {
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
      const uint32_t *st = a.starts + static_cast<int64_t>(t) * a.st_stride;
      s[i] = ld_l2(st + keys[i], keep);
      e[i] = ld_l2(st + keys[i] + 1, keep);
    }
  }
}

// sb[t] = segment start, pre[t] = exclusive prefix of min(m_t, R); returns M = pre[L].
// The cell index after pre: cell[c] = the table holding candidate 4c (for the
// candidates a warp table can take), so a candidate finds its table in a step
// or two instead of walking the prefix.
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
  uint32_t *cell = pre + pre_prefix_words(a.L);
  const uint32_t ncell = cell_words(a.table_words);
#pragma unroll
  for (int i = 0; i < TPL; ++i) {
    const uint32_t t = g.rank() + i * g.size();
    if (t < a.L) {
      const uint32_t c1 = min((pre[t + 1] + 3) >> 2, ncell);
      for (uint32_t c = (pre[t] + 3) >> 2; c < c1; ++c) cell[c] = t;
    }
  }
  g.sync();
  return pre[a.L];
}

// Candidate ids base + j*size + rank (j < kBatch) of the ranges (pre, sb); -1 past M.
// The table of candidate idx comes from the cell index after pre.
template <class G>
__device__ __forceinline__ void load_ids(const G &g, const QArgs &a, const uint32_t *pre, const uint32_t *sb,
                                         uint32_t M, uint32_t base, int32_t (&idv)[kBatch]) {
  const uint64_t keep = l2_policy_keep();
  const uint32_t *cell = pre + pre_prefix_words(a.L);
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    const uint32_t idx = base + j * g.size() + g.rank();
    idv[j] = -1;
    if (idx < M) {
      uint32_t t = cell[idx >> 2];
      while (pre[t + 1] <= idx) ++t;
      idv[j] = ld_l2(a.ids + static_cast<int64_t>(t) * a.id_stride + sb[t] + (idx - pre[t]), keep);
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

// Count table of a query with M candidates, warp path: a power of two >= 2 M
// (load <= 1/2).
__device__ __forceinline__ uint32_t table_size(uint32_t M) {
  uint32_t S = 64;
  while (S < 2 * M) S <<= 1;
  return S;
}

// Count table of the block path: a power of two > 1.5 M (load < 2/3).
__host__ __device__ __forceinline__ uint32_t big_table_size(uint32_t M) {
  uint32_t S = 64;
  while (S < M + M / 2 + 1) S <<= 1;
  return S;
}

__device__ __forceinline__ uint32_t slot_hash(int32_t id, uint32_t lg) {
  return (static_cast<uint32_t>(id) * 0x9E3779B1u) >> (32 - lg);
}

// COUNTFREQUENCY of the warp path into packed entries (S >= 2M slots).  The
// first batch of ids is given (loaded ahead by the caller); later batches are
// loaded here.  The slot of every new entry goes to the list aux (positions
// from a ballot per batch slot, not from a shared counter); misc[4] = E.
__device__ void count_phase_warp(const WarpGroup &g, const QArgs &a, const Region &r, const uint32_t *pre,
                                 const uint32_t *sb, int64_t q, uint32_t M, const int32_t (&first)[kBatch]) {
  const uint32_t S = table_size(M);
  const uint32_t lg = ilog2_pow2(S);
  const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
  for (uint32_t i = g.rank(); i < S; i += g.size()) r.tab[i] = 0;
  g.sync();
  const int32_t excl = a.exclude_self ? static_cast<int32_t>(q) : (a.exclude ? a.exclude[q] : -1);
  uint32_t E = 0;
  int32_t idv[kBatch];
#pragma unroll
  for (int j = 0; j < kBatch; ++j) idv[j] = first[j];
  for (uint32_t base = 0;;) {
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const int32_t id = idv[j];
      bool fresh = false;
      uint32_t h = 0;
      if (id >= 0 && id != excl) {
        const uint32_t tag = (static_cast<uint32_t>(id) + 1u) << 8;
        h = slot_hash(id, lg);
        for (;;) {
          uint32_t cur = r.tab[h];
          if (cur == 0) {
            cur = atomicCAS(&r.tab[h], 0u, tag);
            if (cur == 0) {
              fresh = true;
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
      const uint32_t ball = __ballot_sync(kFull, fresh);
      if (fresh) r.aux[E + __popc(ball & lt)] = h;
      E += __popc(ball);
    }
    base += kBatch * g.size();
    if (base >= M) break;
    load_ids(g, a, pre, sb, M, base, idv);
  }
  if (g.rank() == 0) r.misc[4] = E;
  g.sync();
}

// Sort keys of the distinct candidates listed in aux (warp path); returns E.
__device__ __forceinline__ uint32_t keys_from_list(const WarpGroup &g, const Region &r) {
  const uint32_t E = r.misc[4];
  for (uint32_t i = g.rank(); i < E; i += g.size()) r.aux[i] = sort_key_packed(r.tab[r.aux[i]]);
  g.sync();
  return E;
}

// Block path: the L bucket ranges of query q, split into one candidate stream
// per warp (warp w takes tables w, w + 16, ...).  wpre[w][i] is the start of
// the warp's i-th table in its stream (wpre[w][ntab] = the stream's length) and
// off[w][i] the element offset such that stream position x of that table is
// ids[off + x].  Returns M, the number of candidates; misc[9] = the longest
// stream.
// The head of query q on the block path, thread t < L taking table t: its
// bucket address, then the bucket's segment [s, e).  Split in two so that the
// kernel can have the next queries' loads in flight while it counts one.
__device__ __forceinline__ uint32_t head_key(const QArgs &a, int64_t q) {
  const uint32_t t = threadIdx.x;
  return (q >= 0 && q < a.nq && t < a.L) ? query_key(a, q, t) : a.T;
}
__device__ __forceinline__ void head_range(const QArgs &a, uint32_t key, uint32_t &s, uint32_t &e) {
  const uint32_t t = threadIdx.x;
  s = 0;
  e = 0;
  if (t < a.L && key < a.T) {
    const uint64_t keep = l2_policy_keep();
    const uint32_t *st = a.starts + static_cast<int64_t>(t) * a.st_stride;
    s = ld_l2(st + key, keep);
    e = ld_l2(st + key + 1, keep);
  }
}

__device__ uint32_t build_streams(const BlockGroup &g, const QArgs &a, const Region &r, uint32_t s, uint32_t e) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    r.misc[8] = 0;
    r.misc[9] = 0;
  }
  const uint32_t t = threadIdx.x;  // blockDim >= L: one table per thread
  if (t < a.L) {
    const uint32_t m = e - s;
    r.mt[t] = m < a.R ? m : a.R;
    r.sbk[t] = s;
  }
  g.sync();
  const uint32_t w = static_cast<uint32_t>(warp);
  const uint32_t ntab = a.L > w ? (a.L - w + kBigWarps - 1) / kBigWarps : 0;
  const uint32_t tt = w + kBigWarps * static_cast<uint32_t>(lane);
  const uint32_t v = static_cast<uint32_t>(lane) < ntab ? r.mt[tt] : 0u;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += x;
  }
  const uint32_t total = __shfl_sync(kFull, inc, 31);
  uint32_t *wp = r.wpre + warp * (kMaxTabPerWarp + 1);
  long long *of = r.off + warp * kMaxTabPerWarp;
  if (static_cast<uint32_t>(lane) < ntab) {
    wp[lane] = inc - v;
    of[lane] = static_cast<long long>(tt) * a.id_stride + r.sbk[tt] - (inc - v);
  }
  if (lane == 0) {
    wp[ntab] = total;
    if (total) {
      atomicAdd(&r.misc[8], total);
      atomicMax(&r.misc[9], total);
    }
  }
  g.sync();
  return r.misc[8];
}

// Candidate ids at stream positions base + 32 j + lane (j < kBatch) of this
// warp's stream (tables starts wp, offsets of, length len); -1 past its end.
// A lane's position only grows, so `cur` walks the warp's tables forward.
__device__ __forceinline__ void load_stream_ids(const QArgs &a, const uint32_t *wp, const long long *of, uint32_t len,
                                                uint32_t base, uint32_t &cur, int32_t (&idv)[kBatch]) {
  const uint64_t keep = l2_policy_keep();
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    const uint32_t x = base + 32 * j + lane;
    idv[j] = -1;
    if (x < len) {
      while (wp[cur + 1] <= x) ++cur;
      idv[j] = ld_l2(a.ids + of[cur] + x, keep);
    }
  }
}

// 16-bit counts, two per word: a non-returning add (counts <= L <= 256).
__device__ __forceinline__ void count_add(uint32_t *cnt, uint32_t h) {
  atomicAdd(&cnt[h >> 1], 1u << ((h & 1u) << 4));
}

// COUNTFREQUENCY of one batch of ids (idv[j] < 0: none; the excluded id is
// skipped), block path; every thread of the block calls it.  Rounds of
//   read  : probe from h to this id's tag (placed: count it) or to the first
//           empty slot (to be written); only reads happen in this step;
//   write : store the tag into that slot; only writes happen in this step;
// separated by barriers, so every read sees a stable table and a lost write
// race shows up in the next read step.  Ids still unplaced after kRounds
// rounds are inserted with atomicCAS once the block's writes are done.
__device__ __forceinline__ void count_batch(const BlockGroup &g, const Region &r, uint32_t S, uint32_t lg,
                                            const int32_t (&idv)[kBatch], int32_t excl, bool fresh) {
  constexpr int kRounds = 3;
  uint32_t h[kBatch];
  uint32_t pend = 0;
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    h[j] = 0;
    if (idv[j] >= 0 && idv[j] != excl) {
      pend |= 1u << j;
      h[j] = slot_hash(idv[j], lg);
    }
  }
  g.sync();  // the previous batch's writes are visible
  bool done = false;
  for (int round = 0; round < kRounds; ++round) {
    uint32_t want = 0;
    if (round == 0 && fresh) {
      // the table is empty: the read step would find every home slot empty
      want = pend;
      if (!__syncthreads_or(want != 0)) {
        done = true;
        break;
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j)
        if ((want >> j) & 1u) r.tab[h[j]] = static_cast<uint32_t>(idv[j]) + 1u;
      g.sync();
      continue;
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if ((pend >> j) & 1u) {
        const uint32_t tag = static_cast<uint32_t>(idv[j]) + 1u;
        for (;;) {
          const uint32_t w = r.tab[h[j]];
          if (w == tag) {
            count_add(r.aux, h[j]);
            pend &= ~(1u << j);
            break;
          }
          if (w == 0) {
            want |= 1u << j;
            break;
          }
          h[j] = (h[j] + 1) & (S - 1);
        }
      }
    }
    if (!__syncthreads_or(want != 0)) {
      done = true;
      break;
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      if ((want >> j) & 1u) r.tab[h[j]] = static_cast<uint32_t>(idv[j]) + 1u;
    g.sync();
  }
  if (done) return;
  // the last round's writes are visible: settle them, then CAS the rest
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    if ((pend >> j) & 1u) {
      const uint32_t tag = static_cast<uint32_t>(idv[j]) + 1u;
      for (;;) {
        uint32_t w = r.tab[h[j]];
        if (w == 0) w = atomicCAS(&r.tab[h[j]], 0u, tag);
        if (w == 0 || w == tag) {
          count_add(r.aux, h[j]);
          break;
        }
        h[j] = (h[j] + 1) & (S - 1);
      }
    }
  }
}

// COUNTFREQUENCY of one batch by atomicCAS inserts (linear probing, no
// rounds): for a query of one or two batches (up to 512 ids in a warp's
// stream) this beats the barrier-separated rounds, whose three read/write
// passes per batch cost more than the returning atomics; with more batches
// the rounds win (measured on kdd12-like and url-like queries).
// An insert that finds its id already present marks the slot in r.dup; `fresh`
// counts this thread's new entries.
__device__ __forceinline__ void count_batch_cas(const Region &r, uint32_t S, uint32_t lg,
                                                const int32_t (&idv)[kBatch], int32_t excl, uint32_t &fresh) {
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    if (idv[j] >= 0 && idv[j] != excl) {
      const uint32_t tag = static_cast<uint32_t>(idv[j]) + 1u;
      uint32_t h = slot_hash(idv[j], lg);
      for (;;) {
        uint32_t w = r.tab[h];
        if (w == 0) w = atomicCAS(&r.tab[h], 0u, tag);
        if (w == 0 || w == tag) {
          count_add(r.aux, h);
          if (w == 0)
            ++fresh;
          else
            atomicOr(&r.dup[h >> 5], 1u << (h & 31u));
          break;
        }
        h = (h + 1) & (S - 1);
      }
    }
  }
}

// COUNTFREQUENCY of the block path into a table of S slots (tags in tab,
// counts in aux), over nbatch batches of each warp's stream.  The first batch
// of ids is given (loaded ahead by the caller); later batches are loaded here.
__device__ void count_phase_block(const BlockGroup &g, const QArgs &a, const Region &r, int64_t q, uint32_t nbatch,
                                  const int32_t (&first)[kBatch], uint32_t &cur, uint32_t S) {
  const uint32_t lg = ilog2_pow2(S);
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (uint32_t i = 4 * g.rank(); i < S; i += 4 * g.size()) *reinterpret_cast<uint4 *>(r.tab + i) = z;
  for (uint32_t i = 4 * g.rank(); i < S / 2; i += 4 * g.size()) *reinterpret_cast<uint4 *>(r.aux + i) = z;
  // the selection's histogram and counters start here, so that it needs no
  // barrier of its own before its first pass
  for (uint32_t i = g.rank(); i < 256; i += g.size()) r.hist[i] = 0;
  if (g.rank() == 0) {
    r.misc[0] = 0;  // prefix
    r.misc[1] = 0;  // prefix mask
    r.misc[2] = static_cast<uint32_t>(a.k);  // keys still needed
    r.misc[3] = 0;  // stop
    r.misc[5] = 0;  // keys gathered into the list
    r.misc[7] = 0;  // keys above the prefix range
    r.misc[10] = 0;  // new entries (CAS count)
    r.misc[11] = 0;  // winners gathered
  }
  const int32_t excl = a.exclude_self ? static_cast<int32_t>(q) : (a.exclude ? a.exclude[q] : -1);
  const int warp = threadIdx.x >> 5;
  const uint32_t *wp = r.wpre + warp * (kMaxTabPerWarp + 1);
  const long long *of = r.off + warp * kMaxTabPerWarp;
  const uint32_t ntab = a.L > static_cast<uint32_t>(warp) ? (a.L - warp + kBigWarps - 1) / kBigWarps : 0;
  const uint32_t len = wp[ntab];
  int32_t idv[kBatch];
#pragma unroll
  for (int j = 0; j < kBatch; ++j) idv[j] = first[j];
  if (nbatch <= 2) {
    for (uint32_t i = g.rank(); i < S / 32; i += g.size()) r.dup[i] = 0;
    g.sync();  // the cleared table is visible
    uint32_t fresh = 0;
    for (uint32_t b = 0;;) {
      count_batch_cas(r, S, lg, idv, excl, fresh);
      if (++b >= nbatch) break;
      load_stream_ids(a, wp, of, len, b * 32 * kBatch, cur, idv);
    }
    fresh = __reduce_add_sync(kFull, fresh);
    if ((threadIdx.x & 31) == 0 && fresh) atomicAdd(&r.misc[10], fresh);
  } else {
    for (uint32_t b = 0;;) {
      count_batch(g, r, S, lg, idv, excl, b == 0);
      if (++b >= nbatch) break;
      load_stream_ids(a, wp, of, len, b * 32 * kBatch, cur, idv);
    }
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

// nsel <= 256 winners sorted by one warp.
__device__ __forceinline__ void warp_sort_winners(const QArgs &a, const uint32_t *sel, uint32_t nsel, int64_t q) {
  if (nsel <= 32) warp_sort_and_write<1>(a, sel, nsel, q);
  else if (nsel <= 64) warp_sort_and_write<2>(a, sel, nsel, q);
  else if (nsel <= 128) warp_sort_and_write<4>(a, sel, nsel, q);
  else warp_sort_and_write<8>(a, sel, nsel, q);
}

// nsel <= 256 distinct winners written in descending order by the block:
// winner i goes to position rank(i) = the number of winners larger than it,
// counted by P threads (the largest power of two <= 32 with P * nsel <= the
// block size) and summed over them with shuffles.  Positions nsel .. k - 1 are
// padded.
__device__ __forceinline__ void block_rank_write(const QArgs &a, const uint32_t *sel, uint32_t nsel, int64_t q) {
  uint32_t lp = 5;  // log2 P
  while (lp > 0 && (nsel << lp) > kBigThreads) --lp;
  const uint32_t t = threadIdx.x, P = 1u << lp;
  const uint32_t i = t >> lp, part = t & (P - 1);
  uint32_t key = 0, above = 0;
  if (i < nsel) {
    key = sel[i];
    for (uint32_t j = part; j < nsel; j += P) above += sel[j] > key ? 1u : 0u;
  }
  for (uint32_t o = 1; o < P; o <<= 1) above += __shfl_xor_sync(kFull, above, o);
  if (i < nsel && part == 0 && above < static_cast<uint32_t>(a.k)) {
    __stcs(a.out_ids + q * a.k + above, static_cast<int32_t>(0xFFFFFFu - (key & 0xFFFFFFu)));
    __stcs(a.out_counts + q * a.k + above, static_cast<int32_t>((key >> 24) + 1u));
  }
  for (uint32_t j = nsel + t; j < static_cast<uint32_t>(a.k); j += kBigThreads) {
    __stcs(a.out_ids + q * a.k + j, -1);
    __stcs(a.out_counts + q * a.k + j, 0);
  }
}

// nsel winners sorted by the block (bitonic network over kp slots in shared memory).
__device__ void block_sort_winners(const QArgs &a, uint32_t *sel, uint32_t nsel, int64_t q) {
  for (uint32_t i = nsel + threadIdx.x; i < a.kp; i += blockDim.x) sel[i] = 0;
  __syncthreads();
  for (uint32_t size = 2; size <= a.kp; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < a.kp / 2; i += blockDim.x) {
        const uint32_t lo = (i / stride) * stride * 2 + (i % stride), hi = lo + stride;
        const bool desc = (lo & size) == 0;
        const uint32_t x = sel[lo], y = sel[hi];
        if ((x < y) == desc) {
          sel[lo] = y;
          sel[hi] = x;
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < a.k; j += blockDim.x) {
    const uint32_t key = sel[j];
    __stcs(a.out_ids + q * a.k + j, key ? static_cast<int32_t>(0xFFFFFFu - (key & 0xFFFFFFu)) : -1);
    __stcs(a.out_counts + q * a.k + j, key ? static_cast<int32_t>((key >> 24) + 1u) : 0);
  }
}

// Radix select of the k-th largest of keys[0..E) (SORTBYVALUE, then the first
// k), collection and sorted output.  The digits are very skewed (most counts
// are 1), so the lanes holding lane 0's digit add to its bin once; the others
// add one by one.
template <class G>
__device__ void select_phase(const G &g, const QArgs &a, const Region &r, int64_t q, const uint32_t *keys,
                             uint32_t E) {
  uint32_t *misc = r.misc;  // [0]=prefix [1]=pmask [2]=need [3]=done [5]=nsel
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  if constexpr (G::kIsWarp) {
    if (E <= static_cast<uint32_t>(a.k)) {  // every key wins: sort them where they are
      warp_sort_winners(a, keys, E, q);
      g.sync();
      return;
    }
  }
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
      for (uint32_t base = 0; base < E; base += g.size()) {
        const uint32_t i = base + g.rank();
        const uint32_t key = i < E ? keys[i] : 0u;
        const uint32_t d = (i < E && (key & pmask) == prefix) ? ((key >> shift) & 0xFFu) : 0x100u;
        // lanes sharing lane 0's digit (usually most of them) add once
        const uint32_t d0 = __shfl_sync(kFull, d, 0);
        const uint32_t same = __ballot_sync(kFull, d == d0);
        if (lane == 0) {
          if (d0 != 0x100u) atomicAdd(&r.hist[d0], __popc(same));
        } else if (d != d0 && d != 0x100u) {
          atomicAdd(&r.hist[d], 1u);
        }
      }
      g.sync();
      if (g.leader_warp()) {
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
  uint32_t nsel;
  if constexpr (G::kIsWarp) {
    uint32_t n = 0;
    for (uint32_t base = 0; base < E; base += 32) {
      const uint32_t i = base + lane;
      const uint32_t key = i < E ? keys[i] : 0u;
      const bool win = i < E && key >= thr;
      const uint32_t ball = __ballot_sync(kFull, win);
      const uint32_t pos = n + __popc(ball & lt);
      if (win && pos < a.kp) r.sel[pos] = key;
      n += __popc(ball);
    }
    g.sync();
    nsel = n < a.kp ? n : a.kp;
  } else {
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
    nsel = misc[5] < a.kp ? misc[5] : a.kp;
  }
  if constexpr (G::kIsWarp) {
    warp_sort_winners(a, r.sel, nsel, q);
  } else if (a.kp <= 256) {  // one warp sorts the winners in registers
    if (threadIdx.x < 32) warp_sort_winners(a, r.sel, nsel, q);
  } else {
    block_sort_winners(a, r.sel, nsel, q);
  }
  g.sync();
}

// Ordered in-place compaction of the non-empty entries of tab[0..S) (tags;
// counts in cnt) into their sort keys tab[0..E), four slots per thread and
// round (block path).  Writes never pass the read frontier: an entry's rank
// among the non-empty entries is at most its index, and a round's reads all
// finish before its writes.  `scratch` holds a word per warp.
__device__ uint32_t compact_keys(const BlockGroup &g, uint32_t *tab, const uint32_t *cnt, uint32_t S,
                                 uint32_t *scratch) {
  const int lane = threadIdx.x & 31;
  uint32_t out = 0;
  for (uint32_t base = 0; base < S; base += 4 * g.size()) {
    const uint32_t i = base + 4 * g.rank();
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    uint2 c2 = make_uint2(0u, 0u);
    if (i < S) {
      e = *reinterpret_cast<const uint4 *>(tab + i);
      c2 = *reinterpret_cast<const uint2 *>(cnt + i / 2);
    }
    const uint32_t c = (e.x != 0) + (e.y != 0) + (e.z != 0) + (e.w != 0);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += x;
    }
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 31) scratch[warp] = inc;
    g.sync();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < nwarps; ++w) {
      const uint32_t cw = scratch[w];
      if (w < warp) before += cw;
      total += cw;
    }
    g.sync();
    uint32_t pos = out + before + inc - c;
    if (e.x) tab[pos++] = sort_key(e.x, c2.x & 0xFFFFu);
    if (e.y) tab[pos++] = sort_key(e.y, c2.x >> 16);
    if (e.z) tab[pos++] = sort_key(e.z, c2.y & 0xFFFFu);
    if (e.w) tab[pos] = sort_key(e.w, c2.y >> 16);
    out += total;
  }
  g.sync();
  return out;
}

// Appends key to buf at (*ctr)++ where pred holds, storing only below cap
// (*ctr still counts every key); one shared atomic per warp.  Every lane of
// the warp calls it.
__device__ __forceinline__ void append_warp(uint32_t *buf, uint32_t cap, uint32_t *ctr, bool pred, uint32_t key) {
  const uint32_t ball = __ballot_sync(kFull, pred);
  if (ball == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(ball) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(ctr, static_cast<uint32_t>(__popc(ball)));
  base = __shfl_sync(kFull, base, leader);
  const uint32_t pos = base + __popc(ball & ((1u << lane) - 1u));
  if (pred && pos < cap) buf[pos] = key;
}

// Visits the sort keys of the block-path table (tags in tab, counts in aux):
// f(u, valid, key) for the four slots of each thread and round; every thread
// makes the same number of calls (invalid slots included), so f may use warp
// collectives.
template <class F>
__device__ __forceinline__ void for_table_keys(const Region &r, uint32_t S, F &&f) {
  for (uint32_t base = 0; base < S; base += 4 * kBigThreads) {
    const uint32_t i = base + 4 * threadIdx.x;
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    uint2 c2 = make_uint2(0u, 0u);
    if (i < S) {
      e = *reinterpret_cast<const uint4 *>(r.tab + i);
      c2 = *reinterpret_cast<const uint2 *>(r.aux + i / 2);
    }
    f(0, e.x != 0, e.x ? sort_key(e.x, c2.x & 0xFFFFu) : 0u);
    f(1, e.y != 0, e.y ? sort_key(e.y, c2.x >> 16) : 0u);
    f(2, e.z != 0, e.z ? sort_key(e.z, c2.y & 0xFFFFu) : 0u);
    f(3, e.w != 0, e.w ? sort_key(e.w, c2.y >> 16) : 0u);
  }
}

// Block-path selection, k <= 256: a radix select over the sort keys
// (count - 1) << 24 | (2^24 - 1 - id), 8-bit digits from the top, that stops
// at the first digit where at most 256 keys reach the threshold; those keys
// are collected and the block writes the k best, each at its rank.  Exactly
// one key remains in the threshold digit after the last pass (keys are
// distinct), so it always stops by then.
// The first pass (the count digit) builds the count histogram and gathers the
// keys of entries with count >= 2 into a list (up to kListCap): with dup_known
// (the CAS count marked the slots of ids that arrived again) it reads only the
// marked slots; otherwise it reads the table, tallying the count-1 entries,
// nearly all of them, per thread.  Later
// passes read that list when the threshold count is >= 2 and the list is
// complete; otherwise they read the table, and the keys reaching the
// threshold are gathered into the list once there are at most kListCap.
__device__ void select_from_table(const BlockGroup &g, const QArgs &a, const Region &r, int64_t q, uint32_t S,
                                  bool dup_known) {
  // misc: [0] prefix [1] pmask [2] need [3] stop [4] threshold [5] gathered [6] keys >= threshold
  //       [7] keys above the prefix range [10] new entries (CAS count) [11] winners gathered;
  // [0] .. [3], [5], [7], [10], [11] and hist were set by count_phase_block before its last barrier
  uint32_t *misc = r.misc;
  const int lane = threadIdx.x & 31;
  bool listed = false;
  uint32_t nlist = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    if (pass > 0) {
      for (uint32_t i = g.rank(); i < 256; i += g.size()) r.hist[i] = 0;
      g.sync();
    }
    const uint32_t prefix = misc[0], pmask = misc[1];
    if (pass == 0 && dup_known) {
      // the count >= 2 entries are the slots marked in r.dup: their keys go to
      // the list (one position per warp and round) and their counts to hist;
      // the count-1 entries are the others, misc[10] - (marked slots)
      const uint32_t nw = S / 32;
      for (uint32_t w0 = 0; w0 < nw; w0 += kBigThreads) {
        const uint32_t w = w0 + threadIdx.x;
        uint32_t m = w < nw ? r.dup[w] : 0u;
        const uint32_t nb = __popc(m);
        uint32_t inc = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t x = __shfl_up_sync(kFull, inc, o);
          if (lane >= o) inc += x;
        }
        uint32_t pos = 0;
        if (lane == 31 && inc) pos = atomicAdd(&misc[5], inc);
        pos = __shfl_sync(kFull, pos, 31) + inc - nb;
        uint32_t twos = 0;
        for (; m; m &= m - 1u) {
          const uint32_t slot = 32u * w + static_cast<uint32_t>(__ffs(m) - 1);
          const uint32_t c = (r.aux[slot >> 1] >> ((slot & 1u) << 4)) & 0xFFFFu;
          if (pos < kListCap) r.lst[pos] = sort_key(r.tab[slot], c);
          ++pos;
          if (c == 2)
            ++twos;
          else
            atomicAdd(&r.hist[c - 1], 1u);
        }
        twos = __reduce_add_sync(kFull, twos);
        if (lane == 0 && twos) atomicAdd(&r.hist[1], twos);
      }
    } else if (pass == 0) {
      uint32_t ones = 0;
      for (uint32_t base = 0; base < S; base += 4 * kBigThreads) {
        const uint32_t i = base + 4 * threadIdx.x;
        uint4 e = make_uint4(0u, 0u, 0u, 0u);
        uint2 c2 = make_uint2(0u, 0u);
        if (i < S) {
          e = *reinterpret_cast<const uint4 *>(r.tab + i);
          c2 = *reinterpret_cast<const uint2 *>(r.aux + i / 2);
        }
        const uint32_t t[4] = {e.x, e.y, e.z, e.w};
        const uint32_t c[4] = {c2.x & 0xFFFFu, c2.x >> 16, c2.y & 0xFFFFu, c2.y >> 16};
        uint32_t nm = 0, twos = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (t[u] != 0 && c[u] == 1) ++ones;
          if (t[u] != 0 && c[u] > 1) ++nm;
          if (t[u] != 0 && c[u] == 2) ++twos;
        }
        if (__any_sync(kFull, nm != 0)) {
          // the lanes' count >= 2 entries go to the list at one position per
          // warp and round (an exclusive scan of nm); count-2 entries, the
          // common ones, are summed over the warp before they reach hist
          uint32_t inc = nm;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += x;
          }
          uint32_t pos = 0;
          if (lane == 31) pos = atomicAdd(&misc[5], inc);
          pos = __shfl_sync(kFull, pos, 31) + inc - nm;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (t[u] != 0 && c[u] > 1) {
              if (pos < kListCap) r.lst[pos] = sort_key(t[u], c[u]);
              ++pos;
              if (c[u] > 2) atomicAdd(&r.hist[c[u] - 1], 1u);
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) twos += __shfl_xor_sync(kFull, twos, o);
          if (lane == 0 && twos) atomicAdd(&r.hist[1], twos);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ones += __shfl_xor_sync(kFull, ones, o);
      if (lane == 0 && ones) atomicAdd(&r.hist[0], ones);
    } else if (!listed) {
      for_table_keys(r, S, [&](int, bool valid, uint32_t key) {
        if (valid && (key & pmask) == prefix) atomicAdd(&r.hist[(key >> shift) & 0xFFu], 1u);
      });
    } else {
      for (uint32_t i = g.rank(); i < nlist; i += g.size()) {
        const uint32_t key = r.lst[i];
        if ((key & pmask) == prefix) atomicAdd(&r.hist[(key >> shift) & 0xFFu], 1u);
      }
    }
    g.sync();
    if (g.leader_warp()) {
      if (pass == 0 && dup_known) {  // the count-1 entries: new entries less the marked slots
        if (lane == 0) r.hist[0] += misc[10] - misc[5];
        __syncwarp();
      }
      uint32_t sum = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) sum += r.hist[lane * 8 + i];
      uint32_t suf = sum;  // keys of the range with digit >= lane*8
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_down_sync(kFull, suf, o);
        if (lane + o < 32) suf += x;
      }
      const uint32_t need = misc[2], above_range = misc[7];
      const uint32_t ball = __ballot_sync(kFull, suf >= need);
      if (ball == 0) {
        // fewer keys in the range than needed (only when E < k, first pass): take all
        if (lane == 0) {  // lane 0's suffix is the whole range
          misc[4] = 1u;   // every key is >= 1 (ids < 2^24 - 1)
          misc[6] = above_range + suf;
          misc[3] = 1;
        }
      } else {
        const int ln = 31 - __clz(ball);
        if (lane == ln) {
          uint32_t cum = suf - sum;
          for (int i = 7; i >= 0; --i) {
            const uint32_t h = r.hist[lane * 8 + i];
            if (cum + h >= need) {
              const uint32_t d = static_cast<uint32_t>(lane * 8 + i);
              misc[0] = prefix | (d << shift);
              misc[1] = pmask | (0xFFu << shift);
              misc[2] = need - cum;
              misc[7] = above_range + cum;
              misc[4] = prefix | (d << shift);  // lowest key of the threshold digit
              misc[6] = above_range + cum + h;  // keys >= it
              if (misc[6] <= 256 || shift == 0) misc[3] = 1;
              break;
            }
            cum += h;
          }
        }
      }
    }
    g.sync();
    if (pass == 0) {
      // the list holds every key with count >= 2 unless it overflowed
      const uint32_t gathered = misc[5];
      if (misc[4] >= (1u << 24) && gathered <= kListCap) {
        listed = true;
        nlist = gathered;
      }
    }
    if (misc[3]) break;
    if (!listed && misc[6] <= kListCap) {  // gather the keys >= the threshold once
      const uint32_t thr = misc[4];
      g.sync();
      if (g.rank() == 0) misc[5] = 0;
      g.sync();
      for_table_keys(r, S, [&](int, bool valid, uint32_t key) {
        append_warp(r.lst, kListCap, &misc[5], valid && key >= thr, key);
      });
      g.sync();
      listed = true;
      nlist = misc[5];
    }
  }
  // the loop ended on a barrier: threshold, count and list are final
  const uint32_t thr = misc[4], nsel = misc[6];
  if (listed) {
    for (uint32_t base = 0; base < nlist; base += g.size()) {
      const uint32_t i = base + g.rank();
      const uint32_t key = i < nlist ? r.lst[i] : 0u;
      append_warp(r.hist, 256u, &misc[11], i < nlist && key >= thr, key);
    }
  } else {
    for_table_keys(r, S, [&](int, bool valid, uint32_t key) {
      append_warp(r.hist, 256u, &misc[11], valid && key >= thr, key);
    });
  }
  g.sync();
  block_rank_write(a, r.hist, nsel, q);  // the caller's barrier follows
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
  load_ids(g, a, pre_c, sb_c, table_size(M) <= a.table_words ? M : 0, 0, ids);

  while (q < nq) {
    // the claim of the query after next, and the next query's bucket ranges,
    // are in flight while this one is counted
    unsigned long long qraw = 0;
    if (lane == 0) qraw = atomicAdd(a.q_counter, 1ULL);
    uint32_t sn[TPL], en[TPL];
    load_ranges<TPL>(g, a, keys_n, sn, en);
    const bool fits = table_size(M) <= a.table_words;
    if (M > 0 && fits) count_phase_warp(g, a, r, pre_c, sb_c, static_cast<int64_t>(q), M, ids);

    // stage the next query: its ranges into the other buffer, its first ids in flight
    const unsigned long long qn2 = __shfl_sync(kFull, qraw, 0);
    uint32_t keys_n2[TPL];
    load_query_keys<TPL>(g, a, static_cast<int64_t>(qn2), keys_n2);
    const uint32_t Mn = build_ranges<TPL>(g, a, pre_n, sb_n, sn, en);
    load_ids(g, a, pre_n, sb_n, table_size(Mn) <= a.table_words ? Mn : 0, 0, ids);

    if (M == 0) {
      write_empty(g, a, static_cast<int64_t>(q));
    } else if (!fits) {
      if (lane == 0) a.overflow[atomicAdd(a.over_count, 1ULL)] = static_cast<int64_t>(q);
    } else {
      const uint32_t E = keys_from_list(g, r);
      select_phase(g, a, r, static_cast<int64_t>(q), r.aux, E);
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

// One block per query of the overflow list (all queries with all_queries).
// Tier 1 takes the queries whose candidates fit a.table_words slots at load
// below 2/3 and marks the others overflow[h] = -(q + 1) (with all_queries it
// writes every entry: q or the mark); tier 2 takes exactly the marked ones.
// The block's next queries are staged while it works on one: the bucket
// ranges of the next, the addresses of the one after, and the list entry of
// the third (each load's result is used one iteration later).
__global__ void __launch_bounds__(kBigThreads, 2) query_big_kernel(QArgs a, int all_queries, int tier) {
  extern __shared__ uint32_t smem[];
  const BlockGroup g;
  const Region r = carve_big(smem, a);
  const int64_t count = all_queries ? a.nq : static_cast<int64_t>(*a.over_count);
  constexpr int64_t kNone = INT64_MIN;
  // the list entry of index h (its query in tier 1, the mark tier 1 left in
  // tier 2), kNone past the end
  auto entry = [&](int64_t h) -> int64_t {
    if (h >= count) return kNone;
    return (all_queries && tier == 1) ? h : a.overflow[h];
  };
  // the query an entry stands for in this tier, -1 for none
  auto query_of = [&](int64_t v) -> int64_t {
    if (v == kNone) return -1;
    if (tier == 1) return v;
    return v < 0 ? -v - 1 : -1;
  };
  const int64_t step = gridDim.x;
  int64_t h = blockIdx.x;
  int64_t q = query_of(entry(h));
  uint32_t s_c, e_c;
  head_range(a, head_key(a, q), s_c, e_c);
  int64_t qn = query_of(entry(h + step));
  uint32_t key_n = head_key(a, qn);
  int64_t raw_n2 = entry(h + 2 * step);
  for (; h < count; h += step) {
    uint32_t s_n, e_n;
    head_range(a, key_n, s_n, e_n);
    const int64_t qn2 = query_of(raw_n2);
    const uint32_t key_n2 = head_key(a, qn2);
    const int64_t raw_n3 = entry(h + 3 * step);
    if (q >= 0) {
      const uint32_t M = build_streams(g, a, r, s_c, e_c);
      const uint32_t S = big_table_size(M);
      const bool defer = tier == 1 && S > a.table_words;
      if (tier == 1 && threadIdx.x == 0 && (defer || all_queries)) a.overflow[h] = defer ? -q - 1 : q;
      if (defer) {
        // left to tier 2
      } else if (M == 0) {
        write_empty(g, a, q);
      } else {
        const int warp = threadIdx.x >> 5;
        const uint32_t ntab = a.L > static_cast<uint32_t>(warp) ? (a.L - warp + kBigWarps - 1) / kBigWarps : 0;
        const uint32_t *wp = r.wpre + warp * (kMaxTabPerWarp + 1);
        const uint32_t nbatch = (r.misc[9] + 32 * kBatch - 1) / (32 * kBatch);
        // the CAS count (one or two batches) probes a table twice the size when
        // the region has room: at load <= 1/3 a warp's longest probe chain, which
        // every lane of the warp waits for, is shorter
        const uint32_t St = (nbatch <= 2 && 2 * S <= a.table_words) ? 2 * S : S;
        int32_t ids[kBatch];
        uint32_t cur = 0;
        load_stream_ids(a, wp, r.off + warp * kMaxTabPerWarp, wp[ntab], 0, cur, ids);
        count_phase_block(g, a, r, q, nbatch, ids, cur, St);
        if (a.k <= 256) {
          select_from_table(g, a, r, q, St, nbatch <= 2);
        } else {
          const uint32_t E = compact_keys(g, r.tab, r.aux, St, r.hist);
          select_phase(g, a, r, q, r.tab, E);
        }
      }
      g.sync();
    }
    q = qn;
    qn = qn2;
    s_c = s_n;
    e_c = e_n;
    key_n = key_n2;
    raw_n2 = raw_n3;
  }
}

size_t max_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return static_cast<size_t>(v);
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
  a.st_stride = l.shared ? 0 : static_cast<int64_t>(a.T) + 1;
  a.id_stride = l.shared ? 0 : l.n;
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

  // The warp path takes queries of at most tw / 2 candidates.  In the all-points
  // graph every table's bucket holds the query row itself, so a query has at
  // least L candidates: with L >= tw / 2 (nearly) every query would only be
  // passed on to the block path, and the warp kernel is skipped.
  const uint32_t full_table = next_pow2(2 * l.L * l.R) < 64 ? 64 : next_pow2(2 * l.L * l.R);
  uint32_t tw = l.warp_table ? l.warp_table : 512u;
  if (tw > full_table) tw = full_table;
  // It is skipped too when the index's buckets hold so many points that a
  // typical query would not fit either: expected candidates L * min(points per
  // bucket, R) above twice what the warp table takes (tw / 2).
  const double per_bucket = (l.shared ? static_cast<double>(l.L) * l.n : static_cast<double>(l.n)) / a.T;
  const double expected_m = static_cast<double>(l.L) * (per_bucket < l.R ? per_bucket : static_cast<double>(l.R));
  const bool mostly_big = expected_m > static_cast<double>(tw);
  const bool warp_ok = l.k <= 256 && !(l.exclude_self && 2 * l.L >= tw) && !mostly_big;
  int all = 1;
  if (warp_ok) {
    a.table_words = tw;
    a.region_words = region_words(a);
    while (a.table_words > 64 && static_cast<size_t>(kQWarps) * a.region_words * sizeof(uint32_t) > max_smem_optin()) {
      a.table_words >>= 1;  // a tuned table too large for this device's shared memory
      a.region_words = region_words(a);
    }
    const uint32_t tpl = (l.L + 31) / 32;
    int rc;
    if (tpl <= 1) rc = launch_warp<1>(a, l.nq, stream);
    else if (tpl <= 2) rc = launch_warp<2>(a, l.nq, stream);
    else if (tpl <= 4) rc = launch_warp<4>(a, l.nq, stream);
    else rc = launch_warp<8>(a, l.nq, stream);
    if (rc) return rc;
    all = 0;
  }
  // block path: tier 1 with a 64 KB table (or one sized for L*R when smaller),
  // tier 2 with a table sized for L*R when some query may not fit tier 1
  const uint32_t need = big_table_size(l.L * l.R);
  const uint32_t tw1 = need < kBigTable ? need : kBigTable;
  for (int tier = 1; tier <= (need > tw1 ? 2 : 1); ++tier) {
    a.table_words = tier == 1 ? tw1 : need;
    a.region_words = big_region_words(a);
    const size_t smem_b = static_cast<size_t>(a.region_words) * sizeof(uint32_t);
    if (cudaFuncSetAttribute(query_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_b)) != cudaSuccess)
      return FLASH_ECUDA;
    int per_sm_b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, query_big_kernel, kBigThreads, smem_b) !=
        cudaSuccess)
      return FLASH_ECUDA;
    if (per_sm_b < 1) return FLASH_EINVAL;
    int64_t blocks_b = static_cast<int64_t>(per_sm_b) * num_sms();
    if (all && blocks_b > l.nq) blocks_b = l.nq;
    query_big_kernel<<<static_cast<unsigned>(blocks_b), kBigThreads, smem_b, stream>>>(a, all, tier);
    count_launches(1);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
