// sort.cu -- K2: group every table's points by bucket (the Adding phase of
// Algorithm 2 visits points in id order; a STABLE sort by bucket address
// reproduces that order inside every bucket, so a point's position in its
// bucket segment is its arrival rank).
//
// Each table t is a segment of n addresses keys[t][0..n) (point id = index).
// An address has rb bits; the sentinel 2^rb (rows never inserted) sorts last.
// The sort runs in two stages:
//   1. partition: a stable least-significant-digit radix sort on the high
//      hb = rb - lo bits only (lo = min(rb, 10)), digits of at most 8 bits,
//      so the table falls into 2^hb + 1 segments (the last one holds the
//      sentinels).  Per pass:
//        hist    : per (table, tile) digit histogram (shared-memory atomics);
//        scan    : per table exclusive scan of the [digit][tile] counts;
//        scatter : per (table, tile) stable ranking -- warps take consecutive
//                  32-element rounds, lanes with equal digits in a round
//                  find each other through a shared-memory OR mask, per-warp running counts and a per-digit
//                  prefix over warps keep the tile's element order -- a stable
//                  local sort of the tile by digit in shared memory, and
//                  coalesced writes of each digit run to scan offset +
//                  position in the run.
//      With one pass the scan already holds every segment's start; with more,
//      the first pass also counts all the high bits per table, and the scan of
//      that histogram gives the starts.
//   2. segments: one warp per segment (about n / 2^hb points) counts its 2^lo
//      low digits in shared memory, scans them, writes the bucket starts of
//      its 2^lo buckets and lists the buckets holding more than R points, and
//      places every point at its bucket's offset + its rank among the equal
//      digits before it (32-element rounds in id order, equal digits of a
//      round found through a shared-memory OR mask).
//      The segment of sentinels is copied as it is.
// starts[t][b] = number of addresses < b in table t, for b in [0, 2^rb].
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kSortWarps = 16;  // per (table, tile) block: 16 warps of 8 ranking rounds (measured against 8 and 32)
constexpr int kTile = 4096;         // elements per (table, tile) block, histogram and scatter
constexpr int kMaxBinsSort = 257;   // 8-bit digit + the sentinel value
constexpr uint32_t kFullSmem = 8193;  // high-bit histograms up to 2^13 + 1 values in shared memory
constexpr int kLoBits = 10;         // low address bits sorted per segment (2^10 counters per warp)
constexpr int kSegWarps = 8;        // warps per block of the segment kernel
constexpr int kSegBatch = 4;        // rounds of 32 points a segment warp has in flight (8 measured slower)
constexpr unsigned kFull = 0xFFFFFFFFu;

struct PassArgs {
  int shift, bits, nbins;
  bool top;
};

__device__ __forceinline__ uint32_t digit_of(uint32_t key, const PassArgs &p) {
  return p.top ? (key >> p.shift) : ((key >> p.shift) & ((1u << p.bits) - 1u));
}

// Lanes of the warp holding the same digit d in this round (valid lanes only):
// every valid lane ORs its bit into mask[d], and reads the mask back.  The
// caller clears mask[d] (the round's lowest such lane) after a __syncwarp().
// A shared-memory OR and a load cost a fraction of __match_any_sync here.
__device__ __forceinline__ uint32_t round_peers(uint32_t *mask, uint32_t d, bool valid, int lane) {
  if (valid) atomicOr(&mask[d], 1u << lane);
  __syncwarp();
  return valid ? mask[d] : 0u;
}

// Per (table, tile) digit histogram of one partition pass.  With FULL (the
// first of several passes), also the table's histogram of all the high bits
// (address >> lo, nfull = 2^hb + 1 values with the sentinel), added into
// full[t][.]: its exclusive scan gives every segment's start, so no later pass
// has to read the partitioned addresses again to find them.  Without FULL a
// block takes one tile; with it a few blocks per table walk its tiles, so that
// the high-bit histogram is added once per block.
template <bool FULL>
__global__ void __launch_bounds__(256) radix_hist_kernel(const uint32_t *keys, int64_t n, PassArgs p, uint32_t tile,
                                                          int64_t tiles, uint32_t *hist, uint32_t *full, uint32_t lo,
                                                          uint32_t nfull) {
  __shared__ uint32_t h[kMaxBinsSort + 7];
  extern __shared__ uint32_t hf[];  // [nfull] when FULL and nfull <= kFullSmem
  const uint32_t t = blockIdx.y;
  const bool fsm = FULL && nfull <= kFullSmem;
  if (fsm)
    for (uint32_t i = threadIdx.x; i < nfull; i += blockDim.x) hf[i] = 0;
  const uint32_t *seg = keys + static_cast<int64_t>(t) * n;
  uint32_t *ft = FULL ? full + static_cast<int64_t>(t) * nfull : nullptr;
  for (int64_t ti = blockIdx.x; ti < tiles; ti += FULL ? gridDim.x : tiles) {
    for (int i = threadIdx.x; i < p.nbins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t a = ti * tile, b = min(n, a + static_cast<int64_t>(tile));
    for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
      const uint32_t key = __ldcs(seg + e);
      atomicAdd(&h[digit_of(key, p)], 1u);
      if (FULL) {
        if (fsm)
          atomicAdd(&hf[key >> lo], 1u);
        else
          atomicAdd(&ft[key >> lo], 1u);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p.nbins; i += blockDim.x)
      hist[(static_cast<int64_t>(t) * p.nbins + i) * tiles + ti] = h[i];
  }
  if (fsm) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nfull; i += blockDim.x)
      if (hf[i]) atomicAdd(&ft[i], hf[i]);
  }
}

// exclusive scan of hist[t][0..len) in place, one block per table
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *hist, int64_t len) {
  constexpr int kItems = 4;
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  uint32_t *h = hist + static_cast<int64_t>(blockIdx.x) * len;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < len; base += static_cast<int64_t>(blockDim.x) * kItems) {
    uint32_t v[kItems];
    uint32_t sum = 0;
    const int64_t i0 = base + static_cast<int64_t>(threadIdx.x) * kItems;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      v[j] = (i0 + j < len) ? h[i0 + j] : 0u;
      sum += v[j];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t x = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += x;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < nwarps ? warp_tot[lane] : 0u;
      uint32_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t x = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += x;
      }
      if (lane < nwarps) warp_tot[lane] = wi - w;  // exclusive
    }
    __syncthreads();
    uint32_t run = carry + warp_tot[warp] + inc - sum;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      if (i0 + j < len) h[i0 + j] = run;
      run += v[j];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = run;
    __syncthreads();
  }
}

// Scatter of one (table, tile) block: rank, sort the tile locally by digit
// into shared memory (stable), then write every digit run of the tile to its
// global place with consecutive threads on consecutive addresses.
template <bool FIRST>
__global__ void __launch_bounds__(kSortWarps * 32, 3) radix_scatter_kernel(const uint32_t *keys_in, const int32_t *ids_in,
                                                                       int64_t n, PassArgs p, int64_t tiles,
                                                                       const uint32_t *offs, uint32_t *keys_out,
                                                                       int32_t *ids_out, int nb_pad) {
  extern __shared__ uint32_t sm[];
  uint32_t *skey = sm;                                          // [kTile] keys in digit order
  int32_t *sid = reinterpret_cast<int32_t *>(skey + kTile);     // [kTile] ids in digit order
  uint32_t *wcnt = reinterpret_cast<uint32_t *>(sid + kTile);   // [kSortWarps][nb_pad]
  uint32_t *wpref = wcnt + kSortWarps * nb_pad;                 // [kSortWarps][nb_pad]
  uint32_t *toff = wpref + kSortWarps * nb_pad;                 // [nb_pad] digit offset inside the tile
  uint32_t *gdel = toff + nb_pad;                               // [nb_pad] table offset - tile offset of a digit
  const uint32_t t = blockIdx.y;
  const int64_t ti = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = static_cast<int64_t>(t) * n;
  const int64_t a = ti * kTile;
  const int cnt = static_cast<int>(min(n - a, static_cast<int64_t>(kTile)));
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t *my_cnt = wcnt + warp * nb_pad;
  for (int d = threadIdx.x; d < p.nbins; d += blockDim.x) gdel[d] = offs[(static_cast<int64_t>(t) * p.nbins + d) * tiles + ti];
  uint32_t *my_mask = wpref + warp * nb_pad;  // lanes holding a digit in the current round (step 1 only)
  for (int d = lane; d < p.nbins; d += 32) {
    my_cnt[d] = 0;
    my_mask[d] = 0;
  }
  __syncwarp();

  // 1. load (coalesced) and rank: warp w holds tile elements [w*W, (w+1)*W) in 32-element rounds
  constexpr int kPerWarp = kTile / kSortWarps;
  constexpr int kRounds = kPerWarp / 32;
  uint32_t dr[kRounds];  // digit << 16 | rank among the warp's equal digits
  uint32_t kk[kRounds];
  int32_t vv[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int e = warp * kPerWarp + r * 32 + lane;
    kk[r] = e < cnt ? __ldcs(keys_in + seg + a + e) : 0u;
    if (FIRST)
      vv[r] = static_cast<int32_t>(a + e);
    else
      vv[r] = e < cnt ? __ldcs(ids_in + seg + a + e) : 0;
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int e = warp * kPerWarp + r * 32 + lane;
    const bool valid = e < cnt;
    const uint32_t d = valid ? digit_of(kk[r], p) : 0xFFFFu;
    const uint32_t peers = round_peers(my_mask, d, valid, lane);
    const uint32_t lower = peers & lt_mask;
    const uint32_t before = valid ? my_cnt[d] : 0u;
    __syncwarp();
    if (valid && lower == 0) {
      my_cnt[d] = before + __popc(peers);
      my_mask[d] = 0;
    }
    __syncwarp();
    dr[r] = (d << 16) | (before + __popc(lower));
  }
  __syncthreads();

  // 2. per digit: warp prefixes and the tile count; then offsets of the digits inside the tile
  for (int d = threadIdx.x; d < p.nbins; d += blockDim.x) {
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      wpref[w * nb_pad + d] = acc;
      acc += wcnt[w * nb_pad + d];
    }
    toff[d] = acc;
  }
  __syncthreads();
  if (warp == 0) {
    const int per = (p.nbins + 31) / 32;
    uint32_t sum = 0;
    for (int i = 0; i < per; ++i) {
      const int d = lane * per + i;
      if (d < p.nbins) sum += toff[d];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += x;
    }
    uint32_t run = inc - sum;
    for (int i = 0; i < per; ++i) {
      const int d = lane * per + i;
      if (d < p.nbins) {
        const uint32_t c = toff[d];
        toff[d] = run;
        gdel[d] -= run;  // table offset >= tile offset: counts of the smaller digits of this tile are in both
        run += c;
      }
    }
  }
  __syncthreads();

  // 3. stable local order by digit: keys and ids straight to their tile position
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const uint32_t d = dr[r] >> 16;
    if (d != 0xFFFFu) {
      const uint32_t pos = toff[d] + wpref[warp * nb_pad + d] + (dr[r] & 0xFFFFu);
      skey[pos] = kk[r];
      sid[pos] = vv[r];
    }
  }
  __syncthreads();

  // 4. coalesced writes of the digit runs (independent iterations, unrolled)
  constexpr int kPerThread = kTile / (kSortWarps * 32);
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int i = j * kSortWarps * 32 + static_cast<int>(threadIdx.x);
    if (i < cnt) {
      const uint32_t key = skey[i];
      const int64_t dest = seg + gdel[digit_of(key, p)] + static_cast<uint32_t>(i);
      keys_out[dest] = key;
      ids_out[dest] = sid[i];
    }
  }
}

size_t scatter_smem_bytes(int nb_pad) {
  return sizeof(uint32_t) * (2 * kTile + (2 * kSortWarps + 2) * static_cast<size_t>(nb_pad));
}

__host__ __device__ __forceinline__ uint32_t cpad(uint32_t d) { return d + (d >> 5); }
__host__ __device__ __forceinline__ uint32_t seg_counter_words(uint32_t lo) {
  return cpad(1u << lo) + 1u;
}

struct SegArgs {
  const uint32_t *pkeys;     // [L][n] addresses partitioned by their high bits
  const int32_t *pids;       // [L][n] point ids in the same order
  int64_t n;
  uint32_t L, lo, hb;        // address = (segment << lo) | low digit; 2^hb regular segments + the sentinels
  const uint32_t *seg;       // start of segment s of table t: seg[t * seg_tstride + s * seg_sstride]
  int64_t seg_tstride, seg_sstride;
  int32_t *ids_out;          // [L][n] point ids in (address, id) order
  uint32_t *starts;          // [L][2^rb + 1]
  uint32_t R;
  unsigned long long *heavy_count;  // buckets with more than R points: (t << 32 | b), capacity heavy_cap
  uint64_t *heavy;
  int64_t heavy_cap;
  unsigned long long *claim;  // segment claims (zeroed before the launch)
};

// One warp per segment: count the low digits, scan, write the bucket starts and
// the heavy buckets, place every point (stable).  Segments are claimed from the
// last table backwards: the partition wrote the last tables last, so their
// addresses and ids are the ones still in L2.
__global__ void __launch_bounds__(kSegWarps * 32) segment_sort_kernel(SegArgs a) {
  extern __shared__ uint32_t seg_sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nb = 1u << a.lo, dmask = nb - 1u;
  // counter of digit d at d + d / 32: a lane's run of 32 consecutive digits
  // (the scan) and 32 lanes on consecutive digits both touch 32 distinct banks
  uint32_t *cnt = seg_sm + static_cast<size_t>(warp) * (seg_counter_words(a.lo) + nb);
  uint32_t *msk = cnt + seg_counter_words(a.lo);  // [nb] lanes holding a digit in the current round
  const uint32_t nseg = (1u << a.hb) + 1u;
  const uint64_t total = static_cast<uint64_t>(a.L) * nseg;
  const uint32_t T = 1u << (a.lo + a.hb);
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t keep = l2_policy_keep();
  for (;;) {
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(a.claim, 1ULL);
    g = __shfl_sync(kFull, g, 0);
    if (g >= total) break;
    g = total - 1 - g;
    const uint32_t t = static_cast<uint32_t>(g / nseg), s = static_cast<uint32_t>(g - static_cast<uint64_t>(t) * nseg);
    const uint32_t *sb = a.seg + static_cast<int64_t>(t) * a.seg_tstride;
    const uint32_t so = sb[static_cast<int64_t>(s) * a.seg_sstride];
    const uint32_t se = s + 1 < nseg ? sb[static_cast<int64_t>(s + 1) * a.seg_sstride] : static_cast<uint32_t>(a.n);
    const int64_t tb = static_cast<int64_t>(t) * a.n;
    const uint32_t *pk = a.pkeys + tb;
    const int32_t *pi = a.pids + tb;
    int32_t *out = a.ids_out + tb;
    uint32_t *st = a.starts + static_cast<int64_t>(t) * (static_cast<int64_t>(T) + 1);
    if (s + 1 == nseg) {  // the points never inserted: already in id order
      if (lane == 0) st_l2(st + T, so, keep);
      for (uint32_t i = so + lane; i < se; i += 32) st_l2(out + i, pi[i], keep);
      continue;
    }
    for (uint32_t d = lane; d < nb; d += 32) {
      cnt[cpad(d)] = 0;
      msk[d] = 0;
    }
    __syncwarp();
    // count the low digits (the next kSegBatch * 32 addresses are loaded while as
    // many are counted)
    {
      uint32_t k[kSegBatch], kn[kSegBatch];
#pragma unroll
      for (int r = 0; r < kSegBatch; ++r) {
        const uint32_t i = so + r * 32 + lane;
        k[r] = i < se ? pk[i] : 0xFFFFFFFFu;
      }
      for (uint32_t base = so; base < se; base += kSegBatch * 32) {
#pragma unroll
        for (int r = 0; r < kSegBatch; ++r) {
          const uint32_t i = base + kSegBatch * 32 + r * 32 + lane;
          kn[r] = i < se ? pk[i] : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int r = 0; r < kSegBatch; ++r)
          if (k[r] != 0xFFFFFFFFu) atomicAdd(&cnt[cpad(k[r] & dmask)], 1u);
#pragma unroll
        for (int r = 0; r < kSegBatch; ++r) k[r] = kn[r];
      }
    }
    // exclusive scan in place (lane owns a run of consecutive digits); heavy buckets
    {
      const uint32_t per = (nb + 31) / 32;
      const uint32_t d0 = min(nb, lane * per), d1 = min(nb, d0 + per);
      uint32_t sum = 0;
      for (uint32_t d = d0; d < d1; ++d) {
        const uint32_t c = cnt[cpad(d)];
        sum += c;
        if (c > a.R && a.heavy_count) {
          const unsigned long long h = atomicAdd(a.heavy_count, 1ULL);
          if (static_cast<int64_t>(h) < a.heavy_cap)
            a.heavy[h] = (static_cast<uint64_t>(t) << 32) | ((s << a.lo) | d);
        }
      }
      uint32_t inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += x;
      }
      uint32_t run = so + inc - sum;
      for (uint32_t d = d0; d < d1; ++d) {
        const uint32_t c = cnt[cpad(d)];
        cnt[cpad(d)] = run;
        run += c;
      }
    }
    __syncwarp();
    for (uint32_t d = lane; d < nb; d += 32) st_l2(st + ((s << a.lo) | d), cnt[cpad(d)], keep);
    __syncwarp();
    // place: rank among equal digits of the round, after the earlier rounds
    // (the next kSegBatch * 32 points are loaded while as many are placed)
    uint32_t kk[kSegBatch];
    int32_t id[kSegBatch];
#pragma unroll
    for (int r = 0; r < kSegBatch; ++r) {
      const uint32_t i = so + r * 32 + lane;
      kk[r] = i < se ? pk[i] : 0u;
      id[r] = i < se ? pi[i] : 0;
    }
    for (uint32_t base = so; base < se; base += kSegBatch * 32) {
      uint32_t kn[kSegBatch];
      int32_t idn[kSegBatch];
#pragma unroll
      for (int r = 0; r < kSegBatch; ++r) {
        const uint32_t i = base + kSegBatch * 32 + r * 32 + lane;
        kn[r] = i < se ? pk[i] : 0u;
        idn[r] = i < se ? pi[i] : 0;
      }
#pragma unroll
      for (int r = 0; r < kSegBatch; ++r) {
        const uint32_t i = base + r * 32 + lane;
        if (base + r * 32 < se) {  // warp-uniform
          const bool valid = i < se;
          const uint32_t d = kk[r] & dmask;
          const uint32_t peers = round_peers(msk, d, valid, lane);
          const uint32_t before = valid ? cnt[cpad(d)] : 0u;
          __syncwarp();
          if (valid && (peers & lt_mask) == 0) {
            cnt[cpad(d)] = before + __popc(peers);
            msk[d] = 0;
          }
          __syncwarp();
          if (valid) st_l2(out + before + __popc(peers & lt_mask), id[r], keep);
        }
      }
#pragma unroll
      for (int r = 0; r < kSegBatch; ++r) {
        kk[r] = kn[r];
        id[r] = idn[r];
      }
    }
  }
}

}  // namespace

SortPlan make_sort_plan(uint32_t range_bits, int64_t n, uint32_t L) {
  SortPlan p{};
  p.lo_bits = static_cast<int>(range_bits) < kLoBits ? static_cast<int>(range_bits) : kLoBits;
  p.hi_bits = static_cast<int>(range_bits) - p.lo_bits;
  p.passes = (p.hi_bits + 7) / 8;
  if (p.passes < 1) p.passes = 1;  // hi_bits = 0: one pass still moves the sentinels last
  const int base = p.hi_bits / p.passes, extra = p.hi_bits % p.passes;
  int shift = p.lo_bits, maxb = 0;
  for (int i = 0; i < p.passes; ++i) {
    p.bits[i] = base + (i < extra ? 1 : 0);
    p.shift[i] = shift;
    shift += p.bits[i];
    p.nbins[i] = (1 << p.bits[i]) + (i == p.passes - 1 ? 1 : 0);
    if (p.nbins[i] > maxb) maxb = p.nbins[i];
  }
  p.tile = kTile;
  p.tiles = n > 0 ? (n + p.tile - 1) / p.tile : 0;
  p.hist_words = static_cast<int64_t>(L) * maxb * (p.tiles > 0 ? p.tiles : 1);
  p.seg_words = p.passes > 1 ? static_cast<int64_t>(L) * ((1LL << p.hi_bits) + 1) : 0;
  return p;
}

int sort_tables(const SortPlan &plan, const SortLaunch &s, cudaStream_t stream) {
  const int64_t T = 1LL << s.range_bits;
  if (s.n == 0) {
    return cudaMemsetAsync(s.starts, 0, sizeof(uint32_t) * s.L * (T + 1), stream) == cudaSuccess ? 0 : FLASH_ECUDA;
  }
  // 1. partition by the high bits; passes alternate between (tmp_keys, tmp_ids)
  //    and (keys_out, tmp_ids2)
  const dim3 grid(static_cast<unsigned>(plan.tiles), s.L);
  const uint32_t *kin = s.keys_in;
  const int32_t *vin = nullptr;
  const uint32_t S = 1u << plan.hi_bits;
  if (plan.passes > 1 &&
      cudaMemsetAsync(s.seg, 0, sizeof(uint32_t) * s.L * (static_cast<size_t>(S) + 1), stream) != cudaSuccess)
    return FLASH_ECUDA;
  for (int pass = 0; pass < plan.passes; ++pass) {
    PassArgs pa{plan.shift[pass], plan.bits[pass], plan.nbins[pass], pass == plan.passes - 1};
    uint32_t *kout = pass % 2 == 0 ? s.tmp_keys : s.keys_out;
    int32_t *vout = pass % 2 == 0 ? s.tmp_ids : s.tmp_ids2;
    uint32_t *full = (plan.passes > 1 && pass == 0) ? s.seg : nullptr;
    const size_t hsm = full && S + 1 <= kFullSmem ? sizeof(uint32_t) * (S + 1) : 0;
    // with the high-bit histogram, a few blocks per table walk its tiles (the histogram is
    // added once per block); otherwise a block per tile
    if (full) {
      int64_t hx = (16LL * num_sms() + s.L - 1) / s.L;
      if (hx > plan.tiles) hx = plan.tiles;
      if (hx < 1) hx = 1;
      radix_hist_kernel<true><<<dim3(static_cast<unsigned>(hx), s.L), 256, hsm, stream>>>(
          kin, s.n, pa, plan.tile, plan.tiles, s.hist, full, static_cast<uint32_t>(plan.lo_bits), S + 1);
    } else {
      radix_hist_kernel<false><<<grid, 256, 0, stream>>>(kin, s.n, pa, plan.tile, plan.tiles, s.hist, nullptr, 0, 0);
    }
    radix_scan_kernel<<<s.L, 1024, 0, stream>>>(s.hist, static_cast<int64_t>(pa.nbins) * plan.tiles);
    const int nb_pad = (pa.nbins + 3) & ~3;
    const size_t smem = scatter_smem_bytes(nb_pad);
    auto kern = pass == 0 ? radix_scatter_kernel<true> : radix_scatter_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
      return FLASH_ECUDA;
    kern<<<grid, kSortWarps * 32, smem, stream>>>(kin, vin, s.n, pa, plan.tiles, s.hist, kout, vout, nb_pad);
    count_launches(3);
    kin = kout;
    vin = vout;
  }
  // 2. segment starts: from the scan of a single pass (digit s of table t at
  //    hist[(t * nbins + s) * tiles]), else read off the partitioned addresses
  SegArgs a{};
  a.pkeys = kin;
  a.pids = vin;
  a.n = s.n;
  a.L = s.L;
  a.lo = static_cast<uint32_t>(plan.lo_bits);
  a.hb = static_cast<uint32_t>(plan.hi_bits);
  if (plan.passes == 1) {
    a.seg = s.hist;
    a.seg_tstride = static_cast<int64_t>(plan.nbins[0]) * plan.tiles;
    a.seg_sstride = plan.tiles;
  } else {
    // segment starts: exclusive scan of the high-bit histogram the first pass counted
    radix_scan_kernel<<<s.L, 1024, 0, stream>>>(s.seg, static_cast<int64_t>(S) + 1);
    count_launches(1);
    a.seg = s.seg;
    a.seg_tstride = static_cast<int64_t>(S) + 1;
    a.seg_sstride = 1;
  }
  a.ids_out = s.ids_out;
  a.starts = s.starts;
  a.R = s.R;
  a.heavy_count = s.heavy_count;
  a.heavy = s.heavy;
  a.heavy_cap = s.heavy_cap;
  a.claim = s.claim;
  // 3. one warp per segment
  if (cudaMemsetAsync(s.claim, 0, sizeof(unsigned long long), stream) != cudaSuccess) return FLASH_ECUDA;
  if (s.heavy_count && cudaMemsetAsync(s.heavy_count, 0, sizeof(unsigned long long), stream) != cudaSuccess)
    return FLASH_ECUDA;
  const size_t smem = sizeof(uint32_t) * kSegWarps *
                      (seg_counter_words(static_cast<uint32_t>(plan.lo_bits)) + (1u << plan.lo_bits));
  if (cudaFuncSetAttribute(segment_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return FLASH_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, segment_sort_kernel, kSegWarps * 32, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return FLASH_ECUDA;
  const int64_t segs = static_cast<int64_t>(s.L) * (static_cast<int64_t>(S) + 1);
  int64_t blocks = static_cast<int64_t>(per_sm) * num_sms();
  const int64_t need = (segs + kSegWarps - 1) / kSegWarps;
  if (blocks > need) blocks = need;
  segment_sort_kernel<<<static_cast<unsigned>(blocks), kSegWarps * 32, smem, stream>>>(a);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
