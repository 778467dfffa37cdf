// sort.cu -- K2: group every table's points by bucket (the Adding phase of
// Algorithm 2 visits points in id order; a STABLE sort by bucket address
// reproduces that order inside every bucket, so a point's position in its
// bucket segment is its arrival rank).
//
// Each table t is a segment of n addresses keys[t][0..n) (point id = index).
// A least-significant-digit radix sort with digits of at most 8 bits sorts
// all segments at once; the sentinel address 2^rb (rows never inserted) is
// one extra value of the most significant digit and sorts last.  Per pass:
//   hist    : per (table, tile) digit histogram (shared-memory atomics);
//   scan    : per table exclusive scan of the [digit][tile] counts;
//   scatter : per (table, tile) stable ranking -- warps take consecutive
//             32-element rounds, __match_any_sync ranks equal digits within
//             a round, per-warp running counts and a per-digit prefix over
//             warps keep the tile's element order -- a stable local sort of
//             the tile by digit in shared memory, and coalesced writes of each
//             digit run to scan offset + position in the run.
// Finally the bucket starts: starts[t][b] = number of addresses < b in table
// t, for b in [0, 2^rb]; each key change writes the starts of the buckets it
// skips: a short run by its own thread, a long run by the whole warp.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kSortWarps = 16;  // per (table, tile) block: 16 warps of 8 ranking rounds (measured against 8 and 32)
constexpr int kTile = 4096;         // elements per (table, tile) block, histogram and scatter
constexpr int kMaxBinsSort = 257;   // 8-bit digit + the sentinel value
constexpr unsigned kFull = 0xFFFFFFFFu;

struct PassArgs {
  int shift, bits, nbins;
  bool top;
};

__device__ __forceinline__ uint32_t digit_of(uint32_t key, const PassArgs &p) {
  return p.top ? (key >> p.shift) : ((key >> p.shift) & ((1u << p.bits) - 1u));
}

__global__ void __launch_bounds__(256) radix_hist_kernel(const uint32_t *keys, int64_t n, PassArgs p, uint32_t tile,
                                                          int64_t tiles, uint32_t *hist) {
  __shared__ uint32_t h[kMaxBinsSort + 7];
  const uint32_t t = blockIdx.y;
  const int64_t ti = blockIdx.x;
  for (int i = threadIdx.x; i < p.nbins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t *seg = keys + static_cast<int64_t>(t) * n;
  const int64_t a = ti * tile, b = min(n, a + static_cast<int64_t>(tile));
  for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) atomicAdd(&h[digit_of(__ldcs(seg + e), p)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < p.nbins; i += blockDim.x)
    hist[(static_cast<int64_t>(t) * p.nbins + i) * tiles + ti] = h[i];
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
// in shared memory (stable), then write every digit run of the tile to its
// global place with consecutive threads on consecutive addresses.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kSortWarps * 32) radix_scatter_kernel(const uint32_t *keys_in, const int32_t *ids_in,
                                                                       int64_t n, PassArgs p, int64_t tiles,
                                                                       const uint32_t *offs, uint32_t *keys_out,
                                                                       int32_t *ids_out, int nb_pad) {
  extern __shared__ uint32_t sm[];
  uint32_t *skey = sm;                                          // [kTile] keys, tile order
  int32_t *sid = reinterpret_cast<int32_t *>(skey + kTile);     // [kTile] ids (not FIRST)
  uint32_t *wcnt = reinterpret_cast<uint32_t *>(sid + (FIRST ? 0 : kTile));  // [kSortWarps][nb_pad]
  uint32_t *wpref = wcnt + kSortWarps * nb_pad;                 // [kSortWarps][nb_pad]
  uint32_t *toff = wpref + kSortWarps * nb_pad;                 // [nb_pad] digit offset inside the tile
  uint32_t *goff = toff + nb_pad;                               // [nb_pad] digit offset in the table
  uint16_t *perm = reinterpret_cast<uint16_t *>(goff + nb_pad); // [kTile] tile index in digit order
  const uint32_t t = blockIdx.y;
  const int64_t ti = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = static_cast<int64_t>(t) * n;
  const int64_t a = ti * kTile;
  const int cnt = static_cast<int>(min(n - a, static_cast<int64_t>(kTile)));
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t *my_cnt = wcnt + warp * nb_pad;
  for (int d = threadIdx.x; d < p.nbins; d += blockDim.x) goff[d] = offs[(static_cast<int64_t>(t) * p.nbins + d) * tiles + ti];
  for (int d = lane; d < p.nbins; d += 32) my_cnt[d] = 0;
  __syncwarp();

  // 1. load (coalesced) and rank: warp w holds tile elements [w*W, (w+1)*W) in 32-element rounds
  constexpr int kPerWarp = kTile / kSortWarps;
  constexpr int kRounds = kPerWarp / 32;
  uint32_t dr[kRounds];  // digit << 16 | rank among the warp's equal digits
  uint32_t kk[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int e = warp * kPerWarp + r * 32 + lane;
    kk[r] = e < cnt ? __ldcs(keys_in + seg + a + e) : 0u;
  }
  if (!FIRST) {
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int e = warp * kPerWarp + r * 32 + lane;
      if (e < cnt) sid[e] = __ldcs(ids_in + seg + a + e);
    }
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int e = warp * kPerWarp + r * 32 + lane;
    const bool valid = e < cnt;
    if (valid) skey[e] = kk[r];
    const uint32_t d = valid ? digit_of(kk[r], p) : 0xFFFFu;
    const uint32_t peers = __match_any_sync(kFull, d);
    const uint32_t lower = peers & lt_mask;
    const uint32_t before = valid ? my_cnt[d] : 0u;
    __syncwarp();
    if (valid && lower == 0) my_cnt[d] = before + __popc(peers);
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
        run += c;
      }
    }
  }
  __syncthreads();

  // 3. stable local order by digit
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const uint32_t d = dr[r] >> 16;
    if (d != 0xFFFFu) {
      const int e = warp * kPerWarp + r * 32 + lane;
      perm[toff[d] + wpref[warp * nb_pad + d] + (dr[r] & 0xFFFFu)] = static_cast<uint16_t>(e);
    }
  }
  __syncthreads();

  // 4. coalesced writes of the digit runs
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int e = perm[i];
    const uint32_t key = skey[e];
    const uint32_t d = digit_of(key, p);
    const int64_t dest = seg + goff[d] + (static_cast<uint32_t>(i) - toff[d]);
    const int32_t id = FIRST ? static_cast<int32_t>(a + e) : sid[e];
    if (LAST) {  // final order: the ids stay in L2 for the query phase, the keys only feed the starts
      st_l2(ids_out + dest, id, l2_policy_keep());
      st_l2(keys_out + dest, key, l2_policy_stream());
    } else {
      keys_out[dest] = key;
      ids_out[dest] = id;
    }
  }
}

size_t scatter_smem_bytes(bool first, int nb_pad) {
  return sizeof(uint32_t) * (kTile + (first ? 0 : kTile) + (2 * kSortWarps + 2) * static_cast<size_t>(nb_pad)) +
         sizeof(uint16_t) * kTile;
}

// Also lists the heavy buckets (more than R points) when heavy_count is set:
// the bucket kp ending at element i holds more than R points exactly when the
// element R + 1 places before i has the same address.  Indices are 32-bit
// (tables hold fewer than 2^24 points); each element is loaded once and its
// predecessor comes from the neighbouring lane.
__global__ void __launch_bounds__(256) bucket_starts_kernel(const uint32_t *skeys, int64_t n, uint32_t T,
                                                             uint32_t *starts, uint32_t R,
                                                             unsigned long long *heavy_count, uint64_t *heavy,
                                                             int64_t heavy_cap) {
  const uint32_t t = blockIdx.y;
  const uint32_t *seg = skeys + static_cast<int64_t>(t) * n;
  uint32_t *st = starts + static_cast<int64_t>(t) * (static_cast<int64_t>(T) + 1);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nn = static_cast<uint32_t>(n);
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint64_t keep = l2_policy_keep();
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base <= nn; base += stride) {
    const uint32_t i = base + lane;
    const uint32_t kc = i < nn ? seg[i] : T + 1;  // past the end: above every address
    uint32_t kp = __shfl_up_sync(kFull, kc, 1);
    if (lane == 0) kp = base > 0 ? seg[base - 1] : 0xFFFFFFFFu;  // none before the first element
    // buckets kp + 1 .. min(kc, T) start at i (kp + 1 wraps to 0 for the first element)
    uint32_t lo = 1, hi = 0;
    if (i <= nn) {
      lo = kp + 1;
      hi = kc < T ? kc : T;
      if (heavy_count && kp < T && kp < kc && i > R && seg[i - R - 1] == kp) {
        const unsigned long long h = atomicAdd(heavy_count, 1ULL);
        if (static_cast<int64_t>(h) < heavy_cap) heavy[h] = (static_cast<uint64_t>(t) << 32) | kp;
      }
    }
    // short gaps (the common case: about n / 2^rb addresses per bucket) by the thread itself
    if (lo <= hi && hi - lo < 8) {
      for (uint32_t bkt = lo; bkt <= hi; ++bkt) st_l2(st + bkt, i, keep);
      lo = 1;
      hi = 0;
    }
    uint32_t m = __ballot_sync(kFull, lo <= hi);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const uint32_t glo = __shfl_sync(kFull, lo, src), ghi = __shfl_sync(kFull, hi, src);
      const uint32_t gi = __shfl_sync(kFull, i, src);
      for (uint32_t bkt = glo + lane; bkt <= ghi; bkt += 32) st_l2(st + bkt, gi, keep);
    }
  }
}

}  // namespace

SortPlan make_sort_plan(uint32_t range_bits, int64_t n, uint32_t L) {
  SortPlan p{};
  p.passes = static_cast<int>((range_bits + 7) / 8);
  if (p.passes < 1) p.passes = 1;
  const int base = static_cast<int>(range_bits) / p.passes, extra = static_cast<int>(range_bits) % p.passes;
  int shift = 0, maxb = 0;
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
  return p;
}

int sort_tables(const SortPlan &plan, const SortLaunch &s, cudaStream_t stream) {
  const int64_t T = 1LL << s.range_bits;
  if (s.n == 0) {
    return cudaMemsetAsync(s.starts, 0, sizeof(uint32_t) * s.L * (T + 1), stream) == cudaSuccess ? 0 : FLASH_ECUDA;
  }
  const dim3 grid(static_cast<unsigned>(plan.tiles), s.L);
  const uint32_t *kin = s.keys_in;
  const int32_t *vin = nullptr;
  for (int pass = 0; pass < plan.passes; ++pass) {
    PassArgs pa{plan.shift[pass], plan.bits[pass], plan.nbins[pass], pass == plan.passes - 1};
    const bool to_final = ((plan.passes - 1 - pass) % 2) == 0;
    uint32_t *kout = to_final ? s.keys_out : s.tmp_keys;
    int32_t *vout = to_final ? s.ids_out : s.tmp_ids;
    radix_hist_kernel<<<grid, 256, 0, stream>>>(kin, s.n, pa, plan.tile, plan.tiles, s.hist);
    radix_scan_kernel<<<s.L, 1024, 0, stream>>>(s.hist, static_cast<int64_t>(pa.nbins) * plan.tiles);
    const int nb_pad = (pa.nbins + 3) & ~3;
    const size_t smem = scatter_smem_bytes(pass == 0, nb_pad);
    const bool last = pass == plan.passes - 1;
    auto kern = pass == 0 ? (last ? radix_scatter_kernel<true, true> : radix_scatter_kernel<true, false>)
                          : (last ? radix_scatter_kernel<false, true> : radix_scatter_kernel<false, false>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
      return FLASH_ECUDA;
    kern<<<grid, kSortWarps * 32, smem, stream>>>(kin, vin, s.n, pa, plan.tiles, s.hist, kout, vout, nb_pad);
    count_launches(3);
    kin = kout;
    vin = vout;
  }
  const int64_t blocks_x = (s.n + 1 + 255) / 256;
  const dim3 g2(static_cast<unsigned>(blocks_x < 1024 ? blocks_x : 1024), s.L);
  if (s.heavy_count && cudaMemsetAsync(s.heavy_count, 0, sizeof(unsigned long long), stream) != cudaSuccess)
    return FLASH_ECUDA;
  bucket_starts_kernel<<<g2, 256, 0, stream>>>(s.keys_out, s.n, static_cast<uint32_t>(T), s.starts, s.R,
                                               s.heavy_count, s.heavy, s.heavy_cap);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
