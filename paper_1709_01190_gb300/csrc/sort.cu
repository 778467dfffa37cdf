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
//             warps keep the tile's element order -- and a scatter to
//             scan offset + rank.
// Finally the bucket starts: starts[t][b] = number of addresses < b in table
// t, for b in [0, 2^rb]; each key change writes the starts of the skipped
// buckets, a warp at a time.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kSortWarps = 8;
constexpr int kSortItems = 8;
constexpr int kMaxBinsSort = 257;
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

template <bool FIRST>
__global__ void __launch_bounds__(kSortWarps * 32) radix_scatter_kernel(const uint32_t *keys_in, const int32_t *ids_in,
                                                                       int64_t n, PassArgs p, uint32_t tile, int64_t tiles,
                                                                       const uint32_t *offs, uint32_t *keys_out,
                                                                       int32_t *ids_out) {
  __shared__ uint32_t run[kMaxBinsSort + 7];
  __shared__ uint32_t wcnt[kSortWarps][kMaxBinsSort + 7];
  __shared__ uint32_t wpref[kSortWarps][kMaxBinsSort + 7];
  const uint32_t t = blockIdx.y;
  const int64_t ti = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = static_cast<int64_t>(t) * n;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int d = threadIdx.x; d < p.nbins; d += blockDim.x)
    run[d] = offs[(static_cast<int64_t>(t) * p.nbins + d) * tiles + ti];
  const int64_t a = ti * tile, b = min(n, a + static_cast<int64_t>(tile));
  constexpr int kChunk = kSortWarps * 32 * kSortItems;
  for (int64_t cb = a; cb < b; cb += kChunk) {
    for (int d = lane; d < p.nbins; d += 32) wcnt[warp][d] = 0;
    __syncwarp();
    uint32_t kk[kSortItems], dd[kSortItems], rr[kSortItems];
    int32_t vv[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t e = cb + static_cast<int64_t>(warp) * 32 * kSortItems + r * 32 + lane;
      const bool valid = e < b;
      const uint32_t key = valid ? __ldcs(keys_in + seg + e) : 0u;
      const int32_t val = FIRST ? static_cast<int32_t>(e) : (valid ? __ldcs(ids_in + seg + e) : 0);
      const uint32_t d = valid ? digit_of(key, p) : 0xFFFFu;
      const uint32_t peers = __match_any_sync(kFull, d);
      const uint32_t lower = peers & lt_mask;
      const uint32_t before = valid ? wcnt[warp][d] : 0u;
      __syncwarp();
      if (valid && lower == 0) wcnt[warp][d] = before + __popc(peers);
      __syncwarp();
      kk[r] = key;
      vv[r] = val;
      dd[r] = d;
      rr[r] = before + __popc(lower);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < p.nbins; d += blockDim.x) {
      uint32_t acc = run[d];
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        wpref[w][d] = acc;
        acc += wcnt[w][d];
      }
      run[d] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      if (dd[r] != 0xFFFFu) {
        const int64_t dest = seg + wpref[warp][dd[r]] + rr[r];
        keys_out[dest] = kk[r];
        ids_out[dest] = vv[r];
      }
    }
  }
}

__global__ void __launch_bounds__(256) bucket_starts_kernel(const uint32_t *skeys, int64_t n, uint32_t T,
                                                             uint32_t *starts) {
  const uint32_t t = blockIdx.y;
  const uint32_t *seg = skeys + static_cast<int64_t>(t) * n;
  uint32_t *st = starts + static_cast<int64_t>(t) * (static_cast<int64_t>(T) + 1);
  const int lane = threadIdx.x & 31;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base <= n;
       base += stride) {
    const int64_t i = base + lane;
    int64_t lo = 1, hi = 0;
    if (i <= n) {
      const int64_t kp = i > 0 ? static_cast<int64_t>(seg[i - 1]) : -1;
      const int64_t kc = i < n ? static_cast<int64_t>(seg[i]) : static_cast<int64_t>(T) + 1;
      lo = kp + 1;
      hi = kc < static_cast<int64_t>(T) ? kc : static_cast<int64_t>(T);
    }
    uint32_t m = __ballot_sync(kFull, lo <= hi);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int64_t glo = __shfl_sync(kFull, lo, src), ghi = __shfl_sync(kFull, hi, src);
      const uint32_t gi = static_cast<uint32_t>(__shfl_sync(kFull, i, src));
      for (int64_t bkt = glo + lane; bkt <= ghi; bkt += 32) st[bkt] = gi;
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
  p.tile = n >= (4LL << 20) ? 16384u : 8192u;
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
    if (pass == 0)
      radix_scatter_kernel<true><<<grid, kSortWarps * 32, 0, stream>>>(kin, vin, s.n, pa, plan.tile, plan.tiles,
                                                                       s.hist, kout, vout);
    else
      radix_scatter_kernel<false><<<grid, kSortWarps * 32, 0, stream>>>(kin, vin, s.n, pa, plan.tile, plan.tiles,
                                                                        s.hist, kout, vout);
    count_launches(3);
    kin = kout;
    vin = vout;
  }
  const int64_t blocks_x = (s.n + 1 + 255) / 256;
  const dim3 g2(static_cast<unsigned>(blocks_x < 1024 ? blocks_x : 1024), s.L);
  bucket_starts_kernel<<<g2, 256, 0, stream>>>(s.keys_out, s.n, static_cast<uint32_t>(T), s.starts);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
