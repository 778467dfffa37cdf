// reservoir.cu -- K3: reservoir sampling of every bucket (Algorithm 1 inside
// the ADD of Algorithm 2), done after grouping instead of point by point.
//
// After the stable sort, bucket b of table t is the segment
// ids[t][starts[b] .. starts[b+1]) holding its m arrivals in arrival order.
// Sequential reservoir sampling with fill-first leaves in slot s the LAST
// arrival that wrote it: arrival i < R writes slot i; arrival i >= R writes
// slot j_i = RANDOM([0, i]) when j_i < R.  Every j_i is a counter-based
// function of (seed, t, b, i), so the final slot contents are
//   slot s = arrival max({s} U {i >= R : j_i = s}),
// an order-free max reduction.  Buckets with m <= R are already final.  For
// m > R, one block per bucket draws all j_i in parallel, reduces with
// shared-memory atomicMax, and rewrites slots 0..R-1 of the segment in
// place (it only reads positions >= R and only writes positions < R).
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kResThreads = 256;

__global__ void __launch_bounds__(256) heavy_buckets_kernel(const uint32_t *starts, uint32_t T, uint32_t L,
                                                             uint32_t R, unsigned long long *count, uint64_t *list,
                                                             int64_t cap) {
  const int64_t total = static_cast<int64_t>(L) * T;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t t = g / T, b = g - t * T;
    const uint32_t *st = starts + t * (static_cast<int64_t>(T) + 1);
    const uint32_t m = st[b + 1] - st[b];
    if (m > R) {
      const unsigned long long i = atomicAdd(count, 1ULL);
      if (static_cast<int64_t>(i) < cap) list[i] = (static_cast<uint64_t>(t) << 32) | static_cast<uint64_t>(b);
    }
  }
}

__global__ void __launch_bounds__(kResThreads) reservoir_select_kernel(int32_t *ids, const uint32_t *starts,
                                                                       int64_t n, uint32_t T, uint32_t R, uint64_t r,
                                                                       const unsigned long long *count,
                                                                       const uint64_t *list, int64_t cap, bool shared) {
  extern __shared__ uint32_t win[];
  const int64_t nheavy = min(static_cast<int64_t>(*count), cap);
  for (int64_t h = blockIdx.x; h < nheavy; h += gridDim.x) {
    const uint64_t tb = list[h];
    const uint32_t t = static_cast<uint32_t>(tb >> 32), b = static_cast<uint32_t>(tb);
    const uint32_t *st = starts + static_cast<int64_t>(t) * (static_cast<int64_t>(T) + 1);
    const uint32_t s = st[b], m = st[b + 1] - s;
    int32_t *seg = ids + static_cast<int64_t>(t) * n + s;
    for (uint32_t j = threadIdx.x; j < R; j += blockDim.x) win[j] = j;
    __syncthreads();
    const uint64_t bk = reservoir_bucket_key(r, shared ? kPoolTable : t, b);
    for (uint32_t i = R + threadIdx.x; i < m; i += blockDim.x) {
      const uint32_t j = reservoir_draw(bk, i);
      if (j < R) atomicMax(&win[j], i);
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < R; j += blockDim.x) {
      const uint32_t w = win[j];
      if (w != j) seg[j] = seg[w];
    }
    __syncthreads();
  }
}

// tables [L][nb][R], counts [L][nb] from starts [L][T + 1] (nb <= T buckets per table)
__global__ void __launch_bounds__(256) export_kernel(const int32_t *ids, const uint32_t *starts, int64_t n, uint32_t T,
                                                      uint32_t nb, uint32_t L, uint32_t R, int32_t *tables,
                                                      uint32_t *counts) {
  const int64_t total = static_cast<int64_t>(L) * nb * R;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t tb = g / R, j = g - tb * R;
    const int64_t t = tb / nb, b = tb - t * nb;
    const uint32_t *st = starts + t * (static_cast<int64_t>(T) + 1);
    const uint32_t s = st[b], m = st[b + 1] - s;
    tables[g] = j < m ? ids[t * n + s + j] : -1;
    if (j == 0) counts[tb] = m;
  }
}

}  // namespace

int64_t reservoir_heavy_capacity(int64_t n, uint32_t L, uint32_t R, uint32_t range_bits) {
  // a heavy bucket holds more than R of the table's n points
  const int64_t per_table_by_n = n / (static_cast<int64_t>(R) + 1);
  const int64_t per_table_by_t = 1LL << range_bits;
  const int64_t per = per_table_by_n < per_table_by_t ? per_table_by_n : per_table_by_t;
  return static_cast<int64_t>(L) * per + 1;
}

int launch_reservoir(const ReservoirLaunch &l, cudaStream_t stream) {
  const uint32_t T = 1u << l.range_bits;
  if (l.n == 0) return 0;
  if (!l.heavy_listed) {
    if (cudaMemsetAsync(l.heavy_count, 0, sizeof(unsigned long long), stream) != cudaSuccess) return FLASH_ECUDA;
    const int64_t total = static_cast<int64_t>(l.L) * T;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 16L * num_sms() * 8) blocks = 16L * num_sms() * 8;
    heavy_buckets_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(l.starts, T, l.L, l.R, l.heavy_count,
                                                                            l.heavy, l.heavy_cap);
    count_launches(1);
  }
  const size_t smem = sizeof(uint32_t) * l.R;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(reservoir_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return FLASH_ECUDA;
  reservoir_select_kernel<<<static_cast<unsigned>(num_sms() * 8), kResThreads, smem, stream>>>(
      l.ids, l.starts, l.n, T, l.R, l.r, l.heavy_count, l.heavy, l.heavy_cap, l.shared);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

int launch_export(const int32_t *ids, const uint32_t *starts, int64_t n, uint32_t L, uint32_t R, uint32_t range_bits,
                  uint32_t nb, int32_t *tables, uint32_t *counts, cudaStream_t stream) {
  const uint32_t T = 1u << range_bits;
  const int64_t total = static_cast<int64_t>(L) * nb * R;
  if (total == 0) return 0;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  export_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(ids, starts, n, T, nb, L, R, tables, counts);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

// A shared pool is sorted as one sequence of the L * n (point, table) arrivals in
// row-major order, so a sorted entry is an arrival's position p * L + t.
__global__ void __launch_bounds__(256) positions_to_ids_kernel(int32_t *ids, int64_t n, uint32_t L) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    ids[i] = static_cast<int32_t>(static_cast<uint32_t>(ids[i]) / L);
}

int launch_positions_to_ids(int32_t *ids, int64_t n, uint32_t L, cudaStream_t stream) {
  if (n == 0) return 0;
  positions_to_ids_kernel<<<static_cast<unsigned>(8 * num_sms()), 256, 0, stream>>>(ids, n, L);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
