// add.cu -- ADD of Algorithm 2 continued on an existing index: a batch of
// new points (ids n, n + 1, ...) arrives after the indexed ones.
//
// Algorithm 2 is a stream: in every bucket the new points continue the
// arrival ranks from the bucket's stored count m_old, so after the batch the
// tables equal those of one build over old and new points together.  On the
// grouped layout (ids [L][n] by bucket, reservoir = first min(m, R) ids of a
// segment, segment length = m) that is:
//   merge : bucket b's new segment is its old segment (the reservoir state
//           after m_old arrivals, then the arrivals that were not kept)
//           followed by the batch's points of b in id order (grouped by the
//           same stable sort as a build); its new start is the sum of the old
//           start and the batch's start, both prefix sums over buckets;
//   draws : arrival i (m_old <= i < m_old + m_new) sits at position i of the
//           merged segment.  For i < R it fills slot i (already in place);
//           for i >= max(R, m_old) it draws j = RANDOM([0, i]) (the same
//           counter-based draw as a build) and slot j ends with the LAST such
//           arrival that drew it: a max reduction, as in the reservoir step of
//           a build, reading positions >= R and writing positions < R.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kAddThreads = 256;

// One thread per segment (t, b), b in [0, 2^rb] (b = 2^rb: the points never
// inserted, rows without entries): the merged segment and its start; buckets
// whose merged count needs draws are listed (t << 32 | b).
__global__ void __launch_bounds__(kAddThreads) add_merge_kernel(AddLaunch a) {
  const uint32_t T = 1u << a.range_bits;
  const int64_t total = static_cast<int64_t>(a.L) * (T + 1);
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t t = static_cast<uint32_t>(g / (T + 1)), b = static_cast<uint32_t>(g % (T + 1));
    const int64_t to = static_cast<int64_t>(t) * (T + 1);
    const uint32_t os = a.old_starts[to + b], ns = a.new_starts[to + b];
    const uint32_t oe = b < T ? a.old_starts[to + b + 1] : static_cast<uint32_t>(a.n_old);
    const uint32_t ne = b < T ? a.new_starts[to + b + 1] : static_cast<uint32_t>(a.n_new);
    const uint32_t m_old = oe - os, m_new = ne - ns, start = os + ns;
    a.starts[to + b] = start;
    const int32_t *src_o = a.old_ids + static_cast<int64_t>(t) * a.n_old + os;
    const int32_t *src_n = a.new_ids + static_cast<int64_t>(t) * a.n_new + ns;
    int32_t *dst = a.ids + static_cast<int64_t>(t) * (a.n_old + a.n_new) + start;
    for (uint32_t i = 0; i < m_old; ++i) dst[i] = src_o[i];
    for (uint32_t i = 0; i < m_new; ++i) dst[m_old + i] = src_n[i] + a.id0;
    const uint32_t m = m_old + m_new;
    const uint32_t first_draw = m_old > a.R ? m_old : a.R;
    if (b < T && m_new > 0 && m > first_draw) {
      const unsigned long long h = atomicAdd(a.heavy_count, 1ULL);
      if (static_cast<int64_t>(h) < a.heavy_cap) a.heavy[h] = (static_cast<uint64_t>(t) << 32) | b;
    }
  }
}

// One block per listed bucket: the draws of arrivals max(R, m_old) .. m - 1.
__global__ void __launch_bounds__(kAddThreads) add_reservoir_kernel(AddLaunch a) {
  extern __shared__ uint32_t win[];  // [R]: 1 + the last arrival that drew the slot, 0 = none
  const uint32_t T = 1u << a.range_bits;
  const int64_t n = a.n_old + a.n_new;
  const int64_t nheavy = min(static_cast<int64_t>(*a.heavy_count), a.heavy_cap);
  for (int64_t h = blockIdx.x; h < nheavy; h += gridDim.x) {
    const uint64_t tb = a.heavy[h];
    const uint32_t t = static_cast<uint32_t>(tb >> 32), b = static_cast<uint32_t>(tb);
    const int64_t to = static_cast<int64_t>(t) * (T + 1);
    const uint32_t s = a.starts[to + b], m = a.starts[to + b + 1] - s;
    const uint32_t m_old = a.old_starts[to + b + 1] - a.old_starts[to + b];
    const uint32_t first = m_old > a.R ? m_old : a.R;
    int32_t *seg = a.ids + static_cast<int64_t>(t) * n + s;
    for (uint32_t j = threadIdx.x; j < a.R; j += blockDim.x) win[j] = 0;
    __syncthreads();
    const uint64_t bk = reservoir_bucket_key(a.rkey, t, b);
    for (uint32_t i = first + threadIdx.x; i < m; i += blockDim.x) {
      const uint32_t j = reservoir_draw(bk, i);
      if (j < a.R) atomicMax(&win[j], i + 1u);
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < a.R; j += blockDim.x) {
      const uint32_t w = win[j];
      if (w) seg[j] = seg[w - 1u];
    }
    __syncthreads();
  }
}

}  // namespace

int launch_add(const AddLaunch &a, cudaStream_t stream) {
  if (cudaMemsetAsync(a.heavy_count, 0, sizeof(unsigned long long), stream) != cudaSuccess) return FLASH_ECUDA;
  add_merge_kernel<<<static_cast<unsigned>(8 * num_sms()), kAddThreads, 0, stream>>>(a);
  const size_t smem = sizeof(uint32_t) * a.R;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(add_reservoir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return FLASH_ECUDA;
  add_reservoir_kernel<<<static_cast<unsigned>(8 * num_sms()), kAddThreads, smem, stream>>>(a);
  count_launches(2);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
