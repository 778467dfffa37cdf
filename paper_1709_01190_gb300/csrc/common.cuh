// common.cuh -- definitions shared by the CUDA translation units of libflash.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/flash.h"

namespace flash {

// ---------------------------------------------------------------- seeds
// The method draws five 64-bit words from the user seed: the first five
// outputs of SplitMix64 (Steele, Lea & Flood 2014) started from the seed,
// with the two multipliers forced odd.
//   a1, b1: one-permutation hash pi(i) = (a1*i + b1) >> 32  (Section 2.3)
//   a2, b2: universal map of a K-tuple to a bucket address    (Section 2.2)
//   r     : key of the reservoir decisions                     (Algorithm 1)
struct Seeds {
  uint64_t a1, b1, a2, b2, r, d;  // d: key of the optimal-densification probes
  uint64_t e;                     // key of the bucket -> reservoir map of reservoir sharing
};

__host__ __device__ inline uint64_t sm64_finalize(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

inline Seeds derive_seeds(uint64_t seed) {
  Seeds s;
  uint64_t w[7];
  for (int i = 0; i < 7; ++i) {
    seed += 0x9E3779B97F4A7C15ULL;
    w[i] = sm64_finalize(seed);
  }
  s.a1 = w[0] | 1ULL;
  s.b1 = w[1];
  s.a2 = w[2] | 1ULL;
  s.b2 = w[3];
  s.r = w[4];
  s.d = w[5];
  s.e = w[6];
  return s;
}

// Reservoir sharing (Section 3.5): the reservoir of the shared pool of P that
// bucket b of table t points to, ((F(e ^ (t * 2^32 + b)) >> 32) * P) >> 32
// with F SplitMix64's output function.
__host__ __device__ inline uint32_t pool_index(uint64_t e, uint32_t t, uint32_t b, uint32_t P) {
  const uint64_t u = sm64_finalize(e ^ ((static_cast<uint64_t>(t) << 32) + b));
  return static_cast<uint32_t>(((u >> 32) * P) >> 32);
}
// "Table" of the reservoir draws of a shared pool (no real table uses it).
constexpr uint32_t kPoolTable = 0xFFFFFFFFu;

// log2 of the smallest power of two >= P (at least 1).
inline uint32_t pool_bits_of(uint32_t P) {
  uint32_t b = 1;
  while (b < 31 && (1u << b) < P) ++b;
  return b;
}

// Constant added per step of rotation densification (2^32 / golden ratio).
constexpr uint32_t kRotStep = 0x9E3779B9u;
// Hash of every bin of a row without entries.
constexpr uint32_t kEmptyHash = 0xFFFFFFFFu;

// Implementation limits (checked on the host before any launch).
constexpr uint32_t kMaxBins = 4096;        // K*L
constexpr uint32_t kMaxRangeBits = 30;
constexpr uint32_t kMaxCandidates = 16384; // L*R
constexpr uint32_t kMaxTablesPacked = 256; // count-1 fits 8 bits
constexpr int64_t kMaxPointsPacked = (1LL << 24) - 2;

// -------------------------------------------------------- device errors
// Sticky error bits (FLASH_DEVERR_*), one word per device.
uint32_t *device_error_word();  // library-owned, allocated on first use

__device__ __forceinline__ void raise_error(uint32_t *err, uint32_t bit) {
  if (err) atomicOr(err, bit);
}

// Reservoir random number for arrival rank i of bucket b in table t
// (Algorithms 1 and 2: j = RANDOM([0, i])): a counter-based draw
//   u = F(F(r ^ (t*2^32 + b)) ^ i),  F = SplitMix64's output function,
//   j = ((u >> 32) * (i + 1)) >> 32.
// `bucket_key` is the inner F(r ^ (t*2^32 + b)), computed once per bucket.
__device__ __forceinline__ uint64_t reservoir_bucket_key(uint64_t r, uint32_t t, uint32_t b) {
  return sm64_finalize(r ^ ((static_cast<uint64_t>(t) << 32) + b));
}
__device__ __forceinline__ uint32_t reservoir_draw(uint64_t bucket_key, uint32_t i) {
  uint64_t u = sm64_finalize(bucket_key ^ static_cast<uint64_t>(i));
  return static_cast<uint32_t>(((u >> 32) * (static_cast<uint64_t>(i) + 1ULL)) >> 32);
}

// ------------------------------------------------ L2 eviction priorities
// Per-access hints (no device setting changes): data that a later phase reads
// at random (bucket starts, grouped ids) is kept with evict_last; streams read
// or written once go with evict_first.
// The policies and the loads are pure (no volatile): the compiler may hoist,
// share and schedule them like ordinary loads of data that no kernel writes
// while it runs.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_stream() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_l2(const uint32_t *ptr, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ int32_t ld_l2(const int32_t *ptr, uint64_t pol) {
  int32_t v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
  return v;
}
// Stores of results the writing kernel never reads back: no memory clobber,
// so loads and shared-memory work around them stay schedulable.
__device__ __forceinline__ void st_l2(uint32_t *ptr, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(ptr), "r"(v), "l"(pol));
}
__device__ __forceinline__ void st_l2(int32_t *ptr, int32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(ptr), "r"(v), "l"(pol));
}

inline unsigned div_up(uint64_t a, uint64_t b) { return static_cast<unsigned>((a + b - 1) / b); }

int num_sms();

}  // namespace flash
