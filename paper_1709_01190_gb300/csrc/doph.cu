// doph.cu -- K1: densified one-permutation hashing (Section 2.3, on the
// minwise hash of Eq. 1) of CSR rows, with MapKHashesToAddress (Section 2.2,
// Algorithm 2) fused as an optional epilogue.
//
// One warp hashes one row at a time; rows are handed out dynamically in
// small groups from a global counter, so very uneven row lengths balance.
// Per warp, shared memory holds the row's B = K*L bins and a bitmap of the
// non-empty bins.  The insertion paths give identical results:
//   dense rows  (nnz > B/2, B even): bins start at 0xFFFFFFFF; non-zeros are
//       read as 16-byte vectors, the next 512 of a row prefetched while the
//       current 512 are hashed, each by one shared-memory min reduction
//       (off = pi*B mod 2^32 is even, never all ones, so a bin is non-empty
//       exactly when it is below 0xFFFFFFFF); the columns are range-checked
//       once per row through a running maximum, and a row holding a column
//       out of range is redone element by element; rows with every bin
//       filled skip the bitmap and the densification;
//   element by element (odd B, or the redo): also marks bins whose minimum is
//       all ones, and skips (and flags) columns out of range;
//   sparse rows (nnz <= B/2): 32 non-zeros per round; a bin is set to all
//       ones when the row first touches it (bitmap bit clear), then every lane
//       takes a shared-memory min into its bin and sets the bit, so the row
//       never clears all B bins.
// Densification (rotation): word by word, lane l takes bin 32w + l; an empty
// bin j becomes v[src] + (src - j) * 0x9E3779B9, src the first non-empty bin
// after j, circularly (found from the word bitmap and a ballot summary of the
// non-empty words).  Optimal densification ([36]): an empty bin copies the
// first non-empty bin of its own probe sequence (a SplitMix64 mix of (bin,
// attempt)).
// Emit: the B hashes (coalesced, 16-byte stores when aligned) or the L keys.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace flash {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct DophParams {
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t n_rows, nnz;
  uint32_t dim_u32;  // dim clipped to 2^32-1 (columns are int32)
  uint32_t B, K, L, rb, W, G;  // W = bitmap words, G = summary words
  uint32_t densify;            // 0 rotation, 1 optimal densification
  uint32_t pool, pool_bits;    // keys mode, reservoir sharing: reservoir of each key; sentinel 2^pool_bits
  uint32_t rows_per_grab;
  uint32_t bin_words;  // W * 33 rounded up to a multiple of 4 (room for either layout)
  uint32_t smem_words_per_warp;
  Seeds s;
  uint32_t *out;      // hashes [n][B], or keys [L][ld] (may be null in keys mode)
  uint32_t *out_rm;   // keys mode: optional row-major copy [n][L]
  int64_t ld;  // keys: leading dimension (>= n_rows)
  bool vec_out;
  uint32_t *err;
  unsigned long long *row_counter;
  const int32_t *order;  // optional processing order of the rows (longest first)
  const int32_t *long_rows;    // optional: long rows, hashed first
  const uint32_t *long_count;  // their number (device)
  int64_t long_min;            // non-zeros of a long row
};

// Shared-memory position of bin j.  Sparse rows keep one pad word after every
// 32 bins, so that lane l walking bins 32 l .. 32 l + 31 (the densification)
// and lanes reading consecutive bins both hit 32 different banks; dense rows
// keep the bins unpadded (their insertion loop is the kernel's hot loop).
template <bool PAD>
__device__ __forceinline__ uint32_t bix(uint32_t j) {
  return PAD ? j + (j >> 5) : j;
}

__device__ __forceinline__ void bin_and_offset(uint32_t c, const Seeds &s, uint32_t B, uint32_t &bin,
                                               uint32_t &off) {
  // pi(c) = (a1*c + b1 mod 2^64) >> 32, then split the permuted range into B bins
  uint64_t x = s.a1 * static_cast<uint64_t>(c) + s.b1;
  uint32_t pi = static_cast<uint32_t>(x >> 32);
  uint64_t p = static_cast<uint64_t>(pi) * B;
  bin = static_cast<uint32_t>(p >> 32);
  off = static_cast<uint32_t>(p);
}

__device__ __forceinline__ void insert_dense(uint32_t c, const DophParams &a, uint32_t *bins, uint32_t *mask) {
  if (c >= a.dim_u32) {
    raise_error(a.err, FLASH_DEVERR_COL_RANGE);
    return;
  }
  uint32_t bin, off;
  bin_and_offset(c, a.s, a.B, bin, off);
  // bins only decrease, so a stale read is never smaller than the truth
  if (off <= *reinterpret_cast<volatile uint32_t *>(&bins[bin])) {
    atomicMin(&bins[bin], off);
    if (off == 0xFFFFFFFFu) atomicOr(&mask[bin >> 5], 1u << (bin & 31));  // non-empty, minimum all ones
  }
}

// Element-by-element insertion (odd B, or a row holding a column out of
// range): also records non-zeros whose offset is all ones, and skips (and
// flags) columns out of range.
__device__ __noinline__ void insert_row_checked(const DophParams &a, int64_t start, int64_t end, uint32_t *bins,
                                                uint32_t *mask, uint32_t lane) {
  for (uint32_t j = lane; j < a.W * 32; j += 32) bins[j] = 0xFFFFFFFFu;
  for (uint32_t w = lane; w < a.W; w += 32) mask[w] = 0;
  __syncwarp();
  for (int64_t e = start + lane; e < end; e += 32) insert_dense(static_cast<uint32_t>(a.col[e]), a, bins, mask);
  __syncwarp();
}

// One non-zero of a dense row (B even, column checked later for the whole
// row): pi = ((a1_lo*c + b1) >> 32) + a1_hi*c; (bin, off) = (hi, lo) of pi*B.
// For even B, off = pi*B mod 2^32 is even and never all ones, so a bin is
// non-empty exactly when its value is below 0xFFFFFFFF.
__device__ __forceinline__ void insert_fast(uint32_t c, uint32_t a1_lo, uint32_t a1_hi, uint64_t b1, uint32_t B,
                                            uint32_t *bins) {
  const uint64_t t = static_cast<uint64_t>(a1_lo) * c + b1;
  const uint32_t pi = static_cast<uint32_t>(t >> 32) + a1_hi * c;
  const uint64_t pb = static_cast<uint64_t>(pi) * B;
  atomicMin(&bins[static_cast<uint32_t>(pb >> 32)], static_cast<uint32_t>(pb));  // result unused: red.shared.min
}

// Eight non-zeros of a dense row; mx collects the largest column for the
// row's range check.
__device__ __forceinline__ void insert8(const int4 &x, const int4 &y, uint32_t a1_lo, uint32_t a1_hi, uint64_t b1,
                                        uint32_t B, uint32_t *bins, uint32_t &mx) {
  const uint32_t c[8] = {static_cast<uint32_t>(x.x), static_cast<uint32_t>(x.y), static_cast<uint32_t>(x.z),
                         static_cast<uint32_t>(x.w), static_cast<uint32_t>(y.x), static_cast<uint32_t>(y.y),
                         static_cast<uint32_t>(y.z), static_cast<uint32_t>(y.w)};
  mx = __vimax3_u32(mx, __vimax3_u32(c[0], c[1], c[2]), __vimax3_u32(c[3], c[4], c[5]));
  mx = __vimax3_u32(mx, c[6], c[7]);
#pragma unroll
  for (int i = 0; i < 8; ++i) insert_fast(c[i], a1_lo, a1_hi, b1, B, bins);
}

// Four non-zeros (the partial last group, one 16-byte part at a time).
__device__ __forceinline__ void insert4(const int4 &x, uint32_t a1_lo, uint32_t a1_hi, uint64_t b1, uint32_t B,
                                        uint32_t *bins, uint32_t &mx) {
  const uint32_t c[4] = {static_cast<uint32_t>(x.x), static_cast<uint32_t>(x.y), static_cast<uint32_t>(x.z),
                         static_cast<uint32_t>(x.w)};
  mx = __vimax3_u32(mx, __vimax3_u32(c[0], c[1], c[2]), c[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) insert_fast(c[i], a1_lo, a1_hi, b1, B, bins);
}

// first set bit index >= from in the summary bitmap (G words), circular over W bits
__device__ __forceinline__ int next_word_circular(const uint32_t (&sw)[4], uint32_t G, uint32_t from) {
#pragma unroll
  for (uint32_t g = 0; g < 4; ++g) {
    if (g < G && g >= (from >> 5)) {
      uint32_t m = sw[g];
      if (g == (from >> 5)) m &= (~0u << (from & 31));
      if (m) return static_cast<int>(32 * g + __ffs(m) - 1);
    }
  }
#pragma unroll
  for (uint32_t g = 0; g < 4; ++g) {
    if (g < G && sw[g]) return static_cast<int>(32 * g + __ffs(sw[g]) - 1);
  }
  return -1;
}

// The L table addresses (keys) or the B hashes of row r, all empty (the row
// has no non-zero, or none in range): keys 2^rb, hashes all ones.
template <bool KEYS>
__device__ __forceinline__ void emit_empty(const DophParams &a, int64_t r, uint32_t lane) {
  if (KEYS) {
    const uint32_t T = static_cast<uint32_t>(1ULL << (a.pool ? a.pool_bits : a.rb));
    for (uint32_t t = lane; t < a.L; t += 32) {
      if (a.out) a.out[static_cast<int64_t>(t) * a.ld + r] = T;
      if (a.out_rm) a.out_rm[r * a.L + t] = T;
    }
  } else {
    for (uint32_t j = lane; j < a.B; j += 32) a.out[r * a.B + j] = kEmptyHash;
  }
}

// Sparse row (n <= B/2): 32 non-zeros per round.  A bin is opened at all ones
// by the lanes that touch it first in the row (its bitmap bit still clear),
// then every lane takes the min into it and sets the bit; only bins with the
// bit set are read later, so the row never clears all B bins.
__device__ __forceinline__ void sparse_row(const DophParams &a, int64_t start, int64_t end, uint32_t *bins,
                                           uint32_t *mask, uint32_t lane) {
  for (uint32_t w = lane; w < a.W; w += 32) mask[w] = 0;
  __syncwarp();
  for (int64_t base = start; base < end; base += 32) {
    const int64_t e = base + lane;
    bool valid = e < end;
    uint32_t c = valid ? static_cast<uint32_t>(a.col[e]) : 0u;
    if (valid && c >= a.dim_u32) {
      raise_error(a.err, FLASH_DEVERR_COL_RANGE);
      valid = false;
    }
    uint32_t bin = 0, off = 0;
    if (valid) bin_and_offset(c, a.s, a.B, bin, off);
    const uint32_t bit = 1u << (bin & 31);
    if (valid && !(mask[bin >> 5] & bit)) bins[bix<true>(bin)] = 0xFFFFFFFFu;
    __syncwarp();
    if (valid) {
      atomicMin(&bins[bix<true>(bin)], off);
      atomicOr(&mask[bin >> 5], bit);
    }
    __syncwarp();
  }
}

// Dense row, after its non-zeros are reduced: the bitmap of non-empty bins.
__device__ __forceinline__ void dense_mask(const DophParams &a, const uint32_t *bins, uint32_t *mask,
                                           uint32_t lane) {
  __syncwarp();
  for (uint32_t w = 0; w < a.W; ++w) {
    const uint32_t j = w * 32 + lane;
    const bool ne = j < a.B && bins[j] != 0xFFFFFFFFu;
    const uint32_t m = __ballot_sync(kFull, ne);
    if (lane == 0) mask[w] |= m;
  }
  __syncwarp();
}

// The L keys of row r from its B final bins (MapKHashesToAddress), with the
// number of hashes per table fixed at compile time (KC > 0: the Horner fold
// unrolls) or read from the arguments (KC = 0).
template <int KC, bool PAD>
__device__ __forceinline__ void emit_keys(const DophParams &a, int64_t r, const uint32_t *bins, uint32_t lane) {
  const uint32_t K = KC > 0 ? static_cast<uint32_t>(KC) : a.K;
  const int sh = 64 - static_cast<int>(a.rb);
  const uint64_t a2 = a.s.a2, b2 = a.s.b2;
  for (uint32_t t = lane; t < a.L; t += 32) {
    uint64_t x = 0;
#pragma unroll
    for (uint32_t i = 0; i < K; ++i) x = x * a2 + bins[bix<PAD>(t + i * a.L)];
    uint32_t key = static_cast<uint32_t>((a2 * x + b2) >> sh);
    if (a.pool) key = pool_index(a.s.e, t, key, a.pool);  // the shared reservoir the bucket points to
    if (a.out) a.out[static_cast<int64_t>(t) * a.ld + r] = key;
    if (a.out_rm) a.out_rm[r * a.L + t] = key;
  }
}

// The emit of row r from its B final bins: the L keys or the B hashes.
template <bool KEYS, bool PAD>
__device__ __forceinline__ void emit_row(const DophParams &a, int64_t r, const uint32_t *bins, uint32_t lane) {
  const uint32_t B = a.B;
  if (KEYS) {
    switch (a.K) {
      case 4: emit_keys<4, PAD>(a, r, bins, lane); break;
      case 3: emit_keys<3, PAD>(a, r, bins, lane); break;
      case 2: emit_keys<2, PAD>(a, r, bins, lane); break;
      case 1: emit_keys<1, PAD>(a, r, bins, lane); break;
      default: emit_keys<0, PAD>(a, r, bins, lane); break;
    }
  } else if (a.vec_out && !PAD) {
    uint4 *o = reinterpret_cast<uint4 *>(a.out + r * B);
    const uint4 *src = reinterpret_cast<const uint4 *>(bins);
    for (uint32_t q4 = lane; q4 < B / 4; q4 += 32) __stcs(o + q4, src[q4]);
  } else if (a.vec_out) {
    uint4 *o = reinterpret_cast<uint4 *>(a.out + r * B);
    for (uint32_t q4 = lane; q4 < B / 4; q4 += 32) {
      const uint32_t j = 4 * q4;
      __stcs(o + q4, make_uint4(bins[bix<true>(j)], bins[bix<true>(j + 1)], bins[bix<true>(j + 2)],
                                bins[bix<true>(j + 3)]));
    }
  } else {
    for (uint32_t j = lane; j < B; j += 32) a.out[r * B + j] = bins[bix<PAD>(j)];
  }
  __syncwarp();
}

// Optimal densification ([36], cited in Section 2.3): an empty bin j probes
// bins src_i = ((mix(d ^ (j * 2^32 + i)) >> 32) * B) >> 32, i = 1 .. 8B (mix =
// SplitMix64's output function), and copies the first non-empty one; after 8B
// misses it copies the first non-empty bin to its right, circularly.  Each
// lane searches one empty bin at a time, four probes a step; a lane whose
// search ends takes the next unassigned bin of the row (a warp-uniform counter,
// positions from a ballot), so the warp runs for about the row's total probes
// over 32 lanes, not for the longest search of every round of 32 bins
// (searches are geometric with mean B / non-empty bins, and the longest of 32
// is several times the mean).  Only empty bins are written and only non-empty
// ones read.
__device__ __forceinline__ bool bin_filled(const uint32_t *mask, uint32_t b) { return (mask[b >> 5] >> (b & 31)) & 1u; }

template <bool PAD>
__device__ __noinline__ void optimal_densify(uint32_t *bins, const uint32_t *mask, uint32_t B, uint64_t d,
                                             uint32_t lane) {
  const uint32_t imax = 8u * B;  // a multiple of 4
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t next = 0;  // warp-uniform: the first bin not yet assigned
  uint32_t j = B;     // this lane's bin (B: none)
  uint32_t i = 1;
  uint64_t key = 0;
  bool want = true;  // this lane needs a bin
  for (;;) {
    // hand out bins until every lane that needs one holds an empty bin or the row is done
    while (__any_sync(kFull, want)) {
      const uint32_t req = __ballot_sync(kFull, want);
      if (want) j = next + __popc(req & lt);
      next += __popc(req);
      want = want && j < B && bin_filled(mask, j);
      if (j >= B) j = B;
    }
    if (!__any_sync(kFull, j < B)) break;
    if (j < B) {
      if (i == 1) key = d ^ (static_cast<uint64_t>(j) << 32);  // d ^ (j * 2^32 + i) = key ^ i for i < 2^32
      uint32_t src = 0xFFFFFFFFu;
      uint32_t pr[4];
      bool hit[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t u = sm64_finalize(key ^ static_cast<uint64_t>(i + q));
        pr[q] = static_cast<uint32_t>(((u >> 32) * B) >> 32);
        hit[q] = bin_filled(mask, pr[q]);
      }
#pragma unroll
      for (int q = 3; q >= 0; --q)  // the earliest hit of the four wins
        if (hit[q]) src = pr[q];
      i += 4;
      if (src == 0xFFFFFFFFu && i > imax) {  // the next non-empty bin to the right, circularly (one exists)
        src = j;
        for (uint32_t t = 1; t <= B; ++t) {
          const uint32_t b = j + t < B ? j + t : j + t - B;
          if (bin_filled(mask, b)) {
            src = b;
            break;
          }
        }
      }
      if (src != 0xFFFFFFFFu) {
        bins[bix<PAD>(j)] = bins[bix<PAD>(src)];
        j = B;
        i = 1;
        want = true;
      }
    }
  }
  __syncwarp();
}

// Densification by rotation and the emit of row r (keys or hashes).
template <bool KEYS, bool PAD>
__device__ __forceinline__ void finish_row(const DophParams &a, int64_t r, uint32_t *bins, const uint32_t *mask,
                                           uint32_t lane) {
  const uint32_t B = a.B, W = a.W;
  uint32_t sw[4] = {0, 0, 0, 0};
  uint32_t filled = 0;
#pragma unroll
  for (uint32_t g = 0; g < 4; ++g) {
    const uint32_t w = 32 * g + lane;
    const uint32_t m = (g < a.G && w < W) ? mask[w] : 0u;
    filled += __popc(m);
    sw[g] = __ballot_sync(kFull, m != 0);
  }
  filled = __reduce_add_sync(kFull, filled);
  if (filled == 0) {  // every column was out of range (flagged): hash as an empty row
    emit_empty<KEYS>(a, r, lane);
    __syncwarp();
    return;
  }
  if (filled < B && a.densify) {
    optimal_densify<PAD>(bins, mask, a.B, a.s.d, lane);
  } else if (filled < B && PAD) {
    // lane l walks its words l, l + 32, ... from the top bit down, carrying the
    // nearest filled bin to the right (the first one of the next non-empty word
    // at the start, B further when that is a wrap-around); an empty bin j gets
    // v[src] + (src - j) * C.  With the padded layout, the 32 lanes' bins
    // 32 l + b lie in 32 different banks.  Only empty bins are written and
    // only filled ones read.
    for (uint32_t w = lane; w < W; w += 32) {
      const uint32_t m = mask[w];
      if (m == 0xFFFFFFFFu) continue;
      const int w2 = next_word_circular(sw, a.G, w + 1 < W ? w + 1 : 0);
      const uint32_t m2 = mask[w2];
      const uint32_t s2 = 32u * static_cast<uint32_t>(w2) + (__ffs(m2) - 1);
      const uint32_t cur = s2 + (static_cast<uint32_t>(w2) <= w ? B : 0u);  // wrapped: distance counts B
      const uint32_t j0 = 32u * w;
      // v = the value of bin j + 1 on the way down: an empty bin j takes v + C
      // (= v[src] + (src - j) * C), a filled one its own value
      uint32_t v = bins[bix<true>(s2)] + (cur - (j0 + 32u)) * kRotStep;
#pragma unroll
      for (int b = 31; b >= 0; --b) {
        const uint32_t j = j0 + b;
        if ((m >> b) & 1u) {
          v = bins[bix<true>(j)];
        } else {
          v += kRotStep;
          bins[bix<true>(j)] = v;  // bins past B (last word) are never read
        }
      }
    }
    __syncwarp();
  } else if (filled < B) {
    // word by word, lane l takes bin 32w + l: the words and the next non-empty
    // word are warp-uniform (broadcast reads), bins are consecutive per lane
    // (no bank conflicts).  An empty bin j copies the first non-empty bin
    // after it, circularly: v[j] = v[src] + (src - j) * C, src past B when
    // it wrapped.  Only empty bins are written and only non-empty ones read.
    for (uint32_t w = 0; w < W; ++w) {
      const uint32_t m = mask[w];
      if (m == 0xFFFFFFFFu) continue;
      const uint32_t j = 32u * w + lane;
      const int w2 = next_word_circular(sw, a.G, w + 1);
      const uint32_t m2 = mask[w2];
      if (j < B && !((m >> lane) & 1u)) {
        const uint32_t hi = lane == 31 ? 0u : (m >> (lane + 1)) << (lane + 1);
        const uint32_t src = hi ? 32u * w + (__ffs(hi) - 1) : 32u * static_cast<uint32_t>(w2) + (__ffs(m2) - 1);
        const uint32_t virt = src > j ? src : src + B;  // wrapped: distance counts B
        bins[j] = bins[src] + (virt - j) * kRotStep;
      }
    }
    __syncwarp();
  }
  emit_row<KEYS, PAD>(a, r, bins, lane);
}

// The 16-byte aligned body [a4, a4 + 4 nq) of the row [start, end), from the
// actual address of col (4-byte aligned, checked on the host): element e is
// aligned when (e + mis) % 4 == 0.
__device__ __forceinline__ void row_body(int64_t start, int64_t end, int64_t mis, int64_t &a4, int64_t &nq) {
  a4 = min(((start + mis + 3) & ~static_cast<int64_t>(3)) - mis, end);
  const int64_t b4 = max(a4, ((end + mis) & ~static_cast<int64_t>(3)) - mis);
  nq = (b4 - a4) >> 2;
}

// Four blocks (32 warps) per SM: the loop is latency-bound, and 32 warps beat
// 24 with more registers (measured; five blocks spill).
template <bool KEYS>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4) doph_kernel(DophParams a) {
  extern __shared__ uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  uint32_t *bins = smem + warp * a.smem_words_per_warp;
  uint32_t *mask = bins + a.bin_words;
  const uint32_t B = a.B, W = a.W;
  const uint32_t a1_lo = static_cast<uint32_t>(a.s.a1), a1_hi = static_cast<uint32_t>(a.s.a1 >> 32);
  const uint64_t b1 = a.s.b1;
  const uint32_t dim = a.dim_u32;
  const int4 zero = make_int4(0, 0, 0, 0);
  const int64_t G = a.rows_per_grab;
  const int64_t mis = static_cast<int64_t>((reinterpret_cast<uintptr_t>(a.col) >> 2) & 3u);

  // Rows are claimed G at a time from a global counter; each row's bounds are
  // read when the row starts (the 16-byte groups of the row are prefetched
  // one group ahead).  With a list of long rows, positions [0, nl) are those
  // rows and positions nl + r are the rows in index order, long ones skipped:
  // a long row claimed late would outlast the rest of the launch.
  const int64_t nl = a.long_rows ? static_cast<int64_t>(*a.long_count) : 0;
  const int64_t total = nl + a.n_rows;
  int64_t cpos = 0, cend = 0;
  for (;;) {
    if (cpos >= cend) {
      unsigned long long s0 = 0;
      if (lane == 0) s0 = atomicAdd(a.row_counter, static_cast<unsigned long long>(G));
      s0 = __shfl_sync(kFull, s0, 0);
      if (s0 >= static_cast<unsigned long long>(total)) break;
      cpos = static_cast<int64_t>(s0);
      cend = min(cpos + G, total);
    }
    const int64_t pos = cpos++;
    const bool listed = pos < nl;
    const int64_t r = listed ? static_cast<int64_t>(a.long_rows[pos])
                             : (a.order ? static_cast<int64_t>(a.order[pos - nl]) : pos - nl);
    int64_t start = a.row_ptr[r], end = a.row_ptr[r + 1];
    if (start < 0 || end < start || end > a.nnz) {
      if (lane == 0) raise_error(a.err, FLASH_DEVERR_ROW_PTR);
      start = end = 0;
    }
    if (!listed && nl > 0 && end - start >= a.long_min) continue;  // hashed from the list
    const int64_t n = end - start;
    if (n == 0) {  // empty row: all-ones hashes; never inserted
      emit_empty<KEYS>(a, r, lane);
      __syncwarp();
      continue;
    }

    if (n <= static_cast<int64_t>(B / 2)) {
      sparse_row(a, start, end, bins, mask, lane);
      finish_row<KEYS, true>(a, r, bins, mask, lane);
    } else if (B & 1u) {  // odd B: element by element
      insert_row_checked(a, start, end, bins, mask, lane);
      dense_mask(a, bins, mask, lane);
      finish_row<KEYS, false>(a, r, bins, mask, lane);
    } else {
      // ---- dense row: head up to a 16-byte boundary, 16-byte body in groups
      // of 128 int4 (4 per lane), the last group partial, tail; the columns
      // are range-checked once per row (a row holding one out of range is
      // redone element by element)
      {
        uint4 *b4 = reinterpret_cast<uint4 *>(bins);
        const uint4 ones = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        for (uint32_t q4 = lane; q4 < W * 8; q4 += 32) b4[q4] = ones;
      }
      __syncwarp();
      int64_t a4, nq;
      row_body(start, end, mis, a4, nq);
      const int64_t b4 = a4 + 4 * nq;
      const int4 *body = reinterpret_cast<const int4 *>(a.col + a4);
      const int64_t nfull = nq >> 7;
      uint32_t mx = 0;
      if (start + static_cast<int64_t>(lane) < a4) {
        const uint32_t c = static_cast<uint32_t>(a.col[start + lane]);
        mx = max(mx, c);
        insert_fast(c, a1_lo, a1_hi, b1, B, bins);
      }
      if (b4 + static_cast<int64_t>(lane) < end) {
        const uint32_t c = static_cast<uint32_t>(a.col[b4 + lane]);
        mx = max(mx, c);
        insert_fast(c, a1_lo, a1_hi, b1, B, bins);
      }
      int4 g0 = zero, g1 = zero, g2 = zero, g3 = zero;
      if (nfull > 0) {
        const int4 *p0 = body + lane;
        g0 = __ldcs(p0);
        g1 = __ldcs(p0 + 32);
        g2 = __ldcs(p0 + 64);
        g3 = __ldcs(p0 + 96);
      }
      for (int64_t g = 0; g < nfull; ++g) {
        int4 n0 = g0, n1 = g1, n2 = g2, n3 = g3;
        if (g + 1 < nfull) {
          const int4 *pn = body + ((g + 1) << 7) + lane;
          n0 = __ldcs(pn);
          n1 = __ldcs(pn + 32);
          n2 = __ldcs(pn + 64);
          n3 = __ldcs(pn + 96);
        }
        insert8(g0, g1, a1_lo, a1_hi, b1, B, bins, mx);
        insert8(g2, g3, a1_lo, a1_hi, b1, B, bins, mx);
        g0 = n0;
        g1 = n1;
        g2 = n2;
        g3 = n3;
      }
      if ((nfull << 7) < nq) {
        // the valid 16-byte parts of a lane are a prefix
        const int64_t q0 = (nfull << 7) + lane;
        g0 = q0 < nq ? __ldcs(body + q0) : zero;
        g1 = q0 + 32 < nq ? __ldcs(body + q0 + 32) : zero;
        g2 = q0 + 64 < nq ? __ldcs(body + q0 + 64) : zero;
        g3 = q0 + 96 < nq ? __ldcs(body + q0 + 96) : zero;
        if (q0 < nq) insert4(g0, a1_lo, a1_hi, b1, B, bins, mx);
        if (q0 + 32 < nq) insert4(g1, a1_lo, a1_hi, b1, B, bins, mx);
        if (q0 + 64 < nq) insert4(g2, a1_lo, a1_hi, b1, B, bins, mx);
        if (q0 + 96 < nq) insert4(g3, a1_lo, a1_hi, b1, B, bins, mx);
      }
      __syncwarp();
      const bool bad = __any_sync(kFull, mx >= dim);
      if (bad) insert_row_checked(a, start, end, bins, mask, lane);
      // rows with every bin filled (nearly all dense rows) skip the bitmap and densification
      bool empty_bin = false;
      for (uint32_t j = lane; j < B; j += 32) empty_bin |= bins[j] == 0xFFFFFFFFu;
      if (__any_sync(kFull, empty_bin)) {
        for (uint32_t w = lane; w < W; w += 32) mask[w] = 0;
        dense_mask(a, bins, mask, lane);
        finish_row<KEYS, false>(a, r, bins, mask, lane);
      } else {
        emit_row<KEYS, false>(a, r, bins, lane);
      }
    }
  }
}

// ---- longest-rows-first processing order: rows binned by ceil(log2(nnz + 1))
__global__ void __launch_bounds__(256) row_class_hist_kernel(const int64_t *row_ptr, int64_t n, uint32_t *hist) {
  __shared__ uint32_t h[40];
  if (threadIdx.x < 40) h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t m = row_ptr[r + 1] - row_ptr[r];
    const uint32_t c = m > 0 ? 64u - __clzll(static_cast<unsigned long long>(m)) : 0u;
    atomicAdd(&h[c], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 40 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void row_class_scan_kernel(uint32_t *hist) {  // one thread: offsets, largest class first
  uint32_t run = 0;
  for (int c = 39; c >= 0; --c) {
    const uint32_t v = hist[c];
    hist[c] = run;
    run += v;
  }
}

// rows of class >= cmin go to order[offs[class]++] (cmin = 0: every row)
__global__ void __launch_bounds__(256) row_class_scatter_kernel(const int64_t *row_ptr, int64_t n, uint32_t *offs,
                                                                int32_t *order, uint32_t cmin) {
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t m = row_ptr[r + 1] - row_ptr[r];
    const uint32_t c = m > 0 ? 64u - __clzll(static_cast<unsigned long long>(m)) : 0u;
    if (c >= cmin) order[atomicAdd(&offs[c], 1u)] = static_cast<int32_t>(r);
  }
}

// offsets of the classes >= cmin, largest class first; hist[40] = their rows
__global__ void long_class_scan_kernel(uint32_t *hist, uint32_t cmin) {  // one thread
  uint32_t run = 0;
  for (int c = 39; c >= static_cast<int>(cmin); --c) {
    const uint32_t v = hist[c];
    hist[c] = run;
    run += v;
  }
  hist[40] = run;
}

// 32 x 32 tiles (rows x tables): coalesced reads along the tables of a row,
// coalesced writes along the rows of a table.  A grid of a few blocks per SM
// walks the tiles two at a time (one tile per block would make millions of
// tiny blocks at L = 256); each thread has its eight loads in flight before it
// stores.
__global__ void __launch_bounds__(256) transpose_keys_kernel(const uint32_t *rm, int64_t n, uint32_t L, uint32_t *tm,
                                                              int64_t ld) {
  __shared__ uint32_t tile[2][32][33];
  const uint32_t tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t row_tiles = (n + 31) / 32;
  const int64_t tiles = row_tiles * ((L + 31) / 32);
  for (int64_t ti = blockIdx.x; ti < tiles; ti += 2LL * gridDim.x) {
    uint32_t v[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t tu = ti + u * static_cast<int64_t>(gridDim.x);
      const int64_t r0 = (tu % row_tiles) * 32;
      const uint32_t t0 = static_cast<uint32_t>(tu / row_tiles) * 32;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + ty + 8 * i;
        const uint32_t t = t0 + tx;
        v[u][i] = (tu < tiles && r < n && t < L) ? __ldcs(rm + r * L + t) : 0u;
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i) tile[u][ty + 8 * i][tx] = v[u][i];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t tu = ti + u * static_cast<int64_t>(gridDim.x);
      if (tu < tiles) {
        const int64_t r0 = (tu % row_tiles) * 32;
        const uint32_t t0 = static_cast<uint32_t>(tu / row_tiles) * 32;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t t = t0 + ty + 8 * i;
          const int64_t r = r0 + tx;
          if (r < n && t < L) tm[static_cast<int64_t>(t) * ld + r] = tile[u][tx][ty + 8 * i];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

int launch_transpose_keys(const uint32_t *rm, int64_t n, uint32_t L, uint32_t *tm, int64_t ld, cudaStream_t stream) {
  if (n <= 0) return 0;
  const int64_t tiles = ((n + 31) / 32) * ((L + 31) / 32);
  int64_t blocks = 8LL * num_sms();
  if (blocks > tiles) blocks = tiles;
  transpose_keys_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(rm, n, L, tm, ld);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

int build_row_order(const int64_t *row_ptr, int64_t n, int32_t *order, uint32_t *hist40, cudaStream_t stream) {
  if (n <= 0) return 0;
  if (cudaMemsetAsync(hist40, 0, 40 * sizeof(uint32_t), stream) != cudaSuccess) return FLASH_ECUDA;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 8L * num_sms()) blocks = 8L * num_sms();
  row_class_hist_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(row_ptr, n, hist40);
  row_class_scan_kernel<<<1, 1, 0, stream>>>(hist40);
  row_class_scatter_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(row_ptr, n, hist40, order, 0u);
  count_launches(3);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

int build_long_rows(const int64_t *row_ptr, int64_t n, uint32_t cmin, int32_t *long_rows, uint32_t *hist41,
                    cudaStream_t stream) {
  if (cudaMemsetAsync(hist41, 0, 41 * sizeof(uint32_t), stream) != cudaSuccess) return FLASH_ECUDA;
  if (n <= 0) return 0;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 8L * num_sms()) blocks = 8L * num_sms();
  row_class_hist_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(row_ptr, n, hist41);
  long_class_scan_kernel<<<1, 1, 0, stream>>>(hist41, cmin);
  row_class_scatter_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(row_ptr, n, hist41, long_rows, cmin);
  count_launches(3);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

int launch_doph(const DophLaunch &L, cudaStream_t stream) {
  DophParams a{};
  a.row_ptr = L.row_ptr;
  a.col = L.col;
  a.n_rows = L.n_rows;
  a.nnz = L.nnz;
  a.dim_u32 = static_cast<uint32_t>(L.dim > 0xFFFFFFFFLL ? 0xFFFFFFFFLL : L.dim);
  a.B = L.K * L.L;
  a.K = L.K;
  a.L = L.L;
  a.rb = L.range_bits;
  a.W = (a.B + 31) / 32;
  a.G = (a.W + 31) / 32;
  a.bin_words = (a.W * 33 + 3) & ~3u;
  a.smem_words_per_warp = a.bin_words + ((a.W + 3) & ~3u);
  a.s = L.seeds;
  a.densify = L.densify;
  a.pool = L.keys ? L.pool : 0u;
  a.pool_bits = L.pool_bits;
  a.out = L.out;
  a.out_rm = L.out_rowmajor;
  a.ld = L.ld;
  a.vec_out = !L.keys && (a.B % 4 == 0) && ((reinterpret_cast<uintptr_t>(L.out) & 15) == 0);
  a.err = L.err;
  a.row_counter = L.row_counter;
  a.order = L.order;
  a.long_rows = L.long_rows;
  a.long_count = L.long_count;
  a.long_min = L.long_min;
  const double avg = L.n_rows > 0 ? static_cast<double>(L.nnz) / static_cast<double>(L.n_rows) : 1.0;
  // short rows are claimed several at a time; at most 16, so that the rows in
  // flight stay few enough for their table-major keys to meet in L2 (64 per
  // claim cost the L = 256 shape half its speed in read-modify-writes)
  uint32_t g = static_cast<uint32_t>(2048.0 / (avg + 16.0) + 1.0);
  a.rows_per_grab = g < 1 ? 1 : (g > 16 ? 16 : g);
  if (L.rows_per_grab) a.rows_per_grab = L.rows_per_grab;

  if (L.n_rows == 0) return 0;
  const size_t smem = static_cast<size_t>(kWarpsPerBlock) * a.smem_words_per_warp * sizeof(uint32_t);
  auto kern = L.keys ? doph_kernel<true> : doph_kernel<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return FLASH_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, smem) != cudaSuccess)
    return FLASH_ECUDA;
  if (per_sm < 1) return FLASH_EINVAL;
  const int64_t warps_needed = (L.n_rows + a.rows_per_grab - 1) / a.rows_per_grab;
  int64_t blocks = static_cast<int64_t>(per_sm) * num_sms();
  const int64_t max_useful = (warps_needed + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks > max_useful) blocks = max_useful;
  if (L.max_blocks > 0 && blocks > L.max_blocks) blocks = L.max_blocks;
  if (cudaMemsetAsync(L.row_counter, 0, sizeof(unsigned long long), stream) != cudaSuccess) return FLASH_ECUDA;
  kern<<<static_cast<unsigned>(blocks), kWarpsPerBlock * 32, smem, stream>>>(a);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : FLASH_ECUDA;
}

}  // namespace flash
