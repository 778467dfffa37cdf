/*
 * flash_oracle.c -- plain, slow CPU oracle for FLASH's hot path
 * (Wang, Shrivastava, Wang, Ryu: "FLASH: Randomized Algorithms Accelerated
 * over CPU-GPU for Ultra-High Dimensional Similarity Search").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Every step is written in the order and notation of the paper:
 *   - minwise hash, Eq. 1 (Section 2.1), applied per bin of a one-permutation
 *     hash and densified (Section 2.3);
 *   - MapKHashesToAddress, Section 2.2 and Algorithm 2;
 *   - the Adding phase with reservoir sampling, Algorithms 1 and 2;
 *   - the Querying phase with count-based k-selection, Algorithm 3.
 * Where the paper leaves a choice open (the hash family, densification
 * variant -- rotation, or the optimal densification of [36] the paper cites,
 * chosen by a densify argument --, which K hashes form table t, the
 * random-number generator) the fixed reading is stated at the function that
 * uses it.
 *
 * All arithmetic is on unsigned integers with wrap-around modulo 2^w.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ seeds
 * Section 2.3: DOPH needs only a handful of random numbers.  Reading: the
 * user seed s starts a SplitMix64 sequence (Steele, Lea & Flood, OOPSLA
 * 2014); its first six outputs are a1, b1, a2, b2, r, d with a1, a2 forced
 * odd.
 *   a1, b1 : the permutation surrogate pi (one-permutation hashing)
 *   a2, b2 : MapKHashesToAddress
 *   r      : key of the reservoir random numbers (Algorithm 1 / 2)
 *   d      : key of the probe sequence of optimal densification
 *   e      : key of the bucket -> reservoir map of reservoir sharing       */
typedef struct {
  uint64_t a1, b1, a2, b2, r, d, e;
} oracle_seeds_t;

static uint64_t splitmix64_next(uint64_t *state) {
  uint64_t z;
  *state += 0x9E3779B97F4A7C15ULL;
  z = *state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* the SplitMix64 output function applied to an arbitrary word */
static uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static oracle_seeds_t make_seeds(uint64_t seed) {
  oracle_seeds_t s;
  uint64_t st = seed;
  s.a1 = splitmix64_next(&st) | 1ULL;
  s.b1 = splitmix64_next(&st);
  s.a2 = splitmix64_next(&st) | 1ULL;
  s.b2 = splitmix64_next(&st);
  s.r = splitmix64_next(&st);
  s.d = splitmix64_next(&st);
  s.e = splitmix64_next(&st);
  return s;
}

void oracle_seeds(uint64_t seed, uint64_t out[5]) {
  oracle_seeds_t s = make_seeds(seed);
  out[0] = s.a1;
  out[1] = s.b1;
  out[2] = s.a2;
  out[3] = s.b2;
  out[4] = s.r;
}

/* ---------------------------------------------------------------- DOPH
 * Section 2.3 (one pass, K*L hashes) built on Eq. 1 (minwise hash).
 *
 * Permutation surrogate (reading): pi(i) = (a1*i + b1 mod 2^64) >> 32, the
 * multiply-add-shift universal family.  One permutation is split into
 * B = K*L equal ranges (bins): with p = pi(i) * B (64-bit), the bin is
 * p >> 32 and the position inside the bin is off = p mod 2^32; inside one
 * bin off increases with pi, so "smallest off" is "smallest pi" (Eq. 1).
 *
 * OPH: v[j] = min{ off(i) : x_i != 0, bin(i) = j }, empty if no such i.
 * Two densifications of the empty bins (densify = 0 or 1):
 *  0, rotation (Shrivastava & Li, UAI 2014): an empty bin j takes the value
 *     of the first non-empty bin to its right, circularly, at distance
 *     t >= 1, plus t * 0x9E3779B9 (mod 2^32);
 *  1, optimal densification (the variant Section 2.3 cites as [36]; the
 *     paper does not define it, reading): an empty bin j probes the bins
 *         src_i = ((mix(d XOR (j * 2^32 + i)) >> 32) * B) >> 32,
 *     mix = the SplitMix64 output function (a random hash of (bin,
 *     attempt)), for attempts i = 1, 2, ..., 8B, and copies the value of the
 *     first non-empty one, unchanged; if all 8B probes are empty it copies
 *     the first non-empty bin to its right, circularly, unchanged.
 * An empty row (no non-zeros) hashes to 0xFFFFFFFF in every bin.
 * Values x_i are ignored: the hash sees only the set of non-zero columns.   */
static void doph_row(const int32_t *cols, int64_t nnz, uint32_t B, const oracle_seeds_t *s, uint32_t densify,
                     uint32_t *h, uint32_t *v, uint8_t *filled, uint32_t *next_src) {
  int64_t e;
  uint32_t j;
  if (nnz == 0) {
    for (j = 0; j < B; ++j) h[j] = 0xFFFFFFFFu;
    return;
  }
  memset(filled, 0, B);
  for (e = 0; e < nnz; ++e) {
    uint64_t i = (uint64_t)(uint32_t)cols[e];
    uint32_t pi = (uint32_t)((s->a1 * i + s->b1) >> 32);
    uint64_t p = (uint64_t)pi * (uint64_t)B;
    uint32_t bin = (uint32_t)(p >> 32);
    uint32_t off = (uint32_t)p;
    if (!filled[bin] || off < v[bin]) {
      v[bin] = off;
      filled[bin] = 1;
    }
  }
  /* next_src[j] = first non-empty bin at or to the right of j (circular).
   * Right of the last non-empty bin the search wraps to the first
   * non-empty bin from 0 (one exists: nnz > 0); a backward sweep fills the
   * rest.                                                                  */
  {
    int64_t jj;
    uint32_t cur = 0;
    for (jj = 0; jj < (int64_t)B; ++jj)
      if (filled[jj]) { cur = (uint32_t)jj; break; }
    for (jj = (int64_t)B - 1; jj >= 0; --jj) {
      if (filled[jj]) cur = (uint32_t)jj;
      next_src[jj] = cur;
    }
  }
  for (j = 0; j < B; ++j) {
    uint32_t src = next_src[j];
    if (densify == 0) {
      uint32_t t = src >= j ? src - j : src + B - j;
      h[j] = v[src] + t * 0x9E3779B9u;
    } else if (filled[j]) {
      h[j] = v[j];
    } else {
      uint64_t i;
      for (i = 1; i <= 8ULL * B; ++i) {
        uint64_t u = splitmix64_mix(s->d ^ (((uint64_t)j << 32) | i));
        uint32_t probe = (uint32_t)(((u >> 32) * (uint64_t)B) >> 32);
        if (filled[probe]) { src = probe; break; }
      }
      h[j] = v[src];
    }
  }
}

/* ------------------------------------------------- MapKHashesToAddress
 * Section 2.2 / Algorithm 2: a universal random map of the K-tuple of
 * table t to an address in [0, 2^range_bits).
 * Reading: table t takes the hashes h[t + j*L], j = 0..K-1 (interleaved),
 * folded as x <- x*a2 + h (Horner, mod 2^64) from x = 0; then
 * key = (a2*x + b2 mod 2^64) >> (64 - range_bits).                        */
static uint32_t map_k_hashes_to_address(const uint32_t *h, uint32_t t, uint32_t K, uint32_t L, uint32_t rb,
                                        const oracle_seeds_t *s) {
  uint64_t x = 0;
  uint32_t j;
  for (j = 0; j < K; ++j) x = x * s->a2 + (uint64_t)h[t + j * L];
  return (uint32_t)((s->a2 * x + s->b2) >> (64 - rb));
}

/* -------------------------------------------- reservoir random number
 * Algorithms 1 and 2 draw j = RANDOM([0, i]) for the arrival of rank i
 * (0-based) in bucket b of table t.
 * Reading: a counter-based draw keyed by (r, t, b, i):
 *   u = mix(mix(r XOR (t*2^32 + b)) XOR i),  mix = SplitMix64 output function,
 *   j = ((u >> 32) * (i + 1)) >> 32        (multiply-shift range reduction). */
static uint32_t reservoir_random(uint64_t r, uint32_t t, uint32_t b, uint64_t i) {
  uint64_t u = splitmix64_mix(splitmix64_mix(r ^ (((uint64_t)t << 32) + (uint64_t)b)) ^ i);
  return (uint32_t)(((u >> 32) * (i + 1)) >> 32);
}

/* ADD of Algorithm 2 with Algorithm 1's fill-first rule.
 * Reading: while fewer than R items have arrived the item fills slot
 * counter (Algorithm 1's first loop); afterwards j = RANDOM([0, counter])
 * and the item replaces slot j when j < R (Algorithm 2's test; Algorithm 1
 * prints "<=", which would address slot R, one past the reservoir).       */
static void add(int32_t *reservoir, uint32_t *counter, uint32_t R, uint64_t r, uint32_t t, uint32_t key,
                int32_t point) {
  uint32_t i = *counter;
  if (i < R) {
    reservoir[i] = point;
  } else {
    uint32_t j = reservoir_random(r, t, key, i);
    if (j < R) reservoir[j] = point;
  }
  *counter = i + 1;
}

/* ------------------------------------------------------- public: hashing */

/* hashes of rows [r0, r1) -> out[(r - r0) * B + j], B = K*L               */
int oracle_hash(const int64_t *row_ptr, const int32_t *col, int64_t r0, int64_t r1, uint32_t K, uint32_t L,
                uint64_t seed, uint32_t densify, uint32_t *out) {
  uint32_t B = K * L;
  oracle_seeds_t s = make_seeds(seed);
  uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint8_t *filled = (uint8_t *)malloc(B);
  uint32_t *nx = (uint32_t *)malloc(sizeof(uint32_t) * B);
  int64_t r;
  if (!v || !filled || !nx) { free(v); free(filled); free(nx); return -1; }
  for (r = r0; r < r1; ++r)
    doph_row(col + row_ptr[r], row_ptr[r + 1] - row_ptr[r], B, &s, densify, out + (r - r0) * (int64_t)B, v, filled,
             nx);
  free(v);
  free(filled);
  free(nx);
  return 0;
}

/* table addresses of rows [r0, r1) -> keys[t * ld + (r - r0)]              */
int oracle_keys(const int64_t *row_ptr, const int32_t *col, int64_t r0, int64_t r1, uint32_t K, uint32_t L,
                uint32_t rb, uint64_t seed, uint32_t densify, uint32_t *keys, int64_t ld) {
  uint32_t B = K * L, t;
  oracle_seeds_t s = make_seeds(seed);
  uint32_t *h = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint8_t *filled = (uint8_t *)malloc(B);
  uint32_t *nx = (uint32_t *)malloc(sizeof(uint32_t) * B);
  int64_t r;
  if (!h || !v || !filled || !nx) { free(h); free(v); free(filled); free(nx); return -1; }
  for (r = r0; r < r1; ++r) {
    doph_row(col + row_ptr[r], row_ptr[r + 1] - row_ptr[r], B, &s, densify, h, v, filled, nx);
    for (t = 0; t < L; ++t) keys[(int64_t)t * ld + (r - r0)] = map_k_hashes_to_address(h, t, K, L, rb, &s);
  }
  free(h);
  free(v);
  free(filled);
  free(nx);
  return 0;
}

/* ------------------------------------------- public: the Adding phase
 * Algorithm 2 over every data point in index order 0..N-1.
 * tables[(t * 2^rb + key) * R + slot] (empty slot = -1),
 * counts[t * 2^rb + key] = number of arrivals (not capped at R).
 * Reading: a row with no non-zeros is not inserted anywhere.              */
int oracle_add(const int64_t *row_ptr, const int32_t *col, int64_t n, int32_t id0, uint32_t K, uint32_t L,
               uint32_t R, uint32_t rb, uint64_t seed, uint32_t densify, int32_t *tables, uint32_t *counts);

int oracle_build(const int64_t *row_ptr, const int32_t *col, int64_t n, uint32_t K, uint32_t L, uint32_t R,
                 uint32_t rb, uint64_t seed, uint32_t densify, int32_t *tables, uint32_t *counts) {
  uint64_t T = 1ULL << rb, z;
  for (z = 0; z < (uint64_t)L * T * R; ++z) tables[z] = -1;
  memset(counts, 0, sizeof(uint32_t) * (size_t)((uint64_t)L * T));
  return oracle_add(row_ptr, col, n, 0, K, L, R, rb, seed, densify, tables, counts);
}

/* Algorithm 2 is a stream: ADD continues every bucket's arrival count, so
 * points added later (rows [0, n) of another matrix, point ids id0 + row)
 * extend tables and counts exactly as if they had come after the earlier
 * points in one build.                                                     */
int oracle_add(const int64_t *row_ptr, const int32_t *col, int64_t n, int32_t id0, uint32_t K, uint32_t L,
               uint32_t R, uint32_t rb, uint64_t seed, uint32_t densify, int32_t *tables, uint32_t *counts) {
  uint32_t B = K * L, t;
  uint64_t T = 1ULL << rb;
  oracle_seeds_t s = make_seeds(seed);
  uint32_t *all_hashes = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint8_t *filled = (uint8_t *)malloc(B);
  uint32_t *nx = (uint32_t *)malloc(sizeof(uint32_t) * B);
  int64_t p;
  if (!all_hashes || !v || !filled || !nx) { free(all_hashes); free(v); free(filled); free(nx); return -1; }
  for (p = 0; p < n; ++p) {                                   /* for each DataPoint */
    int64_t nnz = row_ptr[p + 1] - row_ptr[p];
    if (nnz == 0) continue;
    doph_row(col + row_ptr[p], nnz, B, &s, densify, all_hashes, v, filled, nx);   /* AllHashes := DOPH */
    for (t = 0; t < L; ++t) {                                 /* for each Table_t */
      uint32_t key = map_k_hashes_to_address(all_hashes, t, K, L, rb, &s);
      uint64_t bucket = (uint64_t)t * T + key;
      add(tables + bucket * R, counts + bucket, R, s.r, t, key, (int32_t)(id0 + p));   /* ADD */
    }
  }
  free(all_hashes);
  free(v);
  free(filled);
  free(nx);
  return 0;
}

/* The Adding phase of Algorithm 2 for tables t0..t1-1 only, from the table
 * addresses already computed (keys[t * ld + p], as oracle_keys writes
 * them): the points arrive in index order and every ADD is the one
 * oracle_build does, so the tables equal oracle_build's.  Tables are
 * independent (Section 3.4), which lets a driver build them on several
 * threads.  tables / counts as in oracle_build (all L tables).            */
int oracle_build_tables_from_keys(const uint32_t *keys, int64_t ld, const int64_t *row_ptr, int64_t n, uint32_t t0,
                                  uint32_t t1, uint32_t R, uint32_t rb, uint64_t seed, int32_t *tables,
                                  uint32_t *counts) {
  uint64_t T = 1ULL << rb, z;
  oracle_seeds_t s = make_seeds(seed);
  int64_t p;
  uint32_t t;
  for (t = t0; t < t1; ++t) {
    for (z = 0; z < T * R; ++z) tables[(uint64_t)t * T * R + z] = -1;
    memset(counts + (uint64_t)t * T, 0, sizeof(uint32_t) * (size_t)T);
    for (p = 0; p < n; ++p) {
      uint32_t key;
      uint64_t bucket;
      if (row_ptr[p + 1] == row_ptr[p]) continue;  /* empty rows are never inserted */
      key = keys[(int64_t)t * ld + p];
      bucket = (uint64_t)t * T + key;
      add(tables + bucket * R, counts + bucket, R, s.r, t, key, (int32_t)p);
    }
  }
  return 0;
}

/* Algorithm 1 run on the arrival stream of one bucket only: the points p
 * (ascending) with keys_t[p] == key and a non-empty row.  This is the
 * Adding phase restricted to bucket (t, key); used to check single buckets
 * of workloads whose full tables do not fit in host memory.               */
int oracle_bucket(const uint32_t *keys_t, const int64_t *row_ptr, int64_t n, uint32_t t, uint32_t key, uint32_t R,
                  uint64_t seed, int32_t *reservoir, uint32_t *count) {
  oracle_seeds_t s = make_seeds(seed);
  int64_t p;
  uint32_t j;
  for (j = 0; j < R; ++j) reservoir[j] = -1;
  *count = 0;
  for (p = 0; p < n; ++p)
    if (keys_t[p] == key && row_ptr[p + 1] > row_ptr[p]) add(reservoir, count, R, s.r, t, key, (int32_t)p);
  return 0;
}

/* ---------------------------------------- public: KSELECT (Algorithm 3)
 * SORTINPLACE(A); COUNTFREQUENCY: one (id, count) pair per run of equal ids
 * (reading: a run of length c counts c -- the printed loop only increments
 * on equal neighbours, which would give a single occurrence count 0);
 * SORTBYVALUE: count descending, ties by smaller id (reading); return the
 * first k.  The id `exclude` (>= 0) is dropped; missing entries are (-1, 0). */
typedef struct {
  int32_t id;
  int32_t count;
} kv_t;

static int cmp_id(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static int cmp_value(const void *a, const void *b) {
  const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
  if (x->count != y->count) return x->count > y->count ? -1 : 1;
  return (x->id > y->id) - (x->id < y->id);
}

int oracle_kselect(int32_t *A, int64_t n, int32_t exclude, int32_t k, int32_t *out_ids, int32_t *out_counts) {
  kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
  int64_t i, m = 0;
  int32_t q;
  if (!kv) return -1;
  qsort(A, (size_t)n, sizeof(int32_t), cmp_id);                      /* SORTINPLACE(A) */
  for (i = 0; i < n; ++i) {                                           /* COUNTFREQUENCY(A) */
    if (i > 0 && A[i] == A[i - 1]) {
      kv[m - 1].count++;
    } else {
      kv[m].id = A[i];
      kv[m].count = 1;
      m++;
    }
  }
  {
    int64_t w = 0;
    for (i = 0; i < m; ++i)
      if (kv[i].id != exclude) kv[w++] = kv[i];
    m = w;
  }
  qsort(kv, (size_t)m, sizeof(kv_t), cmp_value);                      /* SORTBYVALUEINPLACE */
  for (q = 0; q < k; ++q) {                                           /* KVPair[0:TopK] */
    out_ids[q] = q < m ? kv[q].id : -1;
    out_counts[q] = q < m ? kv[q].count : 0;
  }
  free(kv);
  return 0;
}

/* ------------------------------------ public: the Querying phase
 * Algorithm 3 for query rows [0, nq) against tables built by oracle_build.
 * For each query: AllHashes := DOPH(query); A := concatenation over tables
 * t of the occupied slots of Table_t[Key_t] (the printed "Table_t[Key]");
 * out := KSELECT(A).  exclude may be NULL (no exclusion).
 * Reading: a query row with no non-zeros reports nothing.                 */
int oracle_query(const int32_t *tables, const uint32_t *counts, uint32_t K, uint32_t L, uint32_t R, uint32_t rb,
                 uint64_t seed, uint32_t densify, const int64_t *q_row_ptr, const int32_t *q_col, int64_t nq, int32_t k,
                 const int32_t *exclude, int32_t *out_ids, int32_t *out_counts) {
  uint32_t B = K * L, t;
  uint64_t T = 1ULL << rb;
  oracle_seeds_t s = make_seeds(seed);
  uint32_t *all_hashes = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint8_t *filled = (uint8_t *)malloc(B);
  uint32_t *nx = (uint32_t *)malloc(sizeof(uint32_t) * B);
  int32_t *A = (int32_t *)malloc(sizeof(int32_t) * (size_t)L * R);
  int64_t q;
  if (!all_hashes || !v || !filled || !nx || !A) {
    free(all_hashes); free(v); free(filled); free(nx); free(A);
    return -1;
  }
  for (q = 0; q < nq; ++q) {                                   /* for each QueryPoint */
    int64_t nnz = q_row_ptr[q + 1] - q_row_ptr[q], n = 0;
    int32_t e;
    if (nnz == 0) {
      for (e = 0; e < k; ++e) { out_ids[q * k + e] = -1; out_counts[q * k + e] = 0; }
      continue;
    }
    doph_row(q_col + q_row_ptr[q], nnz, B, &s, densify, all_hashes, v, filled, nx);
    for (t = 0; t < L; ++t) {                                  /* Append A with Table_t[Key_t] */
      uint32_t key = map_k_hashes_to_address(all_hashes, t, K, L, rb, &s);
      uint64_t bucket = (uint64_t)t * T + key;
      uint32_t m = counts[bucket] < R ? counts[bucket] : R, j;
      for (j = 0; j < m; ++j) A[n++] = tables[bucket * R + j];
    }
    oracle_kselect(A, n, exclude ? exclude[q] : -1, k, out_ids + q * k, out_counts + q * k);
  }
  free(all_hashes);
  free(v);
  free(filled);
  free(nx);
  free(A);
  return 0;
}

/* Algorithm 3 for one query whose table addresses are given (q_keys[t]),
 * with every bucket's reservoir rebuilt from the arrival stream by
 * oracle_bucket (keys_all[t * ld + p] for all N points).  Same result as
 * oracle_query on tables from oracle_build; memory O(L*R) instead of the
 * full tables.                                                            */
int oracle_query_one_streamed(const uint32_t *keys_all, int64_t ld, const int64_t *row_ptr, int64_t n, uint32_t L,
                              uint32_t R, uint64_t seed, const uint32_t *q_keys, int q_empty, int32_t k,
                              int32_t exclude, int32_t *out_ids, int32_t *out_counts) {
  int32_t *A = (int32_t *)malloc(sizeof(int32_t) * (size_t)L * R);
  int32_t *res = (int32_t *)malloc(sizeof(int32_t) * R);
  int64_t na = 0;
  uint32_t t;
  if (!A || !res) { free(A); free(res); return -1; }
  if (q_empty) {
    int32_t e;
    for (e = 0; e < k; ++e) { out_ids[e] = -1; out_counts[e] = 0; }
    free(A);
    free(res);
    return 0;
  }
  for (t = 0; t < L; ++t) {
    uint32_t cnt, m, j;
    oracle_bucket(keys_all + (int64_t)t * ld, row_ptr, n, t, q_keys[t], R, seed, res, &cnt);
    m = cnt < R ? cnt : R;
    for (j = 0; j < m; ++j) A[na++] = res[j];
  }
  oracle_kselect(A, na, exclude, k, out_ids, out_counts);
  free(A);
  free(res);
  return 0;
}

/* --------------------------------------- public: all-points k-NN graph
 * Every data point is a query against the index of all points, excluding
 * itself (Section 1; Section 4.3: Initialization + Addition + Querying).  */
int oracle_knn_graph(const int64_t *row_ptr, const int32_t *col, int64_t n, uint32_t K, uint32_t L, uint32_t R,
                     uint32_t rb, uint64_t seed, uint32_t densify, int32_t k, int32_t *out_ids, int32_t *out_counts) {
  uint64_t T = 1ULL << rb;
  int32_t *tables = (int32_t *)malloc(sizeof(int32_t) * (size_t)((uint64_t)L * T * R));
  uint32_t *counts = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)((uint64_t)L * T));
  int32_t *self = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t p;
  int rc;
  if (!tables || !counts || !self) { free(tables); free(counts); free(self); return -1; }
  for (p = 0; p < n; ++p) self[p] = (int32_t)p;
  rc = oracle_build(row_ptr, col, n, K, L, R, rb, seed, densify, tables, counts);
  if (rc == 0)
    rc = oracle_query(tables, counts, K, L, R, rb, seed, densify, row_ptr, col, n, k, self, out_ids, out_counts);
  free(tables);
  free(counts);
  free(self);
  return rc;
}

/* MapKHashesToAddress of table t for one given array of B = K*L hashes. */
uint32_t oracle_address(const uint32_t *h, uint32_t t, uint32_t K, uint32_t L, uint32_t rb, uint64_t seed) {
  oracle_seeds_t s = make_seeds(seed);
  return map_k_hashes_to_address(h, t, K, L, rb, &s);
}


/* ------------------------------------------- reservoir sharing (Section 3.5)
 * Section 3.2 (item 4), Section 3.5 and Figure 3: instead of one reservoir per
 * bucket, one shared pool of P reservoirs (Allocated Range = F * Actual
 * Range, over all L tables: P = F * L * 2^rb) serves every table; a bucket
 * points to a randomly chosen reservoir of the pool.  Readings:
 *   - the pointer of bucket b of table t is a fixed random map
 *       pool(t, b) = ((mix(e XOR (t * 2^32 + b)) >> 32) * P) >> 32,
 *     mix = the SplitMix64 output function, e the seventh SplitMix64 output
 *     of the seed (the paper assigns pool reservoirs at first use; a fixed
 *     map gives the same distribution and keeps the Adding phase
 *     data-parallel);
 *   - a shared reservoir receives its arrivals in the order of Algorithm 2's
 *     loop: points in id order, and for each point the tables in order;
 *   - its random numbers are keyed by (seed, 2^32 - 1, reservoir, arrival
 *     rank), the draw of Algorithms 1 and 2 for a "table" 2^32 - 1 no real
 *     table uses;
 *   - Querying (Algorithm 3) gathers, for every table t, the reservoir its
 *     bucket points to (a reservoir two buckets of the query share is
 *     gathered twice).                                                     */
static uint32_t pool_index(const oracle_seeds_t *s, uint32_t t, uint32_t b, uint32_t P) {
  uint64_t u = splitmix64_mix(s->e ^ (((uint64_t)t << 32) + (uint64_t)b));
  return (uint32_t)(((u >> 32) * (uint64_t)P) >> 32);
}

uint32_t oracle_pool_index(uint32_t t, uint32_t b, uint32_t P, uint64_t seed) {
  oracle_seeds_t s = make_seeds(seed);
  return pool_index(&s, t, b, P);
}

/* Adding phase with reservoir sharing: tables[x * R + slot], counts[x] for
 * the P reservoirs of the pool.                                            */
int oracle_build_shared(const int64_t *row_ptr, const int32_t *col, int64_t n, uint32_t K, uint32_t L, uint32_t R,
                        uint32_t rb, uint64_t seed, uint32_t densify, uint32_t P, int32_t *tables, uint32_t *counts) {
  uint32_t B = K * L, t;
  oracle_seeds_t s = make_seeds(seed);
  uint32_t *all_hashes = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint8_t *filled = (uint8_t *)malloc(B);
  uint32_t *nx = (uint32_t *)malloc(sizeof(uint32_t) * B);
  int64_t p;
  uint64_t z;
  if (!all_hashes || !v || !filled || !nx) { free(all_hashes); free(v); free(filled); free(nx); return -1; }
  for (z = 0; z < (uint64_t)P * R; ++z) tables[z] = -1;
  memset(counts, 0, sizeof(uint32_t) * (size_t)P);
  for (p = 0; p < n; ++p) {                                   /* for each DataPoint */
    int64_t nnz = row_ptr[p + 1] - row_ptr[p];
    if (nnz == 0) continue;
    doph_row(col + row_ptr[p], nnz, B, &s, densify, all_hashes, v, filled, nx);
    for (t = 0; t < L; ++t) {                                 /* for each Table_t */
      uint32_t key = map_k_hashes_to_address(all_hashes, t, K, L, rb, &s);
      uint32_t x = pool_index(&s, t, key, P);                 /* the shared reservoir it points to */
      add(tables + (uint64_t)x * R, counts + x, R, s.r, 0xFFFFFFFFu, x, (int32_t)p);
    }
  }
  free(all_hashes);
  free(v);
  free(filled);
  free(nx);
  return 0;
}

/* Querying phase with reservoir sharing, against tables from
 * oracle_build_shared.                                                     */
int oracle_query_shared(const int32_t *tables, const uint32_t *counts, uint32_t K, uint32_t L, uint32_t R,
                        uint32_t rb, uint64_t seed, uint32_t densify, uint32_t P, const int64_t *q_row_ptr,
                        const int32_t *q_col, int64_t nq, int32_t k, const int32_t *exclude, int32_t *out_ids,
                        int32_t *out_counts) {
  uint32_t B = K * L, t;
  oracle_seeds_t s = make_seeds(seed);
  uint32_t *all_hashes = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * B);
  uint8_t *filled = (uint8_t *)malloc(B);
  uint32_t *nx = (uint32_t *)malloc(sizeof(uint32_t) * B);
  int32_t *A = (int32_t *)malloc(sizeof(int32_t) * (size_t)L * R);
  int64_t q;
  if (!all_hashes || !v || !filled || !nx || !A) {
    free(all_hashes); free(v); free(filled); free(nx); free(A);
    return -1;
  }
  for (q = 0; q < nq; ++q) {
    int64_t nnz = q_row_ptr[q + 1] - q_row_ptr[q], na = 0;
    int32_t e;
    if (nnz == 0) {
      for (e = 0; e < k; ++e) { out_ids[q * k + e] = -1; out_counts[q * k + e] = 0; }
      continue;
    }
    doph_row(q_col + q_row_ptr[q], nnz, B, &s, densify, all_hashes, v, filled, nx);
    for (t = 0; t < L; ++t) {
      uint32_t key = map_k_hashes_to_address(all_hashes, t, K, L, rb, &s);
      uint32_t x = pool_index(&s, t, key, P), m = counts[x] < R ? counts[x] : R, j;
      for (j = 0; j < m; ++j) A[na++] = tables[(uint64_t)x * R + j];
    }
    oracle_kselect(A, na, exclude ? exclude[q] : -1, k, out_ids + q * k, out_counts + q * k);
  }
  free(all_hashes);
  free(v);
  free(filled);
  free(nx);
  free(A);
  return 0;
}
