// internal.h -- launchers shared between the translation units of libflash.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

// The index behind the opaque flash_index handle.
struct flash_index {
  flash_params p;
  flash::Seeds s;
  int64_t n;
  int device;
  int32_t *ids;       // [L][n]: points grouped by bucket; reservoir = first min(m, R) of a segment
  uint32_t *starts;   // [L][2^rb + 1]
  // reservoir sharing (p.share_pool = P > 0): one pool for every table, ids [L * n]
  // grouped by reservoir, starts [2^pool_bits + 1] (reservoirs >= P empty)
  uint32_t pool_bits;
  int64_t bytes;
};

namespace flash {

// Kernel launches issued by the current thread since the last reset
// (reported by flash_last_launch_count()).
void count_launches(int n);
void reset_launch_count();

// ---- K1: DOPH (+ optional key epilogue)
struct DophLaunch {
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t n_rows, nnz, dim;
  uint32_t K, L, range_bits;
  uint32_t densify;  // 0 rotation, 1 optimal densification
  uint32_t pool, pool_bits;  // keys mode, reservoir sharing: reservoir of each key (pool = P > 0); sentinel 2^pool_bits
  Seeds seeds;
  bool keys;         // false: out = hashes [n_rows][K*L]; true: out = keys [L][ld] (or null)
  uint32_t *out;
  uint32_t *out_rowmajor;  // keys mode, optional: keys [n_rows][L]
  int64_t ld;
  uint32_t *err;
  unsigned long long *row_counter;  // 8 bytes of device scratch
  uint32_t rows_per_grab;           // 0 = automatic
  int64_t max_blocks;               // 0 = automatic
  const int32_t *order;             // optional row processing order (null = 0..n-1)
  // optional: rows with at least long_min non-zeros, listed in long_rows[0 .. *long_count)
  // (longest class first), are hashed first and then skipped in index order
  const int32_t *long_rows;
  const uint32_t *long_count;
  int64_t long_min;
};
int launch_doph(const DophLaunch &l, cudaStream_t stream);
// keys [n][L] (row-major) -> keys [L][ld] (table-major), tiled through shared memory
int launch_transpose_keys(const uint32_t *rm, int64_t n, uint32_t L, uint32_t *tm, int64_t ld, cudaStream_t stream);
// order[0..n) = row ids, longest rows first (rows binned by log2 of their length);
// hist40: 40 words of scratch
int build_row_order(const int64_t *row_ptr, int64_t n, int32_t *order, uint32_t *hist40, cudaStream_t stream);
// long_rows[0 .. hist41[40]) = the rows with at least 2^(cmin - 1) non-zeros (log2
// class >= cmin), longest class first; hist41: 41 words of scratch
int build_long_rows(const int64_t *row_ptr, int64_t n, uint32_t cmin, int32_t *long_rows, uint32_t *hist41,
                    cudaStream_t stream);

// ---- K2: per-table stable sort of bucket addresses + bucket starts
// (partition by the high bits, then one warp per segment on the low bits)
struct SortPlan {
  int lo_bits, hi_bits;   // address bits sorted per segment / by the partition
  int passes;             // partition passes (digits of at most 8 bits)
  int shift[4], bits[4], nbins[4];
  uint32_t tile;
  int64_t tiles;          // tiles per table
  int64_t hist_words;     // L * max_nbins * tiles
  int64_t seg_words;      // segment starts after a multi-pass partition (0 for one pass)
};
SortPlan make_sort_plan(uint32_t range_bits, int64_t n, uint32_t L);

struct SortLaunch {
  const uint32_t *keys_in;  // [L][n] bucket addresses in [0, 2^rb]; 2^rb = not inserted
  int64_t n;
  uint32_t L, range_bits;
  int32_t *ids_out;         // [L][n] point ids in (address, id) order
  uint32_t *tmp_keys;       // [L][n]
  int32_t *tmp_ids;         // [L][n]
  uint32_t *keys_out;       // [L][n], partition passes 2, 4, ... (plan.passes > 1)
  int32_t *tmp_ids2;        // [L][n], partition passes 2, 4, ... (plan.passes > 1)
  uint32_t *hist;           // plan.hist_words
  uint32_t *seg;            // plan.seg_words
  uint32_t *starts;         // [L][2^rb + 1]
  unsigned long long *claim;  // 8 bytes of scratch
  // optional: the buckets holding more than R points, listed while the starts
  // are written (t << 32 | b; capacity heavy_cap); null to skip
  uint32_t R;
  unsigned long long *heavy_count;
  uint64_t *heavy;
  int64_t heavy_cap;
};
int sort_tables(const SortPlan &plan, const SortLaunch &s, cudaStream_t stream);

// ---- K3: reservoir selection in buckets with more than R arrivals
struct ReservoirLaunch {
  int32_t *ids;              // [L][n], sorted; reservoirs rewritten in place
  const uint32_t *starts;    // [L][2^rb + 1]
  int64_t n;
  uint32_t L, R, range_bits;
  uint64_t r;                // reservoir key
  bool shared;               // one pool of reservoirs (draws keyed by table 2^32 - 1)
  unsigned long long *heavy_count;  // 8 bytes of scratch
  uint64_t *heavy;           // list of (t << 32 | b), capacity heavy_cap
  int64_t heavy_cap;
  bool heavy_listed;         // the sort already listed the heavy buckets
};
int64_t reservoir_heavy_capacity(int64_t n, uint32_t L, uint32_t R, uint32_t range_bits);
int launch_reservoir(const ReservoirLaunch &l, cudaStream_t stream);

// ---- K4: gather + count + top-k
struct QueryLaunch {
  const uint32_t *qkeys;     // [L][q_ld], or [nq][L] when qkeys_rowmajor
  int64_t q_ld, nq;
  bool qkeys_rowmajor;
  const int32_t *ids;        // index: [L][n]
  const uint32_t *starts;    // index: [L][2^rb + 1]
  int64_t n;
  uint32_t L, R, range_bits;
  int32_t k;
  const int32_t *exclude;    // [nq] or null
  bool exclude_self;         // exclude id q from query q (all-points graph)
  int32_t *out_ids, *out_counts;  // [nq][k]
  bool shared;               // reservoir sharing: every table reads the one pool (ids, starts)
  unsigned long long *counters;   // 3 x 8 bytes of scratch
  int64_t *overflow;         // [nq] scratch
  uint32_t warp_table;       // 0 = automatic; else power of two
};
int launch_query(const QueryLaunch &l, cudaStream_t stream);

// ---- the plain, unbatched path (a baseline; plain.cu)
struct PlainHashLaunch {
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t n_rows, nnz, dim;
  uint32_t B, K, L, range_bits, densify;
  Seeds seeds;
  uint32_t *comp;     // [L][n_rows]: t * (2^rb + 1) + address (the sort keys)
  uint32_t *keys_rm;  // [n_rows][L]: addresses (the queries' keys)
  uint32_t *err;
};
int launch_plain_keys(const PlainHashLaunch &a, cudaStream_t stream);

struct PlainGroupLaunch {
  const uint32_t *comp_in;  // [L][n]
  uint32_t *comp_out;       // [L][n]
  int32_t *ids_in;          // [L][n] scratch (the values: point ids)
  int32_t *ids_out;         // [L][n] the index's grouped ids
  uint32_t *starts;         // [L][2^rb + 1]
  int64_t n;
  uint32_t L, R, range_bits;
  uint64_t rkey;            // reservoir key (Seeds::r)
  void *temp;
  size_t temp_bytes;
};
size_t plain_sort_temp_bytes(int64_t n, uint32_t L, uint32_t range_bits);
int launch_plain_group(const PlainGroupLaunch &g, cudaStream_t stream);

struct PlainQueryLaunch {
  const uint32_t *keys_rm;  // [nq][L]
  const int32_t *ids;       // index [L][n]
  const uint32_t *starts;   // index [L][2^rb + 1]
  int64_t n;
  uint32_t L, R, range_bits;
  int32_t k;
  const int32_t *exclude;
  bool exclude_self;
  int32_t *out_ids, *out_counts;
  uint32_t *cand, *cand2;   // [chunk][L*R] each
  const uint32_t *sorted;   // set by the launcher
  int64_t *seg_begin, *seg_end;  // [chunk]
  void *temp;
  size_t temp_bytes;
};
int64_t plain_query_chunk(uint32_t L, uint32_t R, int64_t nq);
size_t plain_segsort_temp_bytes(int64_t chunk, uint32_t L, uint32_t R);
int launch_plain_query(const PlainQueryLaunch &a, int64_t nq, cudaStream_t stream);

// ---- ADD continued on an existing index (add.cu)
struct AddLaunch {
  const int32_t *old_ids;      // [L][n_old], the index's grouped ids
  const uint32_t *old_starts;  // [L][2^rb + 1]
  int64_t n_old;
  const int32_t *new_ids;      // [L][n_new], the batch grouped by the same sort (ids 0 .. n_new - 1)
  const uint32_t *new_starts;  // [L][2^rb + 1]
  int64_t n_new;
  int32_t *ids;                // [L][n_old + n_new], merged
  uint32_t *starts;            // [L][2^rb + 1], merged
  int32_t id0;                 // id of the batch's first point (n_old)
  uint32_t L, R, range_bits;
  uint64_t rkey;               // reservoir key (Seeds::r)
  unsigned long long *heavy_count;  // 8 bytes of scratch
  uint64_t *heavy;             // buckets with draws, capacity heavy_cap
  int64_t heavy_cap;
};
int launch_add(const AddLaunch &a, cudaStream_t stream);

// ---- quality measures of Section 4.3 by brute force (eval.cu)
struct EvalLaunch {
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t n, dim;
  const int32_t *queries;   // [nq] row ids
  int64_t nq;
  const int32_t *reported;  // [nq][k]
  int32_t k;
  int32_t *nn;              // [nq] nearest neighbour
  double *nn_sim, *sim_at_k;  // [nq]
  uint32_t *mask;           // [dim] scratch
  unsigned long long *best; // [32] scratch
  uint32_t *cand;           // [32][capacity][2] scratch
  uint32_t *ncand;          // [32] scratch
  uint32_t *overflow;       // [1] scratch: a tie list overflowed
  double *cos_slot;         // [32][k] scratch
};
uint32_t eval_candidate_capacity();
int launch_eval(const EvalLaunch &l, cudaStream_t stream);

// ---- dense export of the tables: [L][nb][R] and [L][nb] from starts [L][2^rb + 1]
int launch_export(const int32_t *ids, const uint32_t *starts, int64_t n, uint32_t L, uint32_t R, uint32_t range_bits,
                  uint32_t nb, int32_t *tables, uint32_t *counts, cudaStream_t stream);
// point ids from positions in the row-major (point, table) order of a shared pool: ids[i] /= L
int launch_positions_to_ids(int32_t *ids, int64_t n, uint32_t L, cudaStream_t stream);

}  // namespace flash
