/*
 * flash.h -- C ABI of the GB300 (sm_103a) FLASH hot path.
 *
 * FLASH (Wang, Shrivastava, Wang, Ryu) answers similarity queries over
 * ultra-sparse, ultra-high-dimensional rows without similarity
 * computations: every row is hashed by densified one-permutation minwise
 * hashing (DOPH) into K*L hashes, L hash tables keep a reservoir of at most
 * R point ids per bucket, and a query reports the k ids that occur most
 * often in its L buckets.
 *
 * Conventions shared by every entry point
 *   - Pointers named "device" must be CUDA device (or managed) memory of the
 *     current device; the caller owns them.  Host pointers are named so.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream).  Host-side argument validation happens before
 *     anything is launched; when it fails nothing is launched and an error
 *     code is returned.
 *   - Inputs that can only be checked on the device (column ids outside
 *     [0, dim), row_ptr decreasing or beyond nnz) never cause an
 *     out-of-bounds access: the offending entries are skipped and a sticky
 *     device error flag is raised.  flash_device_error() reads and clears it.
 *   - No call aborts the process.  After an error the output buffers hold
 *     unspecified values.
 *   - Scratch memory is taken from CUDA's stream-ordered allocator
 *     (cudaMallocAsync on `stream`) and returned before the call's work
 *     ends on the stream; flash_set_scratch_budget() caps it.
 *
 * Random choices are fixed functions of flash_params.seed, so results are
 * bit-identical across runs, launch configurations and devices.
 */
#ifndef FLASH_H
#define FLASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
  FLASH_OK = 0,
  FLASH_EINVAL = 1,   /* invalid or unsupported argument (host-side check) */
  FLASH_ENOMEM = 2,   /* device allocation failed or scratch budget exceeded */
  FLASH_ECUDA = 3,    /* a CUDA runtime call failed */
  FLASH_ETIMEOUT = 4, /* reserved: no kernel of this version waits on another, so none is returned */
  FLASH_EDATA = 5     /* invalid input found on the device (see flash_device_error) */
};

/* Device error flag bits reported by flash_device_error(). */
enum {
  FLASH_DEVERR_COL_RANGE = 1u, /* a column id outside [0, dim) was skipped */
  FLASH_DEVERR_ROW_PTR = 2u,   /* a row with end < start or end > nnz was treated as empty */
  FLASH_DEVERR_TIMEOUT = 4u    /* reserved: never raised (no kernel of this version spin-waits) */
};

/* Method parameters (Section 2.2: K hashes per meta-hash, L tables;
 * Section 3.2: reservoirs of size R; Section 4.4.1: 2^range_bits buckets
 * per table).  Limits of the library: K, L, R >= 1; K*L <= 4096;
 * 1 <= range_bits <= 30; L*R <= 16384 (count table of one query); L <= 256
 * and n_rows < 2^24 - 1 for the packed (id, count) query table; with
 * reservoir sharing L * n_rows <= 2^32 - 2^24. */
typedef struct flash_params {
  uint32_t K;
  uint32_t L;
  uint32_t R;
  uint32_t range_bits;
  uint64_t seed;
  /* Densification of the empty bins of a row (Section 2.3): 0 = rotation
   * (Shrivastava & Li 2014: copy the next non-empty bin to the right plus
   * distance * 0x9E3779B9), 1 = optimal densification (the paper's [36]:
   * probe bins by a SplitMix64 mix of (bin, attempt) seeded from `seed`,
   * copy the first non-empty one; after 8*K*L misses copy the next non-empty
   * bin to the right).  Other values are FLASH_EINVAL.  Zero-initialised
   * callers get rotation. */
  uint32_t densify;
  /* Reservoir sharing (Section 3.5): 0 = every bucket has its own reservoir;
   * P > 0 (at most 2^30) = one pool of P reservoirs serves all L tables (the
   * paper's F = P / (L * 2^range_bits)); bucket b of table t points to pool
   * reservoir ((SplitMix64 mix of (t, b) keyed by the seed) * P) >> 32, a
   * shared reservoir receives its arrivals point by point and, for each
   * point, table by table, and a query gathers the reservoir of each of its L
   * buckets.  flash_add and flash_knn_graph_plain do not support it
   * (FLASH_EINVAL); flash_index_export then writes [P][R] and [P]. */
  uint32_t share_pool;
} flash_params;

/* A sparse matrix in CSR form; all pointers are DEVICE pointers.
 *   row_ptr : int64 [n_rows + 1], row r holds entries [row_ptr[r], row_ptr[r+1]);
 *             8-byte aligned
 *   col     : int32 [nnz], column ids in [0, dim); order and repeats within a
 *             row do not matter (a row is the SET of its column ids, Eq. 1);
 *             4-byte aligned (a misaligned pointer is FLASH_EINVAL)
 *   val     : float32 [nnz] or NULL; ignored (DOPH is set-based, Section 2.1)
 *   nnz     : row_ptr[n_rows]; bounds every read of col */
typedef struct flash_csr {
  const int64_t *row_ptr;
  const int32_t *col;
  const float *val;
  int64_t n_rows;
  int64_t nnz;
  int64_t dim;
} flash_csr;

/* Opaque index: the L hash tables of reservoirs built by flash_build. */
typedef struct flash_index flash_index;

typedef struct flash_index_info {
  flash_params params;
  int64_t n_rows;         /* points indexed (row ids 0..n_rows-1) */
  int64_t bytes;          /* device bytes held by the index */
} flash_index_info;

/* DOPH (Section 2.3 on the minwise hash of Eq. 1): K*L hashes per row.
 *   hashes : DEVICE uint32 [n_rows][K*L], row-major.
 * Bin j of row r is the smallest in-bin offset of the row's columns under one
 * permutation split into K*L equal ranges; empty bins are densified as
 * p->densify selects: rotation (first non-empty bin to the right at distance
 * t, plus t*0x9E3779B9) or optimal densification (the first non-empty bin of
 * the bin's own probe sequence, copied).  A row with no entries hashes to
 * 0xFFFFFFFF everywhere. */
int flash_hash(const flash_params *p, const flash_csr *x, uint32_t *hashes, void *stream);

/* MapKHashesToAddress (Section 2.2, Algorithm 2) fused after DOPH: the L
 * bucket addresses of every row.
 *   keys : DEVICE uint32 [L][n_rows] (table-major).  Table t folds the
 *          hashes h[t + j*L], j < K.  A row with no entries gets the value
 *          2^range_bits (it is never inserted into any table). */
int flash_keys(const flash_params *p, const flash_csr *x, uint32_t *keys, void *stream);

/* Adding phase (Algorithm 2 with Algorithm 1's reservoirs): index the rows
 * of x (row id = point id) into L tables of 2^range_bits reservoirs of size
 * R.  Rows arrive in id order; reservoir decisions use a counter-based
 * random number keyed by (seed, table, bucket, arrival rank).
 *   out : receives a library-owned index; free with flash_index_free.
 * The index is complete when the work queued on `stream` completes. */
int flash_build(const flash_params *p, const flash_csr *x, flash_index **out, void *stream);

/* ADD continued (Algorithm 2 is a stream): index the rows of x as new points
 * with ids index->n_rows, index->n_rows + 1, ... .  In every bucket the new
 * points continue the arrival ranks from the bucket's stored count, so the
 * tables afterwards equal those of one flash_build over the old and the new
 * rows together (bit for bit, with the same seed).  The index's tables are
 * replaced by larger ones; the call synchronizes `stream` before it frees the
 * old ones and returns.  FLASH_EINVAL when the index would exceed 2^24 - 2
 * points or belongs to another device than the current one.  On error the
 * index is unchanged. */
int flash_add(flash_index *index, const flash_csr *x, void *stream);

/* Querying phase (Algorithm 3): for every row of q, gather its L buckets,
 * count how often each id occurs and report the k most frequent, ties broken
 * by smaller id.  Missing entries are (-1, 0).  A row with no entries
 * reports nothing.
 *   exclude_ids : DEVICE int32 [q->n_rows] (an id never reported for that
 *                 query, e.g. the query itself) or NULL
 *   out_ids, out_counts : DEVICE int32 [q->n_rows][k] */
int flash_query(const flash_index *index, const flash_csr *q, int32_t k, const int32_t *exclude_ids,
                int32_t *out_ids, int32_t *out_counts, void *stream);

/* flash_query without any device allocation (this entry point has no
 * counterpart in the paper).  For callers that must not allocate device
 * memory -- a latency-critical serving thread, where cudaMalloc can block,
 * synchronize the device or fail under memory pressure, or a program whose
 * device memory belongs entirely to its own pool.  Same arguments and
 * results as flash_query; the caller provides the index and every input and
 * output buffer.  The query's scratch lives in one library-owned device
 * array of 64 MiB per device (held until the process exits); a call needing
 * more (about 4*L*q_rows + 8*q_rows bytes) returns FLASH_EINVAL before
 * launching anything.  All calls on a device share that array and it keeps
 * the last call's contents (the counters are cleared at the start of every
 * call), so calls that overlap on the GPU race: serialize them.  The first
 * call on a device looks the array's device address up; make it before any
 * stream capture.  Invalid input entries are skipped safely but are not
 * reported through flash_device_error(). */
int flash_query_noalloc(const flash_index *index, const flash_csr *q, int32_t k, const int32_t *exclude_ids,
                        int32_t *out_ids, int32_t *out_counts, void *stream);

/* All-points k-NN graph (Section 1 and Section 4.3): build on all rows of x,
 * then query every row against that index excluding itself, reusing the
 * addresses computed for the build.
 *   out_ids, out_counts : DEVICE int32 [n_rows][k] */
int flash_knn_graph(const flash_params *p, const flash_csr *x, int32_t k, int32_t *out_ids, int32_t *out_counts,
                    void *stream);

/* The plain, unbatched GPU path: the same all-points k-NN graph as
 * flash_knn_graph (bit-identical results), computed the straightforward way as
 * a baseline -- one block per row for the hashes, one stable library radix
 * sort for the grouping, Algorithm 1 one thread per bucket, and the query as
 * the paper's own GPU design (Section 3.4.1): gather, segmented sort, count
 * runs, segmented sort by (count, id), first k -- one launch per stage, in
 * chunks of queries.  Needs L * (2^range_bits + 1) <= 2^32.
 *   out_ids, out_counts : DEVICE int32 [n_rows][k] */
int flash_knn_graph_plain(const flash_params *p, const flash_csr *x, int32_t k, int32_t *out_ids,
                          int32_t *out_counts, void *stream);

/* Same as flash_knn_graph with every buffer in HOST memory: the call brings
 * the CSR to the device, runs the graph and copies the results back, then
 * synchronizes `stream`.  Inputs in pinned memory (allocated or registered
 * with CUDA) are read by the hashing kernel in place over the host link;
 * other host memory is first copied to device scratch.  The inputs must not
 * change until the call returns.
 *   row_ptr int64 [n_rows+1], col int32 [nnz] : HOST inputs
 *   out_ids, out_counts int32 [n_rows][k]     : HOST outputs */
int flash_knn_graph_host(const flash_params *p, const int64_t *row_ptr, const int32_t *col, int64_t n_rows,
                         int64_t dim, int32_t k, int32_t *out_ids, int32_t *out_counts, void *stream);

/* Quality measures of Section 4.3 by brute force: for every query row, its
 * nearest neighbour under the cosine of column sets (the gold standard; rows
 * hold distinct column ids; ties to the smaller id; rows without entries have
 * cosine 0 with every row) and the mean cosine of its reported ids.
 *   x                : the indexed rows (DEVICE CSR)
 *   queries          : DEVICE int32 [nq], row ids of x
 *   reported         : DEVICE int32 [nq][k], the ids a query reported (-1 = none)
 *   nn               : DEVICE int32 [nq], the nearest other row
 *   nn_sim, sim_at_k : DEVICE float64 [nq], its cosine, and the mean cosine of
 *                      the reported ids (-1 left out; 0 when none)
 * R@k is then the share of queries whose nn is among their reported ids, S@k
 * the mean of sim_at_k.  Scratch: 4 * dim bytes and a little more.  The call
 * synchronizes `stream`; FLASH_EDATA if some query has more than 512 rows tied
 * (within rounding) for its nearest neighbour. */
int flash_eval_quality(const flash_csr *x, const int32_t *queries, int64_t nq, const int32_t *reported, int32_t k,
                       int32_t *nn, double *nn_sim, double *sim_at_k, void *stream);

/* Release an index (frees its device memory after the work queued on the
 * stream it was built on).  NULL is ignored. */
void flash_index_free(flash_index *index);

int flash_index_get_info(const flash_index *index, flash_index_info *info);

/* Dense copy of the tables, for inspection and tests:
 *   tables : DEVICE int32 [L][2^range_bits][R]; slot s of bucket b of table t;
 *            -1 where the reservoir holds fewer than s+1 ids
 *   counts : DEVICE uint32 [L][2^range_bits]; arrivals per bucket (not capped)
 * With reservoir sharing (share_pool = P): tables [P][R], counts [P], the
 * reservoirs of the pool. */
int flash_index_export(const flash_index *index, int32_t *tables, uint32_t *counts, void *stream);

/* Synchronize `stream`, return the device error flag bits raised since the
 * last call (FLASH_DEVERR_*) and clear them. Returns 0 when clean. */
uint32_t flash_device_error(void *stream);

/* Cap on scratch bytes one call may take (0 = no cap).  Returns the old cap. */
size_t flash_set_scratch_budget(size_t bytes);

/* Scratch bytes flash_knn_graph needs for these sizes (for admission control). */
size_t flash_knn_graph_scratch_bytes(const flash_params *p, int64_t n_rows);

/* Scratch bytes flash_query needs for q_rows query rows. */
size_t flash_query_scratch_bytes(const flash_params *p, int64_t q_rows);

/* Launch knobs chosen by an autotuner (process-wide; every call reads them
 * once when it starts).  Zero means the library's automatic choice.
 *   query_warp_table   : words of the per-warp count table of the query kernel
 *                        (power of two, 64..8192); queries whose candidates do
 *                        not fit go to the block-per-query path
 *   doph_rows_per_grab : rows a warp of the DOPH kernel claims at a time (1..4096)
 *   doph_order         : 0 = rows in index order, 1 = longest rows first
 *                        (rows binned by log2 of their length; results are
 *                        identical, only the schedule changes) */
typedef struct flash_tuning {
  uint32_t query_warp_table;
  uint32_t doph_rows_per_grab;
  uint32_t doph_order;
} flash_tuning;

/* Set the knobs (NULL restores the automatic choices); FLASH_EINVAL if out of range. */
int flash_set_tuning(const flash_tuning *t);
int flash_get_tuning(flash_tuning *t);

/* Per-phase device timing of the calling thread's flash_knn_graph,
 * flash_knn_graph_plain and flash_query calls (instrumentation; off by
 * default).  flash_enable_phase_timing(1) makes later calls record a CUDA
 * event on their stream before each phase (hash, sort, reservoir, query; the
 * plain path: hash, group, query) and at the end; it returns the previous
 * setting.
 * flash_phase_times() waits for the last call's final event and writes up to
 * max_phases durations in milliseconds (ms) and phase names (names, static
 * strings; may be NULL); it returns the number written (0 when disabled). */
int flash_enable_phase_timing(int on);
int flash_phase_times(float *ms, const char **names, int max_phases);

/* Number of CUDA kernels the calling thread's last flash_hash, flash_keys,
 * flash_build, flash_add, flash_query, flash_query_noalloc or flash_knn_graph call
 * launched (memsets of scratch counters are not kernels and are not counted). */
int flash_last_launch_count(void);

/* Human-readable text for a status code. */
const char *flash_strerror(int status);

/* Library version string. */
const char *flash_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FLASH_H */
