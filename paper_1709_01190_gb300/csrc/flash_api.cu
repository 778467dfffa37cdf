// flash_api.cu -- the C ABI declared in include/flash.h: argument checks,
// scratch memory, and the order of kernel launches of every entry point.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace flash {

int num_sms() {
  static thread_local int dev = -1, sms = 0;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return 1;
  if (d != dev) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || sms < 1) sms = 1;
    dev = d;
  }
  return sms;
}

namespace {
thread_local int g_launches = 0;
}
void count_launches(int n) { g_launches += n; }
void reset_launch_count() { g_launches = 0; }

uint32_t *device_error_word() {
  static std::mutex mu;
  static std::map<int, uint32_t *> words;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = words.find(d);
  if (it != words.end()) return it->second;
  uint32_t *p = nullptr;
  if (cudaMalloc(&p, sizeof(uint32_t)) != cudaSuccess) return nullptr;
  if (cudaMemset(p, 0, sizeof(uint32_t)) != cudaSuccess) return nullptr;
  words[d] = p;
  return p;
}

namespace {

std::atomic<size_t> g_scratch_budget{0};

// Optional per-phase timing: when enabled, an event is recorded on the
// call's stream before each phase and at the end; flash_phase_times()
// returns the elapsed milliseconds between consecutive events.
struct PhaseTimer {
  bool enabled = false;
  int n = 0;
  cudaEvent_t ev[8] = {};
  const char *names[8] = {};
  void begin() { n = 0; }
  void mark(const char *name, cudaStream_t s) {
    if (!enabled || n >= 8) return;
    if (!ev[n] && cudaEventCreate(&ev[n]) != cudaSuccess) return;
    names[n] = name;
    cudaEventRecord(ev[n], s);
    ++n;
  }
};
thread_local PhaseTimer g_timer;

// Launch knobs (flash_set_tuning); every call copies them once at its start.
std::mutex g_tuning_mu;
flash_tuning g_tuning = {0, 0, 0};

flash_tuning current_tuning() {
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  return g_tuning;
}

// One stream-ordered allocation carved into 256-byte aligned parts.
// Scratch comes from a stream-ordered pool per device owned by the library,
// which keeps up to a quarter of the device's memory (at least 16 GiB)
// reserved between calls: the device's default pool gives memory back at every
// synchronization, so each call would map its scratch again before its first
// kernel (a 10M-row, L = 256 graph needs about 50 GB of scratch; mapping it
// again cost each call about 50 ms).  Under stream capture the default pool is
// used (graph allocations come from the graph's own memory).
constexpr uint64_t kPoolKeepMin = 16ull << 30;

cudaMemPool_t scratch_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(d);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = d;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    pool = nullptr;
  } else {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      total_b = 0;
    }
    uint64_t keep = total_b / 4 > kPoolKeepMin ? total_b / 4 : kPoolKeepMin;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  pools[d] = pool;
  return pool;
}

class Arena {
 public:
  template <class T>
  void add(T **ptr, int64_t count) {
    parts_.push_back({reinterpret_cast<void **>(ptr), total_});
    total_ += (static_cast<size_t>(count > 0 ? count : 1) * sizeof(T) + 255) & ~static_cast<size_t>(255);
  }
  size_t bytes() const { return total_; }
  int alloc(cudaStream_t s) {
    const size_t cap = g_scratch_budget.load();
    if (cap && total_ > cap) return FLASH_ENOMEM;
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap_status) != cudaSuccess) return FLASH_ECUDA;
    cudaMemPool_t pool = cap_status == cudaStreamCaptureStatusNone ? scratch_pool() : nullptr;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&base_, total_, pool, s) : cudaMallocAsync(&base_, total_, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return FLASH_ENOMEM;
    }
    for (auto &p : parts_) *p.first = static_cast<char *>(base_) + p.second;
    stream_ = s;
    return 0;
  }
  ~Arena() {
    if (base_) cudaFreeAsync(base_, stream_);
  }

 private:
  std::vector<std::pair<void **, size_t>> parts_;
  size_t total_ = 0;
  void *base_ = nullptr;
  cudaStream_t stream_ = nullptr;
};

int check_hash_params(const flash_params *p) {
  if (!p || p->K < 1 || p->L < 1) return FLASH_EINVAL;
  if (p->densify > 1 || p->share_pool > (1u << 30)) return FLASH_EINVAL;
  if (static_cast<uint64_t>(p->K) * p->L > kMaxBins) return FLASH_EINVAL;
  return 0;
}

int check_params(const flash_params *p) {
  if (int rc = check_hash_params(p)) return rc;
  if (p->R < 1 || p->range_bits < 1 || p->range_bits > kMaxRangeBits) return FLASH_EINVAL;
  if (static_cast<uint64_t>(p->L) * p->R > kMaxCandidates) return FLASH_EINVAL;
  if (p->L > kMaxTablesPacked) return FLASH_EINVAL;
  return 0;
}

int check_csr(const flash_csr *x) {
  if (!x || x->n_rows < 0 || x->nnz < 0 || x->dim < 1) return FLASH_EINVAL;
  if (x->n_rows > 0 && !x->row_ptr) return FLASH_EINVAL;
  if (x->nnz > 0 && !x->col) return FLASH_EINVAL;
  // natural alignment of the element types (the kernels find 16-byte boundaries themselves)
  if ((reinterpret_cast<uintptr_t>(x->row_ptr) & 7u) || (reinterpret_cast<uintptr_t>(x->col) & 3u)) return FLASH_EINVAL;
  return 0;
}

DophLaunch doph_args(const flash_params *p, const Seeds &s, const flash_csr *x, bool keys, uint32_t *out, int64_t ld,
                     unsigned long long *counter, const flash_tuning &tu) {
  DophLaunch d{};
  d.rows_per_grab = tu.doph_rows_per_grab;
  d.row_ptr = x->row_ptr;
  d.col = x->col;
  d.n_rows = x->n_rows;
  d.nnz = x->nnz;
  d.dim = x->dim;
  d.K = p->K;
  d.L = p->L;
  d.range_bits = p->range_bits;
  d.densify = p->densify;
  d.pool = p->share_pool;
  d.pool_bits = p->share_pool ? pool_bits_of(p->share_pool) : 0u;
  d.seeds = s;
  d.keys = keys;
  d.out = out;
  d.ld = ld;
  d.err = device_error_word();
  d.row_counter = counter;
  return d;
}

// Optional longest-rows-first order of the rows for the DOPH kernel.
// The DOPH processing order: index order (the default), longest rows first
// (tuning doph_order = 1), or, with allow_long and rows of at least 512
// non-zeros on average, index order after a list of the rows with at least 4x
// the average (rounded up to a power of two), longest class first: one warp
// hashes a row, and a very long row claimed late would outlast the launch
// (webspam-like rows: warps finished at 855 us, the last at 960 us).  The list
// is reserved whenever it is allowed, so that scratch sizes depend on the row
// count alone.
struct RowOrder {
  int32_t *order = nullptr;
  uint32_t *hist = nullptr;
  int32_t *long_rows = nullptr;
  void plan(Arena &ar, const flash_tuning &tu, int64_t n, bool allow_long = false) {
    if (tu.doph_order == 1 && n > 0) {
      ar.add(&order, n);
      ar.add(&hist, 40);
    } else if (allow_long && n > 0) {
      ar.add(&long_rows, n);
      ar.add(&hist, 41);
    }
  }
  int apply(DophLaunch &d, const flash_csr *x, cudaStream_t st) {
    if (order) {
      d.order = order;
      return build_row_order(x->row_ptr, x->n_rows, order, hist, st);
    }
    if (long_rows && x->n_rows > 0 && x->nnz >= 512 * x->n_rows) {
      int64_t long_min = 1;
      while (long_min < 4 * (x->nnz / x->n_rows)) long_min <<= 1;
      uint32_t cmin = 1;  // the log2 class of long_min: floor(log2 m) + 1
      while ((int64_t{1} << (cmin - 1)) < long_min) ++cmin;
      d.long_rows = long_rows;
      d.long_count = hist + 40;
      d.long_min = long_min;
      return build_long_rows(x->row_ptr, x->n_rows, cmin, long_rows, hist, st);
    }
    return 0;
  }
};

// scratch of build: keys, partition ping-pong, histograms, segment starts, heavy list, counters
struct BuildScratch {
  uint32_t *keys = nullptr, *skeys = nullptr, *tkeys = nullptr, *hist = nullptr;
  uint32_t *keys_rm = nullptr;  // row-major addresses (all-points graph; short rows: written first)
  bool transpose = false;       // table-major keys from the row-major ones (short rows)
  int32_t *tids = nullptr, *tids2 = nullptr;
  uint32_t *seg = nullptr;
  uint64_t *heavy = nullptr;
  unsigned long long *counters = nullptr;
  int64_t heavy_cap = 0;
  SortPlan plan{};
  RowOrder ro;
  flash_tuning tu{};
};

// Short rows (fewer non-zeros than tables): DOPH writes the keys row-major
// only, and a tiled transpose makes the table-major copy for the sort.  Written
// directly, the table-major keys of short rows are scattered 4-byte stores
// whose sectors leave L2 half-filled (read-modify-write; 6.6 GB written for
// 2 GB of keys at the kdd12-like shape); long rows amortise them.
void plan_build(Arena &ar, BuildScratch &b, const flash_params *p, int64_t n, int64_t nnz,
                bool rowmajor_keys = false) {
  const int64_t ln = static_cast<int64_t>(p->L) * n;
  b.transpose = nnz < static_cast<int64_t>(p->L) * n;
  if (b.transpose) rowmajor_keys = true;
  b.tu = current_tuning();
  b.ro.plan(ar, b.tu, n, true);
  b.plan = make_sort_plan(p->range_bits, n, p->L);
  b.heavy_cap = reservoir_heavy_capacity(n, p->L, p->R, p->range_bits);
  ar.add(&b.keys, ln);
  if (rowmajor_keys) ar.add(&b.keys_rm, ln);
  ar.add(&b.tkeys, ln);
  ar.add(&b.tids, ln);
  if (b.plan.passes > 1) {
    ar.add(&b.skeys, ln);
    ar.add(&b.tids2, ln);
    ar.add(&b.seg, b.plan.seg_words);
  }
  ar.add(&b.hist, b.plan.hist_words);
  ar.add(&b.heavy, b.heavy_cap);
  ar.add(&b.counters, 8);
}

// Reservoir sharing (p->share_pool = P > 0): one pool of P reservoirs for all
// tables.  The L * n arrivals are sorted as ONE sequence in row-major (point,
// table) order -- Algorithm 2's loop order -- by the reservoir their bucket
// points to (the keys DOPH writes are already pool indices), so a stable sort
// keeps every shared reservoir's arrivals in that order; the sorted entries
// are positions p * L + t, turned into point ids after the reservoir step.
struct SharedScratch {
  uint32_t *keys_rm = nullptr, *tkeys = nullptr, *skeys = nullptr, *hist = nullptr, *seg = nullptr;
  int32_t *tids = nullptr, *tids2 = nullptr;
  uint64_t *heavy = nullptr;
  unsigned long long *counters = nullptr;
  int64_t heavy_cap = 0;
  uint32_t pool_bits = 0;
  SortPlan plan{};
  RowOrder ro;
  flash_tuning tu{};
};

void plan_build_shared(Arena &ar, SharedScratch &b, const flash_params *p, int64_t n) {
  const int64_t ln = static_cast<int64_t>(p->L) * n;
  b.tu = current_tuning();
  b.ro.plan(ar, b.tu, n, true);
  b.pool_bits = pool_bits_of(p->share_pool);
  b.plan = make_sort_plan(b.pool_bits, ln, 1);
  b.heavy_cap = reservoir_heavy_capacity(ln, 1, p->R, b.pool_bits);
  ar.add(&b.keys_rm, ln);
  ar.add(&b.tkeys, ln);
  ar.add(&b.tids, ln);
  if (b.plan.passes > 1) {
    ar.add(&b.skeys, ln);
    ar.add(&b.tids2, ln);
    ar.add(&b.seg, b.plan.seg_words);
  }
  ar.add(&b.hist, b.plan.hist_words);
  ar.add(&b.heavy, b.heavy_cap);
  ar.add(&b.counters, 8);
}

// ids [L * n] and starts [2^pool_bits + 1] of a shared pool
int run_build_shared(const flash_params *p, const Seeds &s, const flash_csr *x, SharedScratch &b, int32_t *ids,
                     uint32_t *starts, cudaStream_t st) {
  const int64_t n = x->n_rows, ln = static_cast<int64_t>(p->L) * n;
  g_timer.mark("hash", st);
  DophLaunch dl = doph_args(p, s, x, true, nullptr, n, b.counters, b.tu);
  dl.out_rowmajor = b.keys_rm;
  int rc = b.ro.apply(dl, x, st);
  if (!rc) rc = launch_doph(dl, st);
  if (rc) return rc;
  g_timer.mark("sort", st);
  SortLaunch sl{};
  sl.keys_in = b.keys_rm;
  sl.n = ln;
  sl.L = 1;
  sl.range_bits = b.pool_bits;
  sl.ids_out = ids;
  sl.tmp_keys = b.tkeys;
  sl.tmp_ids = b.tids;
  sl.keys_out = b.skeys;
  sl.tmp_ids2 = b.tids2;
  sl.hist = b.hist;
  sl.seg = b.seg;
  sl.starts = starts;
  sl.claim = b.counters + 2;
  sl.R = p->R;
  sl.heavy_count = b.counters + 1;
  sl.heavy = b.heavy;
  sl.heavy_cap = b.heavy_cap;
  if ((rc = sort_tables(b.plan, sl, st))) return rc;
  g_timer.mark("reservoir", st);
  ReservoirLaunch rl{};
  rl.ids = ids;
  rl.starts = starts;
  rl.n = ln;
  rl.L = 1;
  rl.R = p->R;
  rl.range_bits = b.pool_bits;
  rl.r = s.r;
  rl.shared = true;
  rl.heavy_count = b.counters + 1;
  rl.heavy = b.heavy;
  rl.heavy_cap = b.heavy_cap;
  rl.heavy_listed = true;
  if ((rc = launch_reservoir(rl, st))) return rc;
  return launch_positions_to_ids(ids, ln, p->L, st);
}

int64_t index_starts_words(const flash_params *p) {
  return p->share_pool ? (1LL << pool_bits_of(p->share_pool)) + 1
                       : static_cast<int64_t>(p->L) * ((1LL << p->range_bits) + 1);
}

// K1 (keys) -> K2 -> K3 into (ids, starts); without K3 when reservoir is false
// (a batch that continues an index: its draws follow the stored counts)
int run_build(const flash_params *p, const Seeds &s, const flash_csr *x, BuildScratch &b, int32_t *ids,
              uint32_t *starts, cudaStream_t st, bool reservoir = true) {
  const int64_t n = x->n_rows;
  g_timer.mark("hash", st);
  DophLaunch dl = doph_args(p, s, x, true, b.transpose ? nullptr : b.keys, n, b.counters, b.tu);
  dl.out_rowmajor = b.keys_rm;
  int rc = b.ro.apply(dl, x, st);
  if (!rc) rc = launch_doph(dl, st);
  if (!rc && b.transpose) rc = launch_transpose_keys(b.keys_rm, n, p->L, b.keys, n, st);
  if (rc) return rc;
  g_timer.mark("sort", st);
  SortLaunch sl{};
  sl.keys_in = b.keys;
  sl.n = n;
  sl.L = p->L;
  sl.range_bits = p->range_bits;
  sl.ids_out = ids;
  sl.tmp_keys = b.tkeys;
  sl.tmp_ids = b.tids;
  sl.keys_out = b.skeys;
  sl.tmp_ids2 = b.tids2;
  sl.hist = b.hist;
  sl.seg = b.seg;
  sl.starts = starts;
  sl.claim = b.counters + 2;
  sl.R = p->R;
  sl.heavy_count = b.counters + 1;
  sl.heavy = b.heavy;
  sl.heavy_cap = b.heavy_cap;
  if ((rc = sort_tables(b.plan, sl, st))) return rc;
  if (!reservoir) return 0;
  g_timer.mark("reservoir", st);
  ReservoirLaunch rl{};
  rl.ids = ids;
  rl.starts = starts;
  rl.n = n;
  rl.L = p->L;
  rl.R = p->R;
  rl.range_bits = p->range_bits;
  rl.r = s.r;
  rl.heavy_count = b.counters + 1;
  rl.heavy = b.heavy;
  rl.heavy_cap = b.heavy_cap;
  rl.heavy_listed = true;
  return launch_reservoir(rl, st);
}

QueryLaunch query_args(const flash_params *p, const uint32_t *qkeys, bool rowmajor, int64_t q_ld, int64_t nq,
                       const int32_t *ids,
                       const uint32_t *starts, int64_t n, int32_t k, const int32_t *exclude, bool exclude_self,
                       int32_t *out_ids, int32_t *out_counts, unsigned long long *counters, int64_t *overflow) {
  QueryLaunch q{};
  q.qkeys = qkeys;
  q.qkeys_rowmajor = rowmajor;
  q.q_ld = q_ld;
  q.nq = nq;
  q.ids = ids;
  q.starts = starts;
  q.n = n;
  q.L = p->L;
  q.R = p->R;
  q.range_bits = p->share_pool ? pool_bits_of(p->share_pool) : p->range_bits;
  q.shared = p->share_pool != 0;
  q.k = k;
  q.exclude = exclude;
  q.exclude_self = exclude_self;
  q.out_ids = out_ids;
  q.out_counts = out_counts;
  q.counters = counters;
  q.overflow = overflow;
  q.warp_table = current_tuning().query_warp_table;
  return q;
}

inline int cuda_ok(cudaError_t e) {
  if (e == cudaSuccess) return 0;
  cudaGetLastError();
  return FLASH_ECUDA;
}

}  // namespace
}  // namespace flash

using namespace flash;

extern "C" {

int flash_hash(const flash_params *p, const flash_csr *x, uint32_t *hashes, void *stream) {
  reset_launch_count();
  if (int rc = check_hash_params(p)) return rc;
  if (int rc = check_csr(x)) return rc;
  if (x->n_rows > 0 && !hashes) return FLASH_EINVAL;
  if (x->n_rows == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const flash_tuning tu = current_tuning();
  Arena ar;
  unsigned long long *counter = nullptr;
  RowOrder ro;
  ar.add(&counter, 1);
  ro.plan(ar, tu, x->n_rows, true);
  if (int rc = ar.alloc(st)) return rc;
  flash_params q = *p;
  q.range_bits = 1;
  DophLaunch dl = doph_args(&q, derive_seeds(p->seed), x, false, hashes, 0, counter, tu);
  if (int rc = ro.apply(dl, x, st)) return rc;
  return launch_doph(dl, st);
}

int flash_keys(const flash_params *p, const flash_csr *x, uint32_t *keys, void *stream) {
  reset_launch_count();
  if (int rc = check_hash_params(p)) return rc;
  if (!p || p->range_bits < 1 || p->range_bits > kMaxRangeBits) return FLASH_EINVAL;
  if (int rc = check_csr(x)) return rc;
  if (x->n_rows > 0 && !keys) return FLASH_EINVAL;
  if (x->n_rows == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const flash_tuning tu = current_tuning();
  // short rows (fewer non-zeros than tables): row-major keys first, then a tiled
  // transpose (the table-major keys of short rows are scattered 4-byte stores)
  const bool transpose = x->nnz < static_cast<int64_t>(p->L) * x->n_rows;
  Arena ar;
  unsigned long long *counter = nullptr;
  uint32_t *rm = nullptr;
  RowOrder ro;
  ar.add(&counter, 1);
  if (transpose) ar.add(&rm, static_cast<int64_t>(p->L) * x->n_rows);
  ro.plan(ar, tu, x->n_rows, true);
  if (int rc = ar.alloc(st)) return rc;
  DophLaunch dl = doph_args(p, derive_seeds(p->seed), x, true, transpose ? nullptr : keys, x->n_rows, counter, tu);
  dl.out_rowmajor = rm;
  if (int rc = ro.apply(dl, x, st)) return rc;
  if (int rc = launch_doph(dl, st)) return rc;
  return transpose ? launch_transpose_keys(rm, x->n_rows, p->L, keys, x->n_rows, st) : 0;
}

int flash_build(const flash_params *p, const flash_csr *x, flash_index **out, void *stream) {
  reset_launch_count();
  if (!out) return FLASH_EINVAL;
  *out = nullptr;
  if (int rc = check_params(p)) return rc;
  if (int rc = check_csr(x)) return rc;
  if (x->n_rows > kMaxPointsPacked) return FLASH_EINVAL;
  if (p->share_pool && static_cast<uint64_t>(p->L) * static_cast<uint64_t>(x->n_rows) > (1ull << 32) - (1ull << 24))
    return FLASH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = x->n_rows;
  flash_index *ix = new (std::nothrow) flash_index();
  if (!ix) return FLASH_ENOMEM;
  ix->p = *p;
  ix->s = derive_seeds(p->seed);
  ix->n = n;
  cudaGetDevice(&ix->device);
  ix->pool_bits = p->share_pool ? pool_bits_of(p->share_pool) : 0u;
  const size_t ids_b = sizeof(int32_t) * static_cast<size_t>(p->L) * static_cast<size_t>(n > 0 ? n : 1);
  const size_t st_b = sizeof(uint32_t) * static_cast<size_t>(index_starts_words(p));
  if (cudaMalloc(&ix->ids, ids_b) != cudaSuccess || cudaMalloc(&ix->starts, st_b) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ix->ids);
    cudaFree(ix->starts);
    delete ix;
    return FLASH_ENOMEM;
  }
  ix->bytes = static_cast<int64_t>(ids_b + st_b);
  int rc = 0;
  if (p->share_pool && n == 0) {
    rc = cuda_ok(cudaMemsetAsync(ix->starts, 0, st_b, st));
  } else if (p->share_pool) {
    Arena ar;
    SharedScratch b;
    plan_build_shared(ar, b, p, n);
    rc = ar.alloc(st);
    if (!rc) rc = run_build_shared(p, ix->s, x, b, ix->ids, ix->starts, st);
  } else {
    Arena ar;
    BuildScratch b;
    plan_build(ar, b, p, n, x->nnz);
    rc = ar.alloc(st);
    if (!rc) rc = run_build(p, ix->s, x, b, ix->ids, ix->starts, st);
  }
  if (rc) {
    cudaStreamSynchronize(st);
    cudaFree(ix->ids);
    cudaFree(ix->starts);
    delete ix;
    return rc;
  }
  *out = ix;
  return 0;
}

int flash_add(flash_index *ix, const flash_csr *x, void *stream) {
  reset_launch_count();
  if (!ix) return FLASH_EINVAL;
  if (int rc = check_csr(x)) return rc;
  if (x->n_rows == 0) return 0;
  if (ix->n + x->n_rows > kMaxPointsPacked) return FLASH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const flash_params *p = &ix->p;
  if (p->share_pool) return FLASH_EINVAL;
  const int64_t n_old = ix->n, n_new = x->n_rows, n = n_old + n_new;
  const int64_t T1 = (1LL << p->range_bits) + 1;
  int cur_dev = 0;
  cudaGetDevice(&cur_dev);
  if (cur_dev != ix->device) return FLASH_EINVAL;
  int32_t *ids = nullptr;
  uint32_t *starts = nullptr;
  const size_t ids_b = sizeof(int32_t) * static_cast<size_t>(p->L) * static_cast<size_t>(n);
  const size_t st_b = sizeof(uint32_t) * static_cast<size_t>(p->L) * static_cast<size_t>(T1);
  if (cudaMalloc(&ids, ids_b) != cudaSuccess || cudaMalloc(&starts, st_b) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ids);
    cudaFree(starts);
    return FLASH_ENOMEM;
  }
  int rc = 0;
  {
    Arena ar;
    BuildScratch b;
    plan_build(ar, b, p, n_new, x->nnz);
    int32_t *bids = nullptr;
    uint32_t *bstarts = nullptr;
    uint64_t *heavy = nullptr;
    unsigned long long *hcount = nullptr;
    const int64_t cap = reservoir_heavy_capacity(n, p->L, p->R, p->range_bits);
    ar.add(&bids, static_cast<int64_t>(p->L) * n_new);
    ar.add(&bstarts, static_cast<int64_t>(p->L) * T1);
    ar.add(&heavy, cap);
    ar.add(&hcount, 1);
    rc = ar.alloc(st);
    if (!rc) rc = run_build(p, ix->s, x, b, bids, bstarts, st, false);
    if (!rc) {
      AddLaunch a{};
      a.old_ids = ix->ids;
      a.old_starts = ix->starts;
      a.n_old = n_old;
      a.new_ids = bids;
      a.new_starts = bstarts;
      a.n_new = n_new;
      a.ids = ids;
      a.starts = starts;
      a.id0 = static_cast<int32_t>(n_old);
      a.L = p->L;
      a.R = p->R;
      a.range_bits = p->range_bits;
      a.rkey = ix->s.r;
      a.heavy_count = hcount;
      a.heavy = heavy;
      a.heavy_cap = cap;
      rc = launch_add(a, st);
    }
  }
  // the old tables are read by the work just queued: wait for it before freeing them
  const int rs = cuda_ok(cudaStreamSynchronize(st));
  if (rc || rs) {
    cudaFree(ids);
    cudaFree(starts);
    return rc ? rc : rs;
  }
  cudaFree(ix->ids);
  cudaFree(ix->starts);
  ix->ids = ids;
  ix->starts = starts;
  ix->n = n;
  ix->bytes = static_cast<int64_t>(ids_b + st_b);
  return 0;
}

int flash_query(const flash_index *ix, const flash_csr *q, int32_t k, const int32_t *exclude_ids, int32_t *out_ids,
                int32_t *out_counts, void *stream) {
  if (!ix || k < 1 || k > 1024) return FLASH_EINVAL;
  reset_launch_count();
  if (int rc = check_csr(q)) return rc;
  if (q->n_rows > 0 && (!out_ids || !out_counts)) return FLASH_EINVAL;
  if (q->n_rows == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const flash_params *p = &ix->p;
  const int64_t nq = q->n_rows;
  const flash_tuning tu = current_tuning();
  Arena ar;
  uint32_t *qkeys = nullptr;
  unsigned long long *counters = nullptr;
  int64_t *overflow = nullptr;
  RowOrder ro;
  ar.add(&qkeys, static_cast<int64_t>(p->L) * nq);
  ar.add(&counters, 8);
  ar.add(&overflow, nq);
  ro.plan(ar, tu, nq);
  if (int rc = ar.alloc(st)) return rc;
  g_timer.begin();
  g_timer.mark("hash", st);
  DophLaunch dl = doph_args(p, ix->s, q, true, nullptr, nq, counters + 3, tu);
  dl.out_rowmajor = qkeys;
  if (int rc = ro.apply(dl, q, st)) return rc;
  if (int rc = launch_doph(dl, st)) return rc;
  g_timer.mark("query", st);
  const int rc = launch_query(query_args(p, qkeys, true, nq, nq, ix->ids, ix->starts, ix->n, k, exclude_ids, false,
                                         out_ids, out_counts, counters, overflow),
                              st);
  g_timer.mark("end", st);
  return rc;
}

int flash_knn_graph(const flash_params *p, const flash_csr *x, int32_t k, int32_t *out_ids, int32_t *out_counts,
                    void *stream) {
  if (int rc = check_params(p)) return rc;
  if (int rc = check_csr(x)) return rc;
  if (k < 1 || k > 1024) return FLASH_EINVAL;
  reset_launch_count();
  if (x->n_rows > kMaxPointsPacked) return FLASH_EINVAL;
  if (x->n_rows > 0 && (!out_ids || !out_counts)) return FLASH_EINVAL;
  if (x->n_rows == 0) return 0;
  if (p->share_pool && static_cast<uint64_t>(p->L) * static_cast<uint64_t>(x->n_rows) > (1ull << 32) - (1ull << 24))
    return FLASH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = x->n_rows;
  const Seeds s = derive_seeds(p->seed);
  if (p->share_pool) {
    Arena ar;
    SharedScratch b;
    plan_build_shared(ar, b, p, n);
    int32_t *ids = nullptr;
    uint32_t *starts = nullptr;
    int64_t *overflow = nullptr;
    ar.add(&ids, static_cast<int64_t>(p->L) * n);
    ar.add(&starts, index_starts_words(p));
    ar.add(&overflow, n);
    if (int rc = ar.alloc(st)) return rc;
    g_timer.begin();
    if (int rc = run_build_shared(p, s, x, b, ids, starts, st)) return rc;
    g_timer.mark("query", st);
    const int rc = launch_query(query_args(p, b.keys_rm, true, n, n, ids, starts, n, k, nullptr, true, out_ids,
                                           out_counts, b.counters + 4, overflow),
                                st);
    g_timer.mark("end", st);
    return rc;
  }
  Arena ar;
  BuildScratch b;
  plan_build(ar, b, p, n, x->nnz, true);
  int32_t *ids = nullptr;
  uint32_t *starts = nullptr;
  int64_t *overflow = nullptr;
  ar.add(&ids, static_cast<int64_t>(p->L) * n);
  ar.add(&starts, static_cast<int64_t>(p->L) * ((1LL << p->range_bits) + 1));
  ar.add(&overflow, n);
  if (int rc = ar.alloc(st)) return rc;
  g_timer.begin();
  if (int rc = run_build(p, s, x, b, ids, starts, st)) return rc;
  g_timer.mark("query", st);
  const int rc = launch_query(query_args(p, b.keys_rm, true, n, n, ids, starts, n, k, nullptr, true, out_ids,
                                         out_counts, b.counters + 4, overflow),
                              st);
  g_timer.mark("end", st);
  return rc;
}

// The plain, unbatched path: the same graph, one launch (or one library sort)
// per stage, no persistent claims, no row order, no tuned knobs.
int flash_knn_graph_plain(const flash_params *p, const flash_csr *x, int32_t k, int32_t *out_ids,
                          int32_t *out_counts, void *stream) {
  if (int rc = check_params(p)) return rc;
  if (int rc = check_csr(x)) return rc;
  if (k < 1 || k > 1024 || p->share_pool) return FLASH_EINVAL;
  reset_launch_count();
  if (x->n_rows > kMaxPointsPacked) return FLASH_EINVAL;
  // the sort keys t * (2^rb + 1) + address must fit 32 bits
  if (static_cast<uint64_t>(p->L) * ((1ull << p->range_bits) + 1) > 0xFFFFFFFFull) return FLASH_EINVAL;
  if (x->n_rows > 0 && (!out_ids || !out_counts)) return FLASH_EINVAL;
  if (x->n_rows == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = x->n_rows, ln = static_cast<int64_t>(p->L) * n;
  const Seeds s = derive_seeds(p->seed);
  const int64_t chunk = plain_query_chunk(p->L, p->R, n);
  const int64_t lr = static_cast<int64_t>(p->L) * p->R;
  Arena ar;
  uint32_t *comp = nullptr, *comp2 = nullptr, *keys_rm = nullptr, *starts = nullptr, *cand = nullptr, *cand2 = nullptr;
  int32_t *ids_in = nullptr, *ids = nullptr;
  int64_t *seg_b = nullptr, *seg_e = nullptr;
  void *temp = nullptr;
  const size_t sort_tb = plain_sort_temp_bytes(n, p->L, p->range_bits);
  const size_t seg_tb = plain_segsort_temp_bytes(chunk, p->L, p->R);
  const size_t tb = sort_tb > seg_tb ? sort_tb : seg_tb;
  ar.add(&comp, ln);
  ar.add(&comp2, ln);
  ar.add(&keys_rm, ln);
  ar.add(&ids_in, ln);
  ar.add(&ids, ln);
  ar.add(&starts, static_cast<int64_t>(p->L) * ((1LL << p->range_bits) + 1));
  ar.add(&cand, chunk * lr);
  ar.add(&cand2, chunk * lr);
  ar.add(&seg_b, chunk);
  ar.add(&seg_e, chunk);
  ar.add(reinterpret_cast<char **>(&temp), static_cast<int64_t>(tb));
  if (int rc = ar.alloc(st)) return rc;
  g_timer.begin();
  g_timer.mark("hash", st);
  PlainHashLaunch h{x->row_ptr, x->col, n, x->nnz, x->dim, p->K * p->L, p->K, p->L, p->range_bits, p->densify, s,
                    comp, keys_rm, device_error_word()};
  if (int rc = launch_plain_keys(h, st)) return rc;
  g_timer.mark("group", st);
  PlainGroupLaunch g{comp, comp2, ids_in, ids, starts, n, p->L, p->R, p->range_bits, s.r, temp, tb};
  if (int rc = launch_plain_group(g, st)) return rc;
  g_timer.mark("query", st);
  PlainQueryLaunch q{};
  q.keys_rm = keys_rm;
  q.ids = ids;
  q.starts = starts;
  q.n = n;
  q.L = p->L;
  q.R = p->R;
  q.range_bits = p->range_bits;
  q.k = k;
  q.exclude = nullptr;
  q.exclude_self = true;
  q.out_ids = out_ids;
  q.out_counts = out_counts;
  q.cand = cand;
  q.cand2 = cand2;
  q.seg_begin = seg_b;
  q.seg_end = seg_e;
  q.temp = temp;
  q.temp_bytes = tb;
  const int rc = launch_plain_query(q, n, st);
  g_timer.mark("end", st);
  return rc;
}

int flash_eval_quality(const flash_csr *x, const int32_t *queries, int64_t nq, const int32_t *reported, int32_t k,
                       int32_t *nn, double *nn_sim, double *sim_at_k, void *stream) {
  reset_launch_count();
  if (int rc = check_csr(x)) return rc;
  if (nq < 0 || k < 1 || (nq > 0 && (!queries || !reported || !nn || !nn_sim || !sim_at_k))) return FLASH_EINVAL;
  if (x->n_rows >= (1LL << 31) || x->dim > 0xFFFFFFFFLL) return FLASH_EINVAL;
  if (nq == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  EvalLaunch l{};
  l.row_ptr = x->row_ptr;
  l.col = x->col;
  l.n = x->n_rows;
  l.dim = x->dim;
  l.queries = queries;
  l.nq = nq;
  l.reported = reported;
  l.k = k;
  l.nn = nn;
  l.nn_sim = nn_sim;
  l.sim_at_k = sim_at_k;
  Arena ar;
  ar.add(&l.mask, x->dim);
  ar.add(&l.best, 32);
  ar.add(&l.cand, 2LL * 32 * eval_candidate_capacity());
  ar.add(&l.ncand, 32);
  ar.add(&l.overflow, 1);
  ar.add(&l.cos_slot, 32LL * k);
  if (int rc = ar.alloc(st)) return rc;
  if (int rc = launch_eval(l, st)) return rc;
  uint32_t over = 0;
  if (cudaMemcpyAsync(&over, l.overflow, sizeof(over), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return FLASH_ECUDA;
  }
  return over ? FLASH_EDATA : 0;
}

// Device address of host memory at p when the device can read it in place
// (memory allocated or registered with CUDA, which has a device mapping);
// null otherwise.
const void *device_view_of_host(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA-known pointer: clear the error
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int flash_knn_graph_host(const flash_params *p, const int64_t *row_ptr, const int32_t *col, int64_t n_rows,
                         int64_t dim, int32_t k, int32_t *out_ids, int32_t *out_counts, void *stream) {
  if (int rc = check_params(p)) return rc;
  if (n_rows < 0 || dim < 1 || k < 1 || k > 1024 || (n_rows > 0 && (!row_ptr || !out_ids || !out_counts)))
    return FLASH_EINVAL;
  if (n_rows == 0) return 0;
  const int64_t nnz = row_ptr[n_rows];
  if (nnz < 0 || (nnz > 0 && !col)) return FLASH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = 0;
  // Pinned (CUDA-allocated or registered) inputs are read by the hashing kernel
  // in place over the host link: the CSR is read exactly once, so a separate
  // copy would only add a pass.  Other host memory is copied first.
  const int64_t *v_rp = static_cast<const int64_t *>(device_view_of_host(row_ptr));
  const int32_t *v_col = nnz > 0 ? static_cast<const int32_t *>(device_view_of_host(col)) : nullptr;
  const bool in_place = v_rp && (nnz == 0 || v_col);
  {
    Arena ar;
    int64_t *d_rp = nullptr;
    int32_t *d_col = nullptr, *d_ids = nullptr, *d_cnt = nullptr;
    if (!in_place) {
      ar.add(&d_rp, n_rows + 1);
      ar.add(&d_col, nnz);
    }
    ar.add(&d_ids, n_rows * k);
    ar.add(&d_cnt, n_rows * k);
    if ((rc = ar.alloc(st))) return rc;
    if (!in_place) {
      rc = cuda_ok(cudaMemcpyAsync(d_rp, row_ptr, sizeof(int64_t) * (n_rows + 1), cudaMemcpyHostToDevice, st));
      if (!rc && nnz > 0) rc = cuda_ok(cudaMemcpyAsync(d_col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
    }
    flash_csr x{in_place ? v_rp : d_rp, in_place ? v_col : d_col, nullptr, n_rows, nnz, dim};
    if (!rc) rc = flash_knn_graph(p, &x, k, d_ids, d_cnt, stream);
    if (!rc) rc = cuda_ok(cudaMemcpyAsync(out_ids, d_ids, sizeof(int32_t) * n_rows * k, cudaMemcpyDeviceToHost, st));
    if (!rc)
      rc = cuda_ok(cudaMemcpyAsync(out_counts, d_cnt, sizeof(int32_t) * n_rows * k, cudaMemcpyDeviceToHost, st));
  }
  const int rs = cuda_ok(cudaStreamSynchronize(st));
  return rc ? rc : rs;
}

void flash_index_free(flash_index *ix) {
  if (!ix) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ix->device);
  cudaFree(ix->ids);
  cudaFree(ix->starts);
  cudaSetDevice(cur);
  delete ix;
}

int flash_index_get_info(const flash_index *ix, flash_index_info *info) {
  if (!ix || !info) return FLASH_EINVAL;
  info->params = ix->p;
  info->n_rows = ix->n;
  info->bytes = ix->bytes;
  return 0;
}

int flash_index_export(const flash_index *ix, int32_t *tables, uint32_t *counts, void *stream) {
  if (!ix || !tables || !counts) return FLASH_EINVAL;
  if (ix->p.share_pool)
    return launch_export(ix->ids, ix->starts, static_cast<int64_t>(ix->p.L) * ix->n, 1, ix->p.R, ix->pool_bits,
                         ix->p.share_pool, tables, counts, static_cast<cudaStream_t>(stream));
  return launch_export(ix->ids, ix->starts, ix->n, ix->p.L, ix->p.R, ix->p.range_bits, 1u << ix->p.range_bits, tables,
                       counts, static_cast<cudaStream_t>(stream));
}

uint32_t flash_device_error(void *stream) {
  uint32_t *w = device_error_word();
  if (!w) return 0xFFFFFFFFu;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return 0xFFFFFFFFu;
  uint32_t v = 0;
  if (cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return 0xFFFFFFFFu;
  if (v) cudaMemset(w, 0, sizeof(uint32_t));
  return v;
}

size_t flash_set_scratch_budget(size_t bytes) { return g_scratch_budget.exchange(bytes); }

size_t flash_knn_graph_scratch_bytes(const flash_params *p, int64_t n_rows) {
  if (check_params(p) || n_rows < 0) return 0;
  Arena ar;
  if (p->share_pool) {
    SharedScratch b;
    plan_build_shared(ar, b, p, n_rows);
  } else {
    BuildScratch b;
    plan_build(ar, b, p, n_rows, static_cast<int64_t>(p->L) * n_rows, true);  // same scratch either way
  }
  int32_t *ids = nullptr;
  uint32_t *starts = nullptr;
  int64_t *overflow = nullptr;
  ar.add(&ids, static_cast<int64_t>(p->L) * n_rows);
  ar.add(&starts, index_starts_words(p));
  ar.add(&overflow, n_rows);
  return ar.bytes();
}

size_t flash_query_scratch_bytes(const flash_params *p, int64_t q_rows) {
  if (check_hash_params(p) || q_rows < 0) return 0;
  // the same carve as flash_query, under the current tuning (the row order adds its scratch)
  Arena ar;
  uint32_t *qkeys = nullptr;
  unsigned long long *counters = nullptr;
  int64_t *overflow = nullptr;
  RowOrder ro;
  ar.add(&qkeys, static_cast<int64_t>(p->L) * q_rows);
  ar.add(&counters, 8);
  ar.add(&overflow, q_rows);
  ro.plan(ar, current_tuning(), q_rows);
  return ar.bytes();
}

const char *flash_strerror(int status) {
  switch (status) {
    case FLASH_OK: return "ok";
    case FLASH_EINVAL: return "invalid or unsupported argument";
    case FLASH_ENOMEM: return "out of device memory or scratch budget";
    case FLASH_ECUDA: return "CUDA runtime error";
    case FLASH_ETIMEOUT: return "bounded device wait expired";
    case FLASH_EDATA: return "invalid input data found on the device";
    default: return "unknown status";
  }
}

int flash_set_tuning(const flash_tuning *t) {
  flash_tuning v = {0, 0, 0};
  if (t) {
    v = *t;
    if (v.query_warp_table && (v.query_warp_table < 64 || v.query_warp_table > 8192 ||
                               (v.query_warp_table & (v.query_warp_table - 1))))
      return FLASH_EINVAL;
    if (v.doph_rows_per_grab > 4096 || v.doph_order > 1) return FLASH_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  g_tuning = v;
  return 0;
}

int flash_get_tuning(flash_tuning *t) {
  if (!t) return FLASH_EINVAL;
  *t = current_tuning();
  return 0;
}

int flash_enable_phase_timing(int on) {
  const int old = g_timer.enabled ? 1 : 0;
  g_timer.enabled = on != 0;
  return old;
}

int flash_phase_times(float *ms, const char **names, int max_phases) {
  PhaseTimer &t = g_timer;
  if (!t.enabled || t.n < 2) return 0;
  if (cudaEventSynchronize(t.ev[t.n - 1]) != cudaSuccess) return -1;
  int m = 0;
  for (int i = 0; i + 1 < t.n && m < max_phases; ++i, ++m) {
    float v = 0.f;
    cudaEventElapsedTime(&v, t.ev[i], t.ev[i + 1]);
    if (ms) ms[m] = v;
    if (names) names[m] = t.names[i];
  }
  return m;
}

int flash_last_launch_count(void) { return g_launches; }

const char *flash_version(void) { return "flash-gb300 0.1 (sm_103a)"; }

}  // extern "C"
