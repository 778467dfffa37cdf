// query_noalloc.cu -- flash_query_noalloc: flash_query without any device
// allocation, for callers that must not allocate device memory.
//
// Who needs it: a latency-critical request thread (cudaMalloc can block or
// synchronize the device and can fail under memory pressure in the middle of
// serving), or a host program whose device memory is owned entirely by its
// own pool and which forbids other allocations.  The caller still provides
// the index and every input and output buffer; only the query's scratch
// (bucket addresses of the query rows, two counters, the overflow list)
// lives in a fixed, file-scope device array below.
//
// Properties of that array (every device that loads the library holds it
// until the process exits):
//   * size: kNoAllocScratchBytes (64 MiB); a call whose scratch
//     4*L*q_rows + 8*q_rows + 256 bytes (rounded to 256-byte parts) would
//     exceed it is rejected with FLASH_EINVAL before anything is launched;
//   * shared by every call on that device and keeps the last call's
//     contents: the counters are cleared (cudaMemsetAsync, no allocation)
//     at the start of each call; everything else is overwritten;
//   * calls that overlap on the GPU (different streams, or host threads
//     racing) use the same memory and race: serialize them.
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and caches it; make that first call before any
// stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace flash {
namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

size_t part(size_t bytes) { return (bytes + 255) & ~static_cast<size_t>(255); }

// Device address of g_noalloc_scratch on the current device (looked up once per device).
int scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FLASH_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FLASH_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return 0;
}

}  // namespace
}  // namespace flash

using namespace flash;

extern "C" int flash_query_noalloc(const flash_index *ix, const flash_csr *q, int32_t k, const int32_t *exclude_ids,
                                   int32_t *out_ids, int32_t *out_counts, void *stream) {
  if (!ix || !q || k < 1 || k > 1024) return FLASH_EINVAL;
  if (q->n_rows < 0 || q->nnz < 0 || q->dim < 1 || (q->n_rows > 0 && !q->row_ptr) || (q->nnz > 0 && !q->col))
    return FLASH_EINVAL;
  if ((reinterpret_cast<uintptr_t>(q->row_ptr) & 7u) || (reinterpret_cast<uintptr_t>(q->col) & 3u)) return FLASH_EINVAL;
  if (q->n_rows > 0 && (!out_ids || !out_counts)) return FLASH_EINVAL;
  reset_launch_count();
  if (q->n_rows == 0) return 0;
  const flash_params *p = &ix->p;
  const int64_t nq = q->n_rows;
  const size_t counters_b = part(8 * sizeof(unsigned long long));
  const size_t keys_b = part(sizeof(uint32_t) * static_cast<size_t>(p->L) * static_cast<size_t>(nq));
  const size_t over_b = part(sizeof(int64_t) * static_cast<size_t>(nq));
  if (counters_b + keys_b + over_b > kNoAllocScratchBytes) return FLASH_EINVAL;
  void *base = nullptr;
  if (int rc = scratch_address(&base)) return rc;
  char *b = static_cast<char *>(base);
  unsigned long long *counters = reinterpret_cast<unsigned long long *>(b);
  uint32_t *qkeys = reinterpret_cast<uint32_t *>(b + counters_b);
  int64_t *overflow = reinterpret_cast<int64_t *>(b + counters_b + keys_b);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  DophLaunch d{};
  d.row_ptr = q->row_ptr;
  d.col = q->col;
  d.n_rows = nq;
  d.nnz = q->nnz;
  d.dim = q->dim;
  d.K = p->K;
  d.L = p->L;
  d.range_bits = p->range_bits;
  d.densify = p->densify;
  d.pool = p->share_pool;
  d.pool_bits = ix->pool_bits;
  d.seeds = ix->s;
  d.keys = true;
  d.out = qkeys;
  d.ld = nq;
  d.err = nullptr;  // input errors are skipped safely but not flagged here (the flag word is allocated)
  d.row_counter = counters + 3;
  if (int rc = launch_doph(d, st)) return rc;

  QueryLaunch l{};
  l.qkeys = qkeys;
  l.q_ld = nq;
  l.nq = nq;
  l.ids = ix->ids;
  l.starts = ix->starts;
  l.n = ix->n;
  l.L = p->L;
  l.R = p->R;
  l.range_bits = p->share_pool ? ix->pool_bits : p->range_bits;
  l.shared = p->share_pool != 0;
  l.k = k;
  l.exclude = exclude_ids;
  l.exclude_self = false;
  l.out_ids = out_ids;
  l.out_counts = out_counts;
  l.counters = counters;
  l.overflow = overflow;
  return launch_query(l, st);
}
