// Seeded synthetic sparse-row generator (CSR) for the FLASH workloads.
//
// This file synthesises inputs only.  It holds none of the method's
// arithmetic (no DOPH, no key map, no reservoir draws); the CPU oracle and
// the CUDA path both consume what it produces.
//
// The paper's datasets (url, webspam, kdd12; Section 4.2, Table 1) are not
// available, so rows are drawn from distributions shaped like them:
//   * row lengths: uniform, clipped lognormal, or Poisson(lambda)+1;
//   * column ids: uniform over [0, D) or Zipf(s) over ranks 1..D, with the
//     rank -> column map a keyed bijection of [0, D) so popular columns are
//     spread over the id range;
//   * optional planted clusters of near-duplicate rows (a fresh seed row,
//     copied, with a fraction of its ids replaced by new draws).
// Within a row, column ids are distinct and sorted ascending.  Every random
// number comes from a counter-based stream keyed by (seed, row), so the
// output does not depend on the number of threads.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---- counter-based generator: Murmur3's 64-bit finalizer over a Weyl sequence
inline uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return k;
}

struct Stream {
  uint64_t state;
  Stream(uint64_t seed, uint64_t domain, uint64_t index) {
    state = fmix64(seed ^ fmix64(domain * 0x632be59bd9b4e019ULL + 0x8cb92ba72f3d8dd7ULL) ^
                   fmix64(index + 0x2545f4914f6cdd1dULL));
  }
  uint64_t next() {
    state += 0xD1B54A32D192ED03ULL;
    return fmix64(state);
  }
  double uniform01() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)
  double uniform_open0() { return ((double)(next() >> 11) + 1.0) * (1.0 / 9007199254740992.0); }  // (0,1]
  uint64_t below(uint64_t n) {  // [0,n), n < 2^32 here (generator only: small bias irrelevant)
    return ((next() >> 32) * n) >> 32;
  }
  double normal() {  // Box-Muller
    double u1 = uniform_open0(), u2 = uniform01();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

enum : uint64_t { DOM_LEN = 1, DOM_IDS = 2, DOM_CLUSTER = 3, DOM_MEMBER = 4, DOM_VAL = 5, DOM_PERM = 6 };

// ---- keyed bijection of [0, n) (4-round Feistel + cycle walking)
struct Bijection {
  uint64_t n;
  int half;
  uint64_t mask;
  uint64_t keys[4];
  Bijection(uint64_t n_, uint64_t seed) : n(n_) {
    int bits = 1;
    while ((1ULL << bits) < n) ++bits;
    half = (bits + 1) / 2;
    mask = (1ULL << half) - 1;
    for (int r = 0; r < 4; ++r) keys[r] = fmix64(seed ^ (0x9d2c5680ULL * (r + 1)));
  }
  uint64_t once(uint64_t x) const {
    uint64_t l = x >> half, r = x & mask;
    for (int k = 0; k < 4; ++k) {
      uint64_t f = fmix64(r ^ keys[k]) & mask;
      uint64_t nl = r, nr = l ^ f;
      l = nl;
      r = nr;
    }
    return (l << half) | r;
  }
  uint64_t operator()(uint64_t x) const {
    do { x = once(x); } while (x >= n);
    return x;
  }
};

// ---- Zipf(s) over ranks {1..n}: rejection-inversion (Hormann & Derflinger,
// ACM TOMACS 1996).  h(x) = x^-s; H is an antiderivative of h.
struct Zipf {
  double s, hx0, hn, squeeze;
  uint64_t n;
  static double helper1(double x) { return std::fabs(x) > 1e-8 ? std::log1p(x) / x : 1.0 - x * (0.5 - x * (1.0 / 3.0 - 0.25 * x)); }
  static double helper2(double x) { return std::fabs(x) > 1e-8 ? std::expm1(x) / x : 1.0 + x * 0.5 * (1.0 + x * (1.0 / 3.0) * (1.0 + 0.25 * x)); }
  double h(double x) const { return std::exp(-s * std::log(x)); }
  double H(double x) const { double lx = std::log(x); return helper2((1.0 - s) * lx) * lx; }
  double Hinv(double y) const {
    double t = y * (1.0 - s);
    if (t < -1.0) t = -1.0;
    return std::exp(helper1(t) * y);
  }
  Zipf(double s_, uint64_t n_) : s(s_), n(n_) {
    hx0 = H(1.5) - 1.0;
    hn = H((double)n + 0.5);
    squeeze = 2.0 - Hinv(H(2.5) - h(2.0));
  }
  uint64_t sample(Stream& rs) const {  // rank in [1, n]
    for (;;) {
      double u = hn + rs.uniform01() * (hx0 - hn);
      double x = Hinv(u);
      double kf = std::floor(x + 0.5);
      if (kf < 1.0) kf = 1.0;
      if (kf > (double)n) kf = (double)n;
      if (kf - x <= squeeze || u >= H(kf + 0.5) - h(kf)) return (uint64_t)kf;
    }
  }
};

}  // namespace

extern "C" {

// Row-length and id distributions.
typedef struct {
  int64_t n_rows;
  int64_t dim;
  int32_t len_kind;  // 0: uniform integer in [len_a, len_b]; 1: lognormal(mu=len_a, sigma=len_b)
                     //    rounded and clipped to [clip_lo, clip_hi]; 2: Poisson(len_a) + 1
  int32_t id_kind;   // 0: uniform over [0, dim); 1: Zipf(zipf_s) over ranks, ranks mapped by a bijection
  double len_a, len_b;
  int64_t clip_lo, clip_hi;
  double zipf_s;
  int64_t n_clusters, cluster_size;  // planted near-duplicate groups (0 = none)
  double resample_frac;              // fraction of a cluster seed row's ids replaced in each member
  uint64_t seed;
} synth_spec;

}  // extern "C"

namespace {

struct Gen {
  const synth_spec& sp;
  Bijection rank_map;
  Bijection row_perm;
  Zipf zipf;
  int64_t n_cluster_rows;
  std::vector<int64_t> cluster_of_row;  // -1 or cluster*cluster_size + member

  explicit Gen(const synth_spec& s)
      : sp(s),
        rank_map((uint64_t)s.dim, fmix64(s.seed ^ 0x5a5a5a5a5a5a5a5aULL)),
        row_perm((uint64_t)(s.n_rows > 0 ? s.n_rows : 1), fmix64(s.seed ^ 0xa5a5a5a5a5a5a5a5ULL)),
        zipf(s.id_kind == 1 ? s.zipf_s : 1.5, (uint64_t)(s.dim > 0 ? s.dim : 1)) {
    n_cluster_rows = s.n_clusters * s.cluster_size;
    if (n_cluster_rows > s.n_rows) n_cluster_rows = s.n_rows;
    cluster_of_row.assign(n_cluster_rows > 0 ? s.n_rows : 0, -1);
    for (int64_t i = 0; i < n_cluster_rows; ++i) cluster_of_row[row_perm((uint64_t)i)] = i;
  }

  int64_t draw_length(Stream& rs) const {
    int64_t n = 0;
    if (sp.len_kind == 0) {
      n = sp.len_a + (int64_t)rs.below((uint64_t)(sp.len_b - sp.len_a + 1));
    } else if (sp.len_kind == 1) {
      double x = std::exp(sp.len_a + sp.len_b * rs.normal());
      double r = std::floor(x + 0.5);
      if (r < (double)sp.clip_lo) r = (double)sp.clip_lo;
      if (r > (double)sp.clip_hi) r = (double)sp.clip_hi;
      n = (int64_t)r;
    } else {
      double lim = std::exp(-sp.len_a), p = 1.0;
      int64_t k = 0;
      do { ++k; p *= rs.uniform01(); } while (p > lim);
      n = (k - 1) + 1;
    }
    if (n > sp.dim) n = sp.dim;
    if (n < 0) n = 0;
    return n;
  }

  uint32_t draw_id(Stream& rs) const {
    if (sp.id_kind == 0) return (uint32_t)rs.below((uint64_t)sp.dim);
    return (uint32_t)rank_map(zipf.sample(rs) - 1);
  }

  // n distinct ids, sorted; excluded ids (sorted) are never produced.
  void distinct_ids(Stream& rs, int64_t n, std::vector<uint32_t>& out, const std::vector<uint32_t>* excl) const {
    out.clear();
    std::vector<uint32_t> fresh;
    while ((int64_t)out.size() < n) {
      fresh.clear();
      for (int64_t i = (int64_t)out.size(); i < n; ++i) fresh.push_back(draw_id(rs));
      out.insert(out.end(), fresh.begin(), fresh.end());
      std::sort(out.begin(), out.end());
      out.erase(std::unique(out.begin(), out.end()), out.end());
      if (excl && !excl->empty()) {
        std::vector<uint32_t> kept;
        kept.reserve(out.size());
        std::set_difference(out.begin(), out.end(), excl->begin(), excl->end(), std::back_inserter(kept));
        out.swap(kept);
      }
    }
  }

  int64_t row_length(int64_t row) const {
    if (n_cluster_rows > 0) {
      int64_t c = cluster_of_row[row];
      if (c >= 0) {
        Stream cs(sp.seed, DOM_CLUSTER, (uint64_t)(c / sp.cluster_size));
        return draw_length(cs);
      }
    }
    Stream rs(sp.seed, DOM_LEN, (uint64_t)row);
    return draw_length(rs);
  }

  void fill_row(int64_t row, int32_t* col, int64_t n, std::vector<uint32_t>& buf, std::vector<uint32_t>& tmp) const {
    int64_t c = n_cluster_rows > 0 ? cluster_of_row[row] : -1;
    if (c < 0) {
      Stream rs(sp.seed, DOM_IDS, (uint64_t)row);
      distinct_ids(rs, n, buf, nullptr);
    } else {
      // seed row of the cluster, shared by every member
      int64_t cl = c / sp.cluster_size, member = c % sp.cluster_size;
      Stream cs(sp.seed, DOM_CLUSTER, (uint64_t)cl);
      int64_t len = draw_length(cs);  // consumes the same numbers as row_length()
      std::vector<uint32_t> seed_ids;
      distinct_ids(cs, len, seed_ids, nullptr);
      // member: replace round(frac*len) ids, chosen by a partial Fisher-Yates
      Stream ms(sp.seed, DOM_MEMBER, (uint64_t)c);
      int64_t nrep = (int64_t)std::floor(sp.resample_frac * (double)len + 0.5);
      std::vector<uint32_t> pool(seed_ids);
      for (int64_t i = 0; i < nrep; ++i) {
        int64_t j = i + (int64_t)ms.below((uint64_t)(len - i));
        std::swap(pool[i], pool[j]);
      }
      std::vector<uint32_t> kept(pool.begin() + nrep, pool.end());
      std::sort(kept.begin(), kept.end());
      // new ids: not in the seed row at all
      distinct_ids(ms, nrep, tmp, &seed_ids);
      buf.clear();
      std::merge(kept.begin(), kept.end(), tmp.begin(), tmp.end(), std::back_inserter(buf));
    }
    for (int64_t i = 0; i < n; ++i) col[i] = (int32_t)buf[i];
  }
};

template <class F>
void parallel_rows(int64_t n, int n_threads, F f) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads == 1 || n < 1024) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=] { f(a, b); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

// Fills row_ptr[0..n_rows] and returns the total nnz (or -1 on bad spec).
int64_t synth_lengths(const synth_spec* sp, int64_t* row_ptr, int n_threads) {
  if (!sp || sp->n_rows < 0 || sp->dim < 1 || sp->dim > 2147483647LL) return -1;
  Gen g(*sp);
  row_ptr[0] = 0;
  parallel_rows(sp->n_rows, n_threads, [&](int64_t a, int64_t b) {
    for (int64_t r = a; r < b; ++r) row_ptr[r + 1] = g.row_length(r);
  });
  for (int64_t r = 0; r < sp->n_rows; ++r) row_ptr[r + 1] += row_ptr[r];
  return row_ptr[sp->n_rows];
}

// Fills col (and val when non-NULL: positive values, unit L2 norm per row).
int synth_fill(const synth_spec* sp, const int64_t* row_ptr, int32_t* col, float* val, int n_threads) {
  if (!sp) return -1;
  Gen g(*sp);
  parallel_rows(sp->n_rows, n_threads, [&](int64_t a, int64_t b) {
    std::vector<uint32_t> buf, tmp;
    for (int64_t r = a; r < b; ++r) {
      int64_t s = row_ptr[r], n = row_ptr[r + 1] - s;
      g.fill_row(r, col + s, n, buf, tmp);
      if (val) {
        Stream vs(sp->seed, DOM_VAL, (uint64_t)r);
        double ss = 0.0;
        for (int64_t i = 0; i < n; ++i) {
          double x = vs.uniform_open0();
          val[s + i] = (float)x;
          ss += x * x;
        }
        double inv = ss > 0.0 ? 1.0 / std::sqrt(ss) : 0.0;
        for (int64_t i = 0; i < n; ++i) val[s + i] = (float)(val[s + i] * inv);
      }
    }
  });
  return 0;
}

// Sample without replacement: out[0..n) = distinct indices of [0, m), keyed by seed.
int synth_sample_rows(int64_t m, int64_t n, uint64_t seed, int64_t* out) {
  if (n > m || n < 0) return -1;
  Bijection b((uint64_t)(m > 0 ? m : 1), fmix64(seed ^ 0x3c3c3c3c3c3c3c3cULL));
  for (int64_t i = 0; i < n; ++i) out[i] = (int64_t)b((uint64_t)i);
  return 0;
}

}  // extern "C"
