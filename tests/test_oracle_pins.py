"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: each checks a property the
paper states (Eq. 1, Eq. 2, Algorithm 1's uniform sample, Section 3.3.2's
binomial count estimator, Appendix B's retrieval probability), a closed form
of a special case, or a brute-force computation of the same definition by a
different route.  CPU only.
"""
import collections
import math
import os

import numpy as np
import pytest

import oracle

C_ROT = 0x9E3779B9
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_of(rows):
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, dtype=np.int32) for r in rows]) if rp[-1] else np.zeros(0, np.int32)
    return rp, col


def rand_set(rng, n, hi=2**31 - 1):
    s = set()
    while len(s) < n:
        s.update(int(x) for x in rng.integers(0, hi, n - len(s)))
    return sorted(s)


# ---------------------------------------------------------------- seeds

def test_seed_words_are_published_splitmix64_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    s = oracle.seeds(0)
    assert [s["a1"], s["b1"], s["a2"], s["b2"], s["r"]] == [vals[0] | 1, vals[1], vals[2] | 1, vals[3], vals[4]]


# ---------------------------------------------------- Eq. 1: minwise hash

def test_minhash_is_a_min_over_elements():
    """B = 1 (K = L = 1): h(x u y) = min(h(x), h(y)) -- the defining property of Eq. 1."""
    rng = np.random.default_rng(1)
    for trial in range(200):
        x = rand_set(rng, int(rng.integers(1, 50)))
        y = rand_set(rng, int(rng.integers(1, 50)))
        u = sorted(set(x) | set(y))
        rp, col = csr_of([x, y, u])
        h = oracle.doph(rp, col, 1, 1, seed=trial)
        assert h[2, 0] == min(h[0, 0], h[1, 0])


def test_oph_bins_are_mins_when_every_bin_is_filled():
    """Rows that fill every bin need no densification: per bin, h_j(x u y) = min(h_j(x), h_j(y))."""
    rng = np.random.default_rng(2)
    for trial in range(20):
        x = rand_set(rng, 3000)
        y = rand_set(rng, 3000)
        u = sorted(set(x) | set(y))
        rp, col = csr_of([x, y, u])
        h = oracle.doph(rp, col, 4, 4, seed=100 + trial)
        assert np.array_equal(h[2], np.minimum(h[0], h[1]))


def test_hash_sees_the_set_only():
    """Order and repetition of the non-zeros do not change any hash (x in {0,1}^D, Eq. 1)."""
    rng = np.random.default_rng(3)
    for trial in range(50):
        x = rand_set(rng, int(rng.integers(1, 300)), hi=10**6)
        shuffled = list(rng.permutation(x)) + list(rng.choice(x, size=min(len(x), 7)))
        rp, col = csr_of([x, shuffled])
        h = oracle.doph(rp, col, 3, 5, seed=trial)
        assert np.array_equal(h[0], h[1])


def _singleton(i, K, L, seed):
    rp, col = csr_of([[i]])
    return oracle.doph(rp, col, K, L, seed)[0]


def _source_bin_of_singleton(h):
    """The only bin s with h[j] = h[s] + ((s - j) mod B) * C for every j (rotation closed form)."""
    B = len(h)
    found = []
    for s in range(B):
        exp = (int(h[s]) + ((s - np.arange(B)) % B) * C_ROT) % 2**32
        if np.array_equal(exp.astype(np.uint32), h):
            found.append(s)
    return found


def test_densification_closed_form_from_singletons():
    """Rotation densification: an empty bin j copies the first non-empty bin to its right at
    distance t and adds t*0x9E3779B9.  Singletons give each element's bin and in-bin value;
    a small set's B hashes must follow from them by min-per-bin + the rotation closed form."""
    K, L = 4, 16
    B = K * L
    rng = np.random.default_rng(4)
    for trial in range(40):
        seed = 7000 + trial
        elems = rand_set(rng, int(rng.integers(1, 6)))
        bins = {}
        for e in elems:
            h1 = _singleton(e, K, L, seed)
            s = _source_bin_of_singleton(h1)
            assert len(s) == 1
            bins.setdefault(s[0], []).append(int(h1[s[0]]))
        v = {s: min(vals) for s, vals in bins.items()}
        exp = np.empty(B, dtype=np.uint32)
        for j in range(B):
            t, src = min(((s - j) % B, s) for s in v)
            exp[j] = (v[src] + t * C_ROT) % 2**32
        rp, col = csr_of([elems])
        assert np.array_equal(oracle.doph(rp, col, K, L, seed)[0], exp)


def _bins_and_values(elems, K, L, seed):
    """Non-empty bin -> its OPH value (min in-bin value), from singletons and the rotation closed form."""
    bins = {}
    for e in elems:
        h1 = _singleton(e, K, L, seed)
        s = _source_bin_of_singleton(h1)
        assert len(s) == 1
        bins.setdefault(s[0], []).append(int(h1[s[0]]))
    return {s: min(vals) for s, vals in bins.items()}


def test_optimal_densification_copies_non_empty_bins():
    """Optimal densification ([36], the variant Section 2.3 cites): a non-empty bin keeps its OPH
    value and an empty bin takes the value of some non-empty bin, unchanged (no offset)."""
    K, L = 4, 16
    B = K * L
    rng = np.random.default_rng(14)
    for trial in range(40):
        seed = 7100 + trial
        elems = rand_set(rng, int(rng.integers(1, 6)))
        v = _bins_and_values(elems, K, L, seed)
        rp, col = csr_of([elems])
        h = oracle.doph(rp, col, K, L, seed, densify=1)[0]
        values = set(v.values())
        for j in range(B):
            if j in v:
                assert h[j] == v[j]
            else:
                assert int(h[j]) in values


def test_optimal_densification_picks_sources_independently_per_bin():
    """Each empty bin draws its source by a hash of (bin, attempt), uniform over the bins: it
    copies each of the f non-empty bins with probability 1/f, independently of its neighbours.
    So the shares p_s of the empty bins copying s have E[sum_s p_s^2] = 1/f + (1 - 1/f)/n_empty,
    and two adjacent empty bins copy the same source with probability sum_s p_s^2 (rotation's
    copies run in long blocks instead: probability near 1)."""
    K, L = 4, 64
    B = K * L
    rng = np.random.default_rng(15)
    same, expect, uniform = [], [], []
    for trial in range(60):
        seed = 7300 + trial
        elems = rand_set(rng, int(rng.integers(2, 6)))
        v = _bins_and_values(elems, K, L, seed)
        if len(set(v.values())) < 2:
            continue
        src_of_value = {val: s for s, val in v.items()}
        rp, col = csr_of([elems])
        h = oracle.doph(rp, col, K, L, seed, densify=1)[0]
        src = [src_of_value[int(x)] for x in h]
        empty = [j for j in range(B) if j not in v]
        share = collections.Counter(src[j] for j in empty)
        p = np.array(list(share.values()), dtype=float) / len(empty)
        pairs = [(j, j + 1) for j in range(B - 1) if j not in v and j + 1 not in v]
        same.append(np.mean([src[a] == src[b] for a, b in pairs]))
        expect.append(float(np.sum(p ** 2)))
        f = len(v)
        uniform.append(1 / f + (1 - 1 / f) / len(empty))
    assert len(same) >= 40
    assert abs(np.mean(expect) - np.mean(uniform)) < 0.05, (np.mean(expect), np.mean(uniform))
    assert abs(np.mean(same) - np.mean(expect)) < 0.08, (np.mean(same), np.mean(expect))


@pytest.mark.parametrize("a_e", [(6, 6), (3, 10)])
def test_optimal_densification_lowers_the_variance_of_the_jaccard_estimate(a_e):
    """[36]'s point: with very sparse rows, rotation copies one non-empty bin into long runs of
    empty ones, so the fraction of matching bins (the estimate of J) varies much more than
    when every empty bin draws its own source.  Both stay unbiased (Eq. 2, pinned above)."""
    a, e = a_e
    rng = np.random.default_rng(20 + a)
    est = {0: [], 1: []}
    for trial in range(300):
        x, y, J = _planted_pair(rng, a, e)
        rp, col = csr_of([x, y])
        for d in (0, 1):
            h = oracle.doph(rp, col, 4, 64, seed=60_000 + trial, densify=d)
            est[d].append(np.mean(h[0] == h[1]))
    assert np.var(est[1]) < np.var(est[0]) / 3, (np.var(est[1]), np.var(est[0]))


def test_optimal_and_rotation_agree_when_every_bin_is_filled():
    """With no empty bin there is nothing to densify: both variants are the OPH bins."""
    rng = np.random.default_rng(16)
    rows = [rand_set(rng, 4000) for _ in range(6)]
    rp, col = csr_of(rows)
    assert np.array_equal(oracle.doph(rp, col, 4, 8, seed=5, densify=0), oracle.doph(rp, col, 4, 8, seed=5, densify=1))


def test_empty_row_hashes_all_ones():
    rp, col = csr_of([[], [5]])
    h = oracle.doph(rp, col, 2, 3, seed=9)
    assert np.all(h[0] == 0xFFFFFFFF)


# ------------------------------------------- Eq. 2: collision = Jaccard

def _planted_pair(rng, a, e):
    pool = rand_set(rng, a + 2 * e)
    rng.shuffle(pool)
    common, ex, ey = pool[:a], pool[a:a + e], pool[a + e:]
    return sorted(common + ex), sorted(common + ey), a / (a + 2 * e)


@pytest.mark.parametrize("dense,densify", [(True, 0), (False, 0), (False, 1)])
@pytest.mark.parametrize("a_e", [(20, 90), (60, 70), (100, 50), (160, 20)])
def test_bin_collision_rate_is_jaccard(dense, densify, a_e):
    """Eq. 2: Pr[h_j(x) = h_j(y)] = J(x, y) for every bin j.  Dense rows (all bins filled)
    check OPH; rows much sparser than B check the densified bins (rotation and optimal
    densification both keep Eq. 2 exact for a random permutation).  Tolerance: 4 standard errors
    of the per-pair mean + 0.01 for the universal hash family standing in for a true permutation."""
    a, e = a_e
    scale = 4 if dense else 0.1
    a, e = max(1, int(a * scale)), max(1, int(e * scale))
    K, L = (4, 8) if dense else (4, 64)
    rng = np.random.default_rng(10 + a + 1000 * e)
    rates, Js = [], []
    for trial in range(300):
        x, y, J = _planted_pair(rng, a, e)
        rp, col = csr_of([x, y])
        h = oracle.doph(rp, col, K, L, seed=50_000 + trial, densify=densify)
        rates.append(np.mean(h[0] == h[1]))
        Js.append(J)
    J = Js[0]
    m, se = np.mean(rates), np.std(rates) / math.sqrt(len(rates))
    assert abs(m - J) <= 4 * se + 0.01, (m, J, se)


@pytest.mark.parametrize("a_e", [(60, 70), (160, 20)])
def test_table_key_collision_rate_is_jaccard_to_the_K(a_e):
    """Section 2.2 / Appendix B: a table address is a function of a K-tuple of hashes, so
    Pr[key_t(x) = key_t(y)] = J^K (+ (1 - J^K) / 2^rb from the universal map)."""
    a, e = a_e
    K, L, rb = 3, 32, 16
    rng = np.random.default_rng(77 + a)
    rates = []
    for trial in range(400):
        x, y, J = _planted_pair(rng, a, e)
        rp, col = csr_of([x, y])
        ks = oracle.keys(rp, col, K, L, rb, seed=90_000 + trial)
        rates.append(np.mean(ks[:, 0] == ks[:, 1]))
    exp = J ** K + (1 - J ** K) / 2 ** rb
    m, se = np.mean(rates), np.std(rates) / math.sqrt(len(rates))
    assert abs(m - exp) <= 4 * se + 0.01, (m, exp, se)


def test_table_keys_are_uniform_over_the_range():
    """The universal map spreads unrelated rows evenly over the 2^rb addresses (chi-square)."""
    from scipy import stats
    rng = np.random.default_rng(5)
    rows = [rand_set(rng, int(rng.integers(5, 40))) for _ in range(20_000)]
    rp, col = csr_of(rows)
    rb = 8
    ks = oracle.keys(rp, col, 2, 4, rb, seed=31)
    for t in range(4):
        obs = np.bincount(ks[t], minlength=2 ** rb)
        assert stats.chisquare(obs).pvalue > 1e-4


# ------------------------------------- Algorithm 1: reservoir sampling

def _stream_trials(m, R, n_trials):
    keys_t = np.zeros(m, dtype=np.uint32)
    rp = np.arange(m + 1, dtype=np.int64)  # every row non-empty
    out = np.empty((n_trials, R), dtype=np.int32)
    for i in range(n_trials):
        res, cnt = oracle.bucket(keys_t, rp, t=i % 97, key=0, R=R, seed=123_456 + i // 97)
        assert cnt == m
        out[i] = res
    return out


def test_reservoir_keeps_every_arrival_while_not_full():
    """m <= R: Algorithm 1's first loop, slots 0..m-1 hold the arrivals in order."""
    for m, R in [(1, 4), (5, 8), (32, 32)]:
        res = _stream_trials(m, R, 5)
        exp = np.full(R, -1, dtype=np.int32)
        exp[:m] = np.arange(m)
        assert np.all(res == exp)


@pytest.mark.parametrize("m,R", [(8, 4), (40, 4), (130, 16)])
def test_reservoir_is_a_uniform_sample(m, R):
    """Section 2.4: the reservoir is a uniform sample, so every arrival is kept with
    probability R/m and every pair with R(R-1)/(m(m-1)).  Chi-square on single inclusions,
    z-test on the (first, last) pair."""
    from scipy import stats
    n = 30_000
    res = _stream_trials(m, R, n)
    assert np.all(res >= 0)
    assert all(len(set(r)) == R for r in res[:1000])
    inc = np.bincount(res.ravel(), minlength=m)
    assert stats.chisquare(inc, f_exp=np.full(m, n * R / m)).pvalue > 1e-4
    both = np.mean(np.any(res == 0, axis=1) & np.any(res == m - 1, axis=1))
    p2 = R * (R - 1) / (m * (m - 1))
    assert abs(both - p2) <= 4.5 * math.sqrt(p2 * (1 - p2) / n)


# ------------------------------------------------ Algorithm 3: KSELECT

def test_kselect_matches_counting_by_dictionary():
    """KSELECT (sort + run-length + sort by value) equals a hash-map count sorted by
    (count desc, id asc), with the excluded id removed and (-1, 0) padding."""
    rng = np.random.default_rng(6)
    for trial in range(300):
        n = int(rng.integers(0, 400))
        A = rng.integers(0, int(rng.integers(1, 60)), n).astype(np.int32)
        excl = int(rng.integers(-1, 5))
        k = int(rng.integers(1, 80))
        ids, cnt = oracle.kselect(A, k, excl)
        c = collections.Counter(int(a) for a in A)
        c.pop(excl, None)
        best = sorted(c.items(), key=lambda kv: (-kv[1], kv[0]))[:k]
        exp_ids = [i for i, _ in best] + [-1] * (k - len(best))
        exp_cnt = [v for _, v in best] + [0] * (k - len(best))
        assert ids.tolist() == exp_ids and cnt.tolist() == exp_cnt


# -------------------------- Algorithms 2 + 3 against brute-force collisions

def _small_workload(n=1500, seed=8):
    from paper_1709_01190_gb300 import synth
    w = synth.WORKLOADS["tiny_plain"]
    spec = w.data.replace(n_rows=n, n_clusters=60, seed=seed)
    return synth.generate(spec, n_threads=2)


def _max_occupancy(ks):
    return int(max(np.bincount(row).max() for row in ks))


def test_tables_hold_whole_buckets_when_R_exceeds_occupancy():
    """R >= every bucket's size: each reservoir is its whole bucket, in point order."""
    c = _small_workload()
    K, L, rb, seed = 2, 6, 10, 4242
    ks = oracle.keys(c.row_ptr, c.col, K, L, rb, seed)
    R = _max_occupancy(ks)
    tables, counts = oracle.build_tables(c.row_ptr, c.col, K, L, R, rb, seed)
    assert counts.max() <= R
    nonempty = np.diff(c.row_ptr) > 0
    for t in range(L):
        for b in np.unique(ks[t]):
            members = np.nonzero((ks[t] == b) & nonempty)[0]
            assert counts[t, b] == len(members)
            assert np.array_equal(tables[t, b, :len(members)], members)
            assert np.all(tables[t, b, len(members):] == -1)
    assert int(counts.sum()) == L * int(nonempty.sum())


def test_counts_are_table_collisions_when_R_exceeds_occupancy():
    """With R >= every bucket's size, count(q, x) = #{t : key_t(q) = key_t(x)} (Section 3.3.2's
    collision count), computed here by comparing key columns directly; the top-k is that count
    vector sorted by (count desc, id asc)."""
    c = _small_workload()
    K, L, rb, seed, k = 2, 12, 9, 99, 40
    ks = oracle.keys(c.row_ptr, c.col, K, L, rb, seed)
    R = _max_occupancy(ks)
    tables, counts = oracle.build_tables(c.row_ptr, c.col, K, L, R, rb, seed)
    assert counts.max() <= R
    n = c.n_rows
    q_ids = np.arange(0, n, 37)
    sub = c.rows(q_ids)
    ids, cnt = oracle.query(tables, counts, K, L, R, rb, seed, sub.row_ptr, sub.col, k, exclude=q_ids)
    nonempty = np.diff(c.row_ptr) > 0
    for qi, q in enumerate(q_ids):
        coll = (ks == ks[:, [q]]).sum(axis=0)
        coll[~nonempty] = 0
        coll[q] = 0
        order = sorted((int(-coll[x]), int(x)) for x in np.nonzero(coll)[0])[:k]
        exp_ids = [x for _, x in order] + [-1] * (k - len(order))
        exp_cnt = [-c_ for c_, _ in order] + [0] * (k - len(order))
        assert ids[qi].tolist() == exp_ids and cnt[qi].tolist() == exp_cnt


def test_candidate_count_total_is_the_gathered_reservoir_size():
    """Sum of all counts = sum over tables of min(bucket size, R), minus the excluded id's hits;
    no count exceeds L."""
    c = _small_workload(n=1200, seed=11)
    K, L, rb, R, seed = 3, 10, 7, 8, 5
    ks = oracle.keys(c.row_ptr, c.col, K, L, rb, seed)
    tables, counts = oracle.build_tables(c.row_ptr, c.col, K, L, R, rb, seed)
    q_ids = np.arange(0, c.n_rows, 29)
    sub = c.rows(q_ids)
    big_k = L * R
    ids, cnt = oracle.query(tables, counts, K, L, R, rb, seed, sub.row_ptr, sub.col, big_k, exclude=q_ids)
    for qi, q in enumerate(q_ids):
        gathered = [tables[t, ks[t, q], :min(int(counts[t, ks[t, q]]), R)] for t in range(L)]
        total = sum(len(g) for g in gathered)
        self_hits = sum(int(np.sum(g == q)) for g in gathered)
        assert int(cnt[qi].sum()) == total - self_hits
        assert cnt[qi].max() <= L


def test_empty_rows_are_not_inserted_and_report_nothing():
    rp, col = csr_of([[1, 2, 3], [], [1, 2, 3], [4]])
    K, L, R, rb, seed = 2, 3, 4, 6, 1
    tables, counts = oracle.build_tables(rp, col, K, L, R, rb, seed)
    assert int(counts.sum()) == L * 3
    assert not np.any(tables == 1)
    ids, cnt = oracle.query(tables, counts, K, L, R, rb, seed, rp, col, 3, exclude=np.arange(4, dtype=np.int32))
    assert ids[1].tolist() == [-1, -1, -1] and cnt[1].tolist() == [0, 0, 0]
    assert ids[0].tolist()[:1] == [2] and cnt[0].tolist()[:1] == [L]


# -------------------- Section 3.3.2 and Appendix B: count statistics

@pytest.mark.parametrize("a_e", [(40, 30), (90, 10)])
def test_mean_count_and_retrieval_follow_appendix_b(a_e):
    """For a planted pair (q, x) with Jaccard J and reservoirs that never overflow, the count of
    x in q's gathered buckets is Binomial(L, J^K) (Section 3.3.2), so its mean is L*J^K and
    Pr[x retrieved] = 1 - (1 - J^K)^L (Appendix B with every alpha_i = 1)."""
    a, e = a_e
    K, L, R, rb = 2, 16, 64, 16
    rng = np.random.default_rng(a * 7 + e)
    counts_seen, retrieved = [], []
    J = None
    for trial in range(300):
        x, y, J = _planted_pair(rng, a, e)
        noise = [rand_set(rng, a + e) for _ in range(4)]
        rows = [x, y] + noise
        rp, col = csr_of(rows)
        tables, counts = oracle.build_tables(rp, col, K, L, R, rb, seed=3_000 + trial)
        ids, cnt = oracle.query(tables, counts, K, L, R, rb, 3_000 + trial, rp[:2], col[:len(x)], 6,
                                exclude=np.array([0], dtype=np.int32))
        row = dict(zip(ids[0].tolist(), cnt[0].tolist()))
        c_ = row.get(1, 0)
        counts_seen.append(c_)
        retrieved.append(c_ > 0)
    p = J ** K
    m = np.mean(counts_seen)
    assert abs(m - L * p) <= 4 * math.sqrt(L * p * (1 - p) / len(counts_seen)) + 0.02 * L
    pr = 1 - (1 - p) ** L
    assert abs(np.mean(retrieved) - pr) <= 4 * math.sqrt(pr * (1 - pr) / len(retrieved)) + 0.02


# ------------------------------------------------------ internal consistency

def test_streamed_buckets_and_queries_equal_the_full_build():
    c = _small_workload(n=900, seed=12)
    K, L, rb, R, seed, k = 3, 8, 6, 4, 77, 12
    ks = oracle.keys(c.row_ptr, c.col, K, L, rb, seed)
    tables, counts = oracle.build_tables(c.row_ptr, c.col, K, L, R, rb, seed)
    for t in range(L):
        for b in range(0, 2 ** rb, 5):
            res, cnt = oracle.bucket(ks[t], c.row_ptr, t, b, R, seed)
            assert cnt == counts[t, b] and np.array_equal(res, tables[t, b])
    ids, cnt = oracle.knn_graph(c.row_ptr, c.col, K, L, R, rb, seed, k)
    for q in range(0, c.n_rows, 53):
        i2, c2 = oracle.query_streamed(ks, c.row_ptr, L, R, seed, ks[:, q], c.row_ptr[q + 1] == c.row_ptr[q], k, q)
        assert np.array_equal(i2, ids[q]) and np.array_equal(c2, cnt[q])


# -------------------------------- one permutation split into B ranges

def test_oph_bins_split_one_permutation_into_equal_ranges():
    """One-permutation hashing (Section 2.3): the B bins are B equal consecutive ranges of ONE
    permutation.  With B = 1 a singleton's hash is its permuted position pi (Eq. 1); with B bins
    the same element must sit in bin floor(pi*B / 2^32) at in-bin position (pi*B) mod 2^32."""
    rng = np.random.default_rng(14)
    for trial in range(60):
        seed = 11_000 + trial
        i = int(rng.integers(0, 2**31 - 1))
        pi = int(_singleton(i, 1, 1, seed)[0])
        for K, L in [(1, 3), (4, 16), (3, 128)]:
            h = _singleton(i, K, L, seed)
            s = _source_bin_of_singleton(h)
            B = K * L
            assert s == [(pi * B) >> 32]
            assert int(h[s[0]]) == (pi * B) % 2**32


def test_each_column_lands_in_a_uniform_bin_over_seeds():
    """pi is a random permutation (Section 2.1): over seeds, any fixed column -- including
    column 0 -- falls into each of the B bins equally often (chi-square)."""
    from scipy import stats
    K, L = 2, 4
    B = K * L
    for col in [0, 1, 2, 12345, 2**31 - 2]:
        bins = [_source_bin_of_singleton(_singleton(col, K, L, seed))[0] for seed in range(1600)]
        assert stats.chisquare(np.bincount(bins, minlength=B)).pvalue > 1e-4


def test_address_map_is_universal_on_k_tuples():
    """MapKHashesToAddress is a universal random map of the K-tuple (Section 2.2): over seeds,
    two different tuples share an address with probability about 2^-rb -- also when one tuple
    is a reordering of the other or differs in a single coordinate."""
    K, L, rb = 4, 3, 6
    B = K * L
    rng = np.random.default_rng(15)
    n_seeds = 3000
    pairs = []
    for _ in range(6):
        h = rng.integers(0, 2**32, B, dtype=np.uint64).astype(np.uint32)
        g = h.copy()
        idx = [1 + j * L for j in range(K)]          # table 1's tuple, reordered
        g[idx] = h[idx[::-1]]
        pairs.append((h, g))
        g2 = h.copy()
        g2[1 + 2 * L] ^= np.uint32(1)                # one coordinate, one bit
        pairs.append((h, g2))
        g3 = h.copy()
        g3[1] = np.uint32((int(h[1]) + 1) % 2**32)   # first coordinate + 1
        pairs.append((h, g3))
    for h, g in pairs:
        same = sum(oracle.address(h, 1, K, L, rb, s) == oracle.address(g, 1, K, L, rb, s) for s in range(n_seeds))
        p = 2.0 ** -rb
        assert same <= n_seeds * 2 * p + 4 * math.sqrt(n_seeds * 2 * p), same


def test_adding_in_batches_continues_every_bucket_stream():
    """Algorithm 2 is a stream: tables built from the first rows, then extended by ADD with the
    rest (point ids continuing), equal the tables of one build over all rows -- the arrival
    counts continue, so every later reservoir draw uses the same rank as in one pass."""
    from paper_1709_01190_gb300 import synth
    w = synth.WORKLOADS["tiny_plain"].scaled(2_000)
    c = synth.generate(w.data)
    K, L, R, rb, seed = 3, 8, 4, 6, 11  # few buckets: every reservoir overflows
    et, ec = oracle.build_tables(c.row_ptr, c.col, K, L, R, rb, seed)
    for cut in (1, 700, 1999):
        t, n = oracle.build_tables(c.row_ptr[:cut + 1], c.col[:c.row_ptr[cut]], K, L, R, rb, seed)
        rp2 = c.row_ptr[cut:] - c.row_ptr[cut]
        oracle.add_rows(t, n, rp2, c.col[c.row_ptr[cut]:], cut, K, L, R, rb, seed)
        assert np.array_equal(t, et) and np.array_equal(n, ec), cut
    assert ec.max() > 4 * R


# ----------------------------------------- reservoir sharing (Section 3.5)

def test_shared_pool_map_is_uniform_and_independent_across_tables():
    """Each bucket points to a uniformly random reservoir of the pool (chi-square over the pool), and
    the reservoirs two tables pick for the same address are independent (chi-square over pairs)."""
    from scipy import stats
    P = 37
    cells = np.zeros(P, dtype=np.int64)
    pairs = np.zeros((P, P), dtype=np.int64)
    for b in range(4000):
        x0 = oracle.pool_index(0, b, P, 77)
        x1 = oracle.pool_index(5, b, P, 77)
        cells[x0] += 1
        cells[x1] += 1
        pairs[x0, x1] += 1
    assert cells.min() >= 0 and int(cells.sum()) == 8000
    assert stats.chisquare(cells).pvalue > 1e-4
    small = np.zeros((6, 6), dtype=np.int64)  # pairs folded into 6 x 6 cells of ~equal mass
    for i in range(P):
        for j in range(P):
            small[i * 6 // P, j * 6 // P] += pairs[i, j]
    exp = np.outer(np.bincount(np.arange(P) * 6 // P, minlength=6), np.bincount(np.arange(P) * 6 // P,
                                                                               minlength=6)) * 4000 / P / P
    assert stats.chisquare(small.ravel(), f_exp=exp.ravel() * small.sum() / exp.sum()).pvalue > 1e-4


def test_shared_reservoirs_receive_arrivals_point_by_point_then_table_by_table():
    """R above every shared reservoir's size: reservoir x holds exactly the (point, table) arrivals
    whose bucket points to x, in Algorithm 2's loop order (points in id order, tables in order),
    found here by enumerating the keys; every arrival lands in one reservoir."""
    c = _small_workload(n=900, seed=13)
    K, L, rb, seed, P = 2, 5, 8, 31, 600
    ks = oracle.keys(c.row_ptr, c.col, K, L, rb, seed)
    nonempty = np.diff(c.row_ptr) > 0
    streams = collections.defaultdict(list)
    for p in range(c.n_rows):
        if not nonempty[p]:
            continue
        for t in range(L):
            streams[oracle.pool_index(t, int(ks[t, p]), P, seed)].append(p)
    R = max(len(v) for v in streams.values())
    tables, counts = oracle.build_tables_shared(c.row_ptr, c.col, K, L, R, rb, seed, P)
    assert int(counts.sum()) == L * int(nonempty.sum())
    for x in range(P):
        got = tables[x]
        exp = streams.get(x, [])
        assert counts[x] == len(exp)
        assert got[:len(exp)].tolist() == exp and np.all(got[len(exp):] == -1)


def test_one_shared_reservoir_closed_form():
    """P = 1 with R above L * (non-empty rows): the one reservoir holds every point L times in a
    row, and every query gathers it L times, so every other non-empty point counts L^2; the top-k
    is the smallest such ids."""
    c = _small_workload(n=60, seed=5)
    K, L, rb, seed, k = 2, 3, 6, 9, 12
    nonempty = np.nonzero(np.diff(c.row_ptr) > 0)[0]
    R = L * len(nonempty)
    tables, counts = oracle.build_tables_shared(c.row_ptr, c.col, K, L, R, rb, seed, 1)
    assert tables[0].tolist() == np.repeat(nonempty, L).tolist() and counts[0] == R
    q = np.array([int(nonempty[3]), int(nonempty[0])])
    sub = c.rows(q)
    ids, cnt = oracle.query_shared(tables, counts, K, L, R, rb, seed, 1, sub.row_ptr, sub.col, k,
                                   exclude=q.astype(np.int32))
    for i, qq in enumerate(q):
        exp = [int(x) for x in nonempty if x != qq][:k]
        assert ids[i].tolist() == exp + [-1] * (k - len(exp))
        assert cnt[i].tolist() == [L * L] * len(exp) + [0] * (k - len(exp))


def test_collision_free_pool_changes_nothing():
    """A pool so large that no two used buckets share a reservoir, with R above every occupancy:
    every query gathers exactly the unshared index's buckets, so the graphs agree."""
    c = _small_workload(n=700, seed=21)
    K, L, rb, k = 2, 6, 7, 15
    P = 2**20
    for seed in range(50, 80):  # a seed whose used buckets map to distinct reservoirs
        ks = oracle.keys(c.row_ptr, c.col, K, L, rb, seed)
        used = {(t, int(b)) for t in range(L) for b in np.unique(ks[t])}
        if len({oracle.pool_index(t, b, P, seed) for t, b in used}) == len(used):
            break
    else:
        pytest.fail("no collision-free seed")
    R = _max_occupancy(ks)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, K, L, R, rb, seed, k)
    si, sn = oracle.knn_graph_shared(c.row_ptr, c.col, K, L, R, rb, seed, k, P)
    assert np.array_equal(ei, si) and np.array_equal(en, sn)
