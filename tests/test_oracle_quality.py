"""Pins of the brute-force quality measures (Section 4.3: R@k, S@k) -- CPU only.

Each checks the brute force against a different route (Python set arithmetic,
dense dot products) or a property the measures must have.  The last test runs
the oracle's all-points graph on planted near-duplicates and checks that the
method's lists are far more similar to their queries than random lists.
"""
import math

import numpy as np

import oracle
from oracle import quality
from paper_1709_01190_gb300 import synth


def _rows(rng, n, dim, lo=1, hi=40):
    return [sorted(set(int(x) for x in rng.integers(0, dim, int(rng.integers(lo, hi))))) for _ in range(n)]


def _csr(rows):
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, dtype=np.int64) for r in rows]) if rp[-1] else np.zeros(0, np.int64)
    return rp, col


def test_set_cosine_matches_python_sets():
    rng = np.random.default_rng(1)
    rows = _rows(rng, 60, 200) + [[]]
    rp, col = _csr(rows)
    qs = [0, 5, 17, 60]
    sim = quality.cosine_to_all(rp, col, 200, qs)
    for a, q in enumerate(qs):
        for b, r in enumerate(rows):
            x, y = set(rows[q]), set(r)
            exp = len(x & y) / math.sqrt(len(x) * len(y)) if x and y else 0.0
            assert abs(sim[a, b] - exp) < 1e-12


def test_value_cosine_matches_dense_dot_products_and_ignores_scale():
    rng = np.random.default_rng(2)
    rows = _rows(rng, 40, 100)
    rp, col = _csr(rows)
    val = rng.random(len(col)) + 0.1
    dense = np.zeros((40, 100))
    for i in range(40):
        dense[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    qs = [3, 9]
    sim = quality.cosine_to_all(rp, col, 100, qs, val)
    nrm = np.linalg.norm(dense, axis=1)
    for a, q in enumerate(qs):
        assert np.allclose(sim[a], dense @ dense[q] / (nrm * nrm[q]), atol=1e-12)
    scaled = val * np.repeat(rng.random(40) * 5 + 0.5, np.diff(rp))
    assert np.allclose(quality.cosine_to_all(rp, col, 100, qs, scaled), sim, atol=1e-12)


def test_self_similarity_is_one_and_disjoint_rows_zero():
    rp, col = _csr([[1, 2, 3], [4, 5], [1, 2, 3], [3, 4]])
    sim = quality.cosine_to_all(rp, col, 10, [0, 1])
    assert np.allclose([sim[0, 0], sim[0, 2], sim[0, 1], sim[1, 1]], [1.0, 1.0, 0.0, 1.0], atol=1e-12)
    assert abs(sim[0, 3] - 1 / math.sqrt(6)) < 1e-12


def test_exact_lists_have_full_recall_and_the_highest_similarity():
    rng = np.random.default_rng(3)
    rows = _rows(rng, 300, 80, 3, 20)
    rp, col = _csr(rows)
    qs = np.arange(0, 300, 7)
    sim = quality.cosine_to_all(rp, col, 80, qs)
    nn = quality.nearest_neighbours(sim, qs)
    k = 10
    s = sim.copy()
    s[np.arange(len(qs)), qs] = -np.inf
    exact = np.argsort(-s, axis=1, kind="stable")[:, :k]
    assert quality.recall_at_k(exact, nn) == 1.0
    best = quality.similarity_at_k(exact, sim)
    for trial in range(20):
        other = rng.integers(0, 300, size=(len(qs), k))
        assert quality.similarity_at_k(other, sim) <= best + 1e-12
    # ties go to the smaller id; a missing entry is left out of S@k
    assert nn[0] == np.flatnonzero(s[0] == s[0].max())[0]
    short = exact.copy()
    short[:, 1:] = -1
    assert abs(quality.similarity_at_k(short, sim) - np.mean(sim[np.arange(len(qs)), exact[:, 0]])) < 1e-12


def test_flash_lists_find_planted_near_duplicates():
    """tiny_plain plants clusters of near-duplicates (Jaccard about 0.36 between two of them).
    With K = 2 and L = 64 a pair collides in Binomial(64, J^2) tables (Appendix B; mean about
    8), so the method's top-10 lists hold the nearest neighbour of nearly every query that has
    a near-duplicate (cosine above 0.5), and are far more similar to the query than random lists."""
    w = synth.WORKLOADS["tiny_plain"].scaled(3_000)
    c = synth.generate(w.data)
    ids, _ = oracle.knn_graph(c.row_ptr, c.col, 2, 64, 32, 15, w.params.seed, 10)
    qs = np.arange(0, c.n_rows, 3)
    sim = quality.cosine_to_all(c.row_ptr, c.col, c.dim, qs)
    nn = quality.nearest_neighbours(sim, qs)
    planted = sim[np.arange(len(qs)), nn] > 0.5
    assert planted.sum() >= 100
    assert quality.recall_at_k(ids[qs][planted], nn[planted]) > 0.8
    rng = np.random.default_rng(4)
    rand = rng.integers(0, c.n_rows, size=(len(qs), 10))
    s_flash = quality.similarity_at_k(ids[qs][planted], sim[planted])
    s_random = quality.similarity_at_k(rand[planted], sim[planted])
    assert s_flash > 1.5 * s_random, (s_flash, s_random)


def test_exact_set_nearest_neighbours_agree_with_float_argmax_away_from_ties():
    """The exact nearest neighbour of column sets equals the float64 argmax of the cosines except
    where two cosines are equal as numbers (there the smaller id wins); on these rows, whose
    planted near-duplicates make ties rare, the two agree wherever the best cosine is unique."""
    from oracle import quality
    from paper_1709_01190_gb300 import synth
    c = synth.generate(synth.WORKLOADS["tiny_plain"].data.replace(n_rows=1500, n_clusters=80, seed=3))
    qs = np.arange(0, c.n_rows, 7)
    sim = quality.cosine_to_all(c.row_ptr, c.col, c.dim, qs)
    nn_f = quality.nearest_neighbours(sim, qs)
    nn_x = quality.nearest_neighbours_of_sets(c.row_ptr, c.col, c.dim, qs)
    s2 = sim.copy()
    s2[np.arange(len(qs)), qs] = -np.inf
    best = s2.max(axis=1)
    unique = (np.abs(s2 - best[:, None]) <= 1e-12 * np.maximum(best[:, None], 1e-300)).sum(axis=1) == 1
    assert unique.mean() > 0.5
    assert np.array_equal(nn_f[unique], nn_x[unique])
    # where the best cosine is shared, the exact answer is the smallest id among the tied rows
    for i in np.nonzero(~unique)[0]:
        tied = np.nonzero(np.abs(s2[i] - best[i]) <= 1e-12 * max(best[i], 1e-300))[0]
        assert nn_x[i] == tied.min()


def test_exact_set_nearest_neighbour_tie_goes_to_the_smaller_id():
    """Row 0 shares 2 of its 3 columns with row 1 (4 columns) and 3 with row 2: row 1 wins at 16
    columns for row 2 (c^2/|B| = 1 against 9/16); at 9 columns both have c^2/|B| = 1, cosines equal
    as numbers, and the smaller id wins.  A row sharing no column gets the smallest other id."""
    from oracle import quality
    rows = [[0, 1, 2], [0, 1, 10, 11], [0, 1, 2, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32],
            [100]]
    rp = np.zeros(len(rows) + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.array(r, np.int32) for r in rows])
    # cos(0,1) = 2/sqrt(3*4), cos(0,2) = 3/sqrt(3*16): c^2/|B| = 4/4 = 1 and 9/16 -> row 1 wins
    assert quality.nearest_neighbours_of_sets(rp, col, 200, [0]).tolist() == [1]
    rows[2] = [0, 1, 2, 20, 21, 22, 23, 24, 25]  # c^2/|B| = 9/9 = 1: a tie with row 1
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.array(r, np.int32) for r in rows])
    assert quality.nearest_neighbours_of_sets(rp, col, 200, [0]).tolist() == [1]
    assert quality.nearest_neighbours_of_sets(rp, col, 200, [3]).tolist() == [0]  # no shared column
