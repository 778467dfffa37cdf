"""Quality measures of Section 4.3 (R@k, S@k) by brute force -- TEST INFRASTRUCTURE.

Only ``tests/`` import this module.  It computes exact cosine similarities of
sampled query rows to every row with a sparse matrix product, then:
  R@k : the mean, over the queries, of 1 when the query's nearest neighbour
        (highest cosine among the other rows) is among its k reported ids;
  S@k : the mean, over the queries, of the average cosine of its reported
        ids with the query.
Readings where Section 4.3 is silent: the similarity is the cosine of the
rows' values when they have values, else of their column sets (a row with
no entries has similarity 0 with every row); ties for the nearest neighbour
go to the smaller id; in S@k the missing entries (-1) of a short list are
left out, and a query with no reported id counts 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _matrix(row_ptr, col, val, dim):
    n = len(row_ptr) - 1
    data = np.ones(len(col), dtype=np.float64) if val is None else np.asarray(val, dtype=np.float64)
    m = sp.csr_matrix((data, np.asarray(col, dtype=np.int64), np.asarray(row_ptr, dtype=np.int64)), shape=(n, dim))
    m.sum_duplicates()
    if val is None:
        m.data[:] = 1.0  # a row is the set of its columns
    return m


def cosine_to_all(row_ptr, col, dim, queries, val=None) -> np.ndarray:
    """float64 [len(queries)][n_rows]: cosine of each query row (an index into the rows) with every row."""
    m = _matrix(row_ptr, col, val, dim)
    norm = np.sqrt(np.asarray(m.multiply(m).sum(axis=1)).ravel())
    q = m[np.asarray(queries, dtype=np.int64)]
    dots = (q @ m.T).toarray()
    den = norm[np.asarray(queries, dtype=np.int64)][:, None] * norm[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        sim = np.where(den > 0, dots / np.where(den > 0, den, 1.0), 0.0)
    return sim


def nearest_neighbours(sim, queries) -> np.ndarray:
    """The highest-cosine row other than the query itself (ties: the smaller id)."""
    s = np.array(sim, dtype=np.float64, copy=True)
    s[np.arange(len(queries)), np.asarray(queries, dtype=np.int64)] = -np.inf
    return np.argmax(s, axis=1)


def nearest_neighbours_of_sets(row_ptr, col, dim, queries) -> np.ndarray:
    """nearest_neighbours for the cosine of column sets, with ties decided exactly: the cosine
    c / sqrt(|A| |B|) of two sets sharing c columns orders like c^2 / |B| for a fixed query, so
    rows are compared by integer cross multiplication (Python integers) -- two rows whose cosines
    are equal as numbers are a tie, which goes to the smaller id, whatever float rounding says."""
    m = _matrix(row_ptr, col, None, dim)
    lens = np.asarray(m.getnnz(axis=1), dtype=np.int64)
    q = m[np.asarray(queries, dtype=np.int64)]
    inter = (q @ m.T).tocsr()
    out = np.empty(len(queries), dtype=np.int64)
    for i, qq in enumerate(np.asarray(queries, dtype=np.int64)):
        row = inter.getrow(i)
        best = None  # (c, len, id)
        for r, c in zip(row.indices.tolist(), np.rint(row.data).astype(np.int64).tolist()):
            if r == qq or c <= 0:
                continue
            if best is None or c * c * best[1] > best[0] * best[0] * lens[r] or (
                    c * c * best[1] == best[0] * best[0] * lens[r] and r < best[2]):
                best = (c, int(lens[r]), r)
        out[i] = best[2] if best is not None else (1 if qq == 0 else 0)
    return out


def recall_at_k(ids, nn) -> float:
    """R@k: the share of queries whose nearest neighbour is among their reported ids [nq][k]."""
    ids = np.asarray(ids)
    return float(np.mean([nn[i] in ids[i] for i in range(len(nn))]))


def similarity_at_k(ids, sim) -> float:
    """S@k: the mean over queries of the average cosine of the reported ids (-1 entries left out)."""
    ids = np.asarray(ids)
    out = []
    for i in range(ids.shape[0]):
        got = ids[i][ids[i] >= 0]
        out.append(float(np.mean(sim[i, got])) if len(got) else 0.0)
    return float(np.mean(out))
