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
