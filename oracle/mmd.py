"""Maximum mean discrepancy between two sets of sounds -- TEST INFRASTRUCTURE
(plain numpy, FP64).

The paper measures the similarity of two audio corpora X and Y of n sounds
each by an MMD built directly on a distance d between sounds (Sec. 5, the
MMD equation):

    MMD(X, Y) = 1/(n n) * sum over i, j < n of
                [2 d(x_i, y_j) - d(x_i, x_j) - d(y_i, y_j)],

with d an l1 distance between embeddings of the sounds (the paper's d is
OpenL3 embeddings under l1; the library's own embedding is its log-mel
feature vector). The sums run over all ordered pairs, the diagonal
d(x_i, x_i) = 0 included. For sets of unequal size the same statistic
reads 2/(n_x n_y) sum d(x, y) - 1/n_x^2 sum d(x, x') - 1/n_y^2 sum d(y, y').
Diversity within one corpus is the MMD between the two halves of a random
50/50 partition; between corpora, of n sounds drawn from each; the paper
averages many such trials (Sec. 5).
"""
from __future__ import annotations

import numpy as np


def l1_distances(emb) -> np.ndarray:
    """Pairwise l1 distances d[i][j] = sum_k |e_i[k] - e_j[k]| of the rows
    of emb [m][dim], in FP64."""
    e = np.asarray(emb, dtype=np.float64)
    m = e.shape[0]
    d = np.zeros((m, m))
    for i in range(m):
        d[i] = np.abs(e - e[i]).sum(axis=1)
    return d


def mmd_from_distances(dist, x_idx, y_idx) -> float:
    """The MMD statistic of the index sets x_idx and y_idx (rows of one
    pooled distance matrix)."""
    d = np.asarray(dist, dtype=np.float64)
    x = np.asarray(x_idx)
    y = np.asarray(y_idx)
    nx, ny = len(x), len(y)
    sxy = d[np.ix_(x, y)].sum()
    sxx = d[np.ix_(x, x)].sum()
    syy = d[np.ix_(y, y)].sum()
    return 2.0 * sxy / (nx * ny) - sxx / (nx * nx) - syy / (ny * ny)


def mmd(ex, ey) -> float:
    """The paper's formula written out pair by pair (small sets only)."""
    ex = np.asarray(ex, dtype=np.float64)
    ey = np.asarray(ey, dtype=np.float64)
    n = len(ex)
    assert len(ey) == n
    total = 0.0
    for i in range(n):
        for j in range(n):
            total += (2.0 * np.abs(ex[i] - ey[j]).sum() - np.abs(ex[i] - ex[j]).sum()
                      - np.abs(ey[i] - ey[j]).sum())
    return total / (n * n)


def mmd_trials(dist, labels) -> np.ndarray:
    """One MMD per row of labels [trials][m] (0: in X, 1: in Y, otherwise
    left out) over the pooled distance matrix."""
    lab = np.asarray(labels)
    out = np.zeros(lab.shape[0])
    for t in range(lab.shape[0]):
        out[t] = mmd_from_distances(dist, np.where(lab[t] == 0)[0], np.where(lab[t] == 1)[0])
    return out
