"""Output selections computed from the oracle's dense trajectory.

TEST INFRASTRUCTURE ONLY: used by the tests, never by the product path.
Plain numpy restatements of the definitions:

- U_sparse / V_sparse (the result slots of Sec. 3.2): a sparse matrix with
  the layout of U (rows node * n_comp + compartment, one column per tspan
  point) or of V (rows node * n_v + index) whose pattern marks where the
  solver writes the state; its values are U's (V's) at those places.  The
  pattern is given in compressed-column form (colptr, row).
- prevalence(cases ~ at_risk, type) (the summary the SISe_sp example of Sec.
  4.2 plots), per replicate and tspan point:
    pop  sum over nodes of the cases / sum over nodes of those at risk;
    nop  nodes with at least one case / nodes with anyone at risk;
    wnp  per node, cases / at risk.
  Reading (the paper defines nop in words only, as the proportion of nodes
  with at least one infected individual): the denominator of nop counts the
  nodes with at least one individual at risk, so empty nodes are not part of
  the population; a zero denominator gives NaN.
"""
import numpy as np


def sparse_values(X, colptr, row, per_node):
    """Values of a dense trajectory X [R][M][Nn][per_node] at the pattern
    (colptr [M + 1], row [nnz]); returns [R][nnz]."""
    colptr = np.asarray(colptr, dtype=np.int64)
    row = np.asarray(row, dtype=np.int64)
    R = X.shape[0]
    out = np.zeros((R, row.size), dtype=X.dtype)
    for m in range(colptr.size - 1):
        for e in range(colptr[m], colptr[m + 1]):
            node, q = divmod(int(row[e]), per_node)
            out[:, e] = X[:, m, node, q]
    return out


def prevalence_counts(U, cases, at_risk):
    """Per replicate and tspan point: (sum of cases, sum at risk, nodes with
    a case, nodes with anyone at risk) for compartment index lists `cases`
    and `at_risk`; returns int64 [R][M][4]."""
    U = np.asarray(U, dtype=np.int64)
    c = U[..., list(cases)].sum(axis=-1)
    r = U[..., list(at_risk)].sum(axis=-1)
    return np.stack([c.sum(axis=-1), r.sum(axis=-1), (c > 0).sum(axis=-1),
                     (r > 0).sum(axis=-1)], axis=-1).astype(np.int64)


def prevalence(U, cases, at_risk, kind="pop"):
    """pop / nop: [R][M]; wnp: [R][M][Nn] (NaN where nobody is at risk)."""
    U = np.asarray(U, dtype=np.int64)
    with np.errstate(invalid="ignore", divide="ignore"):
        if kind == "wnp":
            c = U[..., list(cases)].sum(axis=-1).astype(np.float64)
            r = U[..., list(at_risk)].sum(axis=-1).astype(np.float64)
            return np.where(r > 0, c / np.where(r > 0, r, 1.0), np.nan)
        k = prevalence_counts(U, cases, at_risk).astype(np.float64)
        num, den = (k[..., 0], k[..., 1]) if kind == "pop" else (k[..., 2], k[..., 3])
        if kind not in ("pop", "nop"):
            raise ValueError(kind)
        return np.where(den > 0, num / np.where(den > 0, den, 1.0), np.nan)
