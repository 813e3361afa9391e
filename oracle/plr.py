"""Section 5.1: partitioned low-rank (PLR) compression and matrix-vector product.

Test infrastructure: see the package docstring.

Algorithm 5 (compression) recursively splits a block 2 x 2 until its
epsilon-rank is at most r_max; Algorithm 6 applies the resulting quadtree
recursively; the paper then flattens the tree into a "sparse factorization"
(a list of leaves) to avoid recursion.  Readings where the paper is loose:

* threshold: the paper tests the (r_max+1)-th singular value against epsilon;
  here the test is relative, sigma_{r_max+1} < epsilon * sigma_1 with sigma_1
  the largest singular value of the whole uncompressed block, and a leaf keeps
  rank r = #{sigma_i >= epsilon sigma_1} (<= r_max);
* a block with min(m, n) <= r_max is always a leaf (it has no sigma_{r_max+1});
* a leaf whose factors would take at least as much storage as the block
  (r (m + n) >= m n) is stored dense;
* the first half of a split takes ceil(m/2) rows (and ceil(n/2) columns); the
  printed Algorithm 6 overlaps the halves of x by one entry, read here as the
  plain block product y_i = sum_j H_ij x_j.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Node:
    """A PLR node: id 'c' (leaf, data = (U Sigma, V^t) or dense) or 'h' (2 x 2 children)."""

    kind: str
    rows: tuple  # (r0, r1) in the parent block
    cols: tuple
    US: np.ndarray | None = None  # m x r  (U Sigma)
    Vt: np.ndarray | None = None  # r x n
    dense: np.ndarray | None = None
    children: list | None = None


def compress(M: np.ndarray, r_max: int, eps: float, sigma1: float | None = None, r0: int = 0, c0: int = 0) -> Node:
    """Algorithm 5: PLR(M, r_max, eps)."""
    m, n = M.shape
    if sigma1 is None:
        sigma1 = np.linalg.norm(M, 2) if M.size else 0.0
    rows, cols = (r0, r0 + m), (c0, c0 + n)
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    thresh = eps * sigma1
    if min(m, n) <= r_max or s[r_max] < thresh:
        r = int(np.sum(s >= thresh)) if s.size else 0
        r = min(r, r_max)
        if r * (m + n) >= m * n:
            return Node("c", rows, cols, dense=M.copy())
        return Node("c", rows, cols, US=U[:, :r] * s[:r], Vt=Vh[:r])
    mh, nh = (m + 1) // 2, (n + 1) // 2
    kids = []
    for i, (ra, rb) in enumerate(((0, mh), (mh, m))):
        for j, (ca, cb) in enumerate(((0, nh), (nh, n))):
            kids.append(compress(M[ra:rb, ca:cb], r_max, eps, sigma1, r0 + ra, c0 + ca))
    return Node("h", rows, cols, children=kids)


def matvec(H: Node, x: np.ndarray) -> np.ndarray:
    """Algorithm 6: recursive PLR matrix-vector (or matrix-matrix) product; x is local to H."""
    if H.kind == "c":
        if H.dense is not None:
            return H.dense @ x
        return H.US @ (H.Vt @ x)
    m = H.rows[1] - H.rows[0]
    y = np.zeros((m,) + x.shape[1:], dtype=np.result_type(x, np.complex128))
    for child in H.children:
        ra, rb = child.rows[0] - H.rows[0], child.rows[1] - H.rows[0]
        ca, cb = child.cols[0] - H.cols[0], child.cols[1] - H.cols[0]
        y[ra:rb] += matvec(child, x[ca:cb])
    return y


def leaves(H: Node) -> list:
    """The flattened leaf list ("sparse factorization" form of Section 5.1)."""
    if H.kind == "c":
        return [H]
    out = []
    for c in H.children:
        out += leaves(c)
    return out


def leaf_matvec(leaf_list: list, m: int, x: np.ndarray) -> np.ndarray:
    """y = sum over leaves of U_b (V_b^t x_b) (+ dense leaves): the flattened product."""
    y = np.zeros((m,) + x.shape[1:], dtype=np.complex128)
    for lf in leaf_list:
        xs = x[lf.cols[0] : lf.cols[1]]
        if lf.dense is not None:
            y[lf.rows[0] : lf.rows[1]] += lf.dense @ xs
        else:
            y[lf.rows[0] : lf.rows[1]] += lf.US @ (lf.Vt @ xs)
    return y


def compressed_entries(H: Node) -> int:
    """Stored complex entries of a PLR matrix."""
    tot = 0
    for lf in leaves(H):
        tot += lf.dense.size if lf.dense is not None else lf.US.size + lf.Vt.size
    return tot


def to_dense(H: Node) -> np.ndarray:
    m, n = H.rows[1] - H.rows[0], H.cols[1] - H.cols[0]
    A = np.zeros((m, n), dtype=np.complex128)
    for lf in leaves(H):
        blk = lf.dense if lf.dense is not None else lf.US @ lf.Vt
        A[lf.rows[0] - H.rows[0] : lf.rows[1] - H.rows[0], lf.cols[0] - H.cols[0] : lf.cols[1] - H.cols[0]] = blk
    return A
