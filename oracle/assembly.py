"""Global Hessian assembly by definition (Sec. 5.1-5.2).

Sec. 5.2 encodes every 3x3 block with a 64-bit key whose high 32 bits are
the first index and whose low 32 bits are the second, sorts the keys so
duplicates become adjacent, and reduces each run (Alg. FastHashReduction,
Alg. FastSegmentReduction).  Whatever the parallel schedule, the result is
fixed: one block per distinct key, equal to the sum of the input blocks
with that key, in ascending key order.  Sec. 5.3 stores only the diagonal
and upper blocks ("Sorted Symmetric Block Coordinates"), so inputs with
row > col describe the implied lower triangle and are not consumed.

Test infrastructure only (see the package docstring).
"""

import numpy as np


def hash_key(r, c):
    """64-bit key: first index in the high 32 bits, second in the low 32 (Sec. 5.2)."""
    return (np.asarray(r, dtype=np.int64) << 32) | np.asarray(c, dtype=np.int64)


def assemble(rows, cols, blocks):
    """Reduce (r, c, 3x3) triplets to sorted upper-triangle blocks.

    Returns (rid, cid, au): int32 block rows / cols and float64 (U, 3, 3)
    blocks, ordered by key (row-major), each the plain sequential sum of
    the inputs sharing that key.  Inputs with r > c are ignored.
    """
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    blocks = np.asarray(blocks, dtype=np.float64).reshape(-1, 3, 3)
    keep = rows <= cols
    keys = hash_key(rows[keep], cols[keep])
    uk, inv = np.unique(keys, return_inverse=True)
    kept = blocks[keep].reshape(-1, 9)
    # per entry: the sum, in input order, of the values sharing a key
    R = np.stack([np.bincount(inv, weights=kept[:, e], minlength=uk.size) for e in range(9)], -1)
    return (uk >> 32).astype(np.int32), (uk & 0xFFFFFFFF).astype(np.int32), R.reshape(-1, 3, 3)


def assemble_dict(rows, cols, blocks):
    """Same result via a Python dict (brute force, for tiny inputs)."""
    acc = {}
    for r, c, b in zip(np.asarray(rows).tolist(), np.asarray(cols).tolist(), np.asarray(blocks)):
        if r > c:
            continue
        acc[(r, c)] = acc.get((r, c), 0.0) + np.asarray(b, dtype=np.float64)
    ks = sorted(acc)
    rid = np.array([k[0] for k in ks], dtype=np.int32)
    cid = np.array([k[1] for k in ks], dtype=np.int32)
    au = np.array([acc[k] for k in ks]).reshape(-1, 3, 3)
    return rid, cid, au


def row_ptr(n_rows, rid):
    """BSR row pointer of the sorted upper blocks: blocks of row r are [ptr[r], ptr[r+1])."""
    counts = np.bincount(rid, minlength=n_rows)
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def to_dense(n_rows, rid, cid, au):
    """Full symmetric dense matrix (3n x 3n) from the stored upper blocks."""
    A = np.zeros((3 * n_rows, 3 * n_rows))
    for r, c, b in zip(rid.tolist(), cid.tolist(), au):
        A[3 * r : 3 * r + 3, 3 * c : 3 * c + 3] += b
        if r != c:
            A[3 * c : 3 * c + 3, 3 * r : 3 * r + 3] += b.T
    return A


def head_segmented_reduce(values, heads, width=32):
    """Semantics of a warp head-segmented reduction (Sec. 5.2's worked example).

    ``values`` and ``heads`` are split into warps of ``width`` lanes; within a
    warp a segment starts at every lane whose head flag is set (lane 0 always
    starts one).  The output at each segment's first lane is the segment sum;
    other lanes hold None.
    """
    values = list(values)
    heads = list(heads)
    out = [None] * len(values)
    for w0 in range(0, len(values), width):
        start = None
        for i in range(w0, min(w0 + width, len(values))):
            if i == w0 or heads[i]:
                start = i
                out[start] = 0
            out[start] = out[start] + values[i]
    return out


def abd_jacobian_weights(xbar):
    """w = [1, xbar_1, xbar_2, xbar_3] so that J = [w_0 I, w_1 I, w_2 I, w_3 I] (Sec. 3.1).

    x_i = A xbar_i + p with q = [p; a_1; a_2; a_3], a_k the columns of A.
    """
    xbar = np.asarray(xbar, dtype=np.float64).reshape(3)
    return np.array([1.0, xbar[0], xbar[1], xbar[2]])


def assemble_abd(rows, cols, blocks, body_of_node, xbar, n_fem):
    """Two-level reduction of mixed FEM / affine-body blocks (Sec. 5.1, Sec. 5.2).

    Full-space node i belongs to affine body body_of_node[i] >= 0, or is a
    FEM vertex (-1).  Block rows of the result: FEM vertex v keeps its index
    (v < n_fem); body b owns block rows n_fem + 4b .. n_fem + 4b + 3 (its 12
    reduced DOFs as four 3-vectors).  Level 1: reduce all 3x3 blocks per node
    pair (r, c).  Level 2: map each reduced pair through the Jacobians,
    J_r^T C J_c, whose (a, b) 3x3 sub-block is w_a(r) w_b(c) C, giving 16,
    4 or 1 sub-blocks (Sec. 5.2's unification), then reduce again by key.
    Inputs are taken as the full symmetric matrix's upper triangle in the
    *full-space* numbering (row <= col); node-pair blocks that map to a lower
    body block position are transposed into the upper triangle.  An index
    n_nodes + 4b + a (n_nodes = len(body_of_node)) is body b's own reduced
    block row a: the 3x3 sub-blocks of a body's 12 x 12 Hessian (Sec. 5.2's
    ABD-ABD block type) pass level 2 unchanged.
    """
    rid1, cid1, c1 = assemble(rows, cols, blocks)
    out_r, out_c, out_b = [], [], []
    body_of_node = np.asarray(body_of_node)
    for r, c, C in zip(rid1.tolist(), cid1.tolist(), c1):
        for sym in ((r, c, C),) if r == c else ((r, c, C), (c, r, C.T)):
            rr, cc, CC = sym
            n_nodes = len(body_of_node)
            br = int(body_of_node[rr]) if rr < n_nodes else None
            bc = int(body_of_node[cc]) if cc < n_nodes else None
            if br is None:
                rows_r, w_r = [n_fem + rr - n_nodes], [1.0]
            elif br < 0:
                rows_r, w_r = [rr], [1.0]
            else:
                rows_r, w_r = [n_fem + 4 * br + a for a in range(4)], abd_jacobian_weights(xbar[rr])
            if bc is None:
                rows_c, w_c = [n_fem + cc - n_nodes], [1.0]
            elif bc < 0:
                rows_c, w_c = [cc], [1.0]
            else:
                rows_c, w_c = [n_fem + 4 * bc + a for a in range(4)], abd_jacobian_weights(xbar[cc])
            for a, R in enumerate(rows_r):
                for b, Cc in enumerate(rows_c):
                    if R <= Cc:
                        out_r.append(R)
                        out_c.append(Cc)
                        out_b.append(w_r[a] * w_c[b] * CC)
    if not out_r:
        return np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros((0, 3, 3))
    return assemble(np.array(out_r), np.array(out_c), np.array(out_b))
