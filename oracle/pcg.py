"""Preconditioned conjugate gradients and the symmetric block SpMV (Sec. 3.2, Sec. 5.3).

PCG solves P d = -grad E (Sec. 3.2) for an SPD P.  The paper's "modified
PCG" of GIPC is not defined in the text; this is textbook PCG with x0 = 0,
r0 = b, stopping when the recurrence residual satisfies
||r_k||_2 <= tol * ||b||_2, the iteration count being the number of
matrix-vector products.  Several right-hand sides run as independent
recurrences.

The SpMV is the product with the full symmetric matrix whose diagonal and
upper blocks are stored (Sec. 5.3, Alg. SRBK): y_r += H x_c for every stored
block H = A_rc and, off the diagonal, y_c += H^T x_r.

Test infrastructure only (see the package docstring).
"""

import numpy as np
import scipy.sparse as sp


class SymmetricMatrix:
    """The full symmetric matrix of the stored diagonal + upper blocks (Sec. 5.3).

    Block (r, c) of the stored list and, off the diagonal, its transpose at
    (c, r) are laid out as a scipy block-sparse (BSR) matrix; ``A @ x`` is
    then the library's sparse product.  x: (3n,) or (3n, k).
    """

    def __init__(self, n, rid, cid, au):
        rid = np.asarray(rid, dtype=np.int64)
        cid = np.asarray(cid, dtype=np.int64)
        au = np.asarray(au, dtype=np.float64).reshape(-1, 3, 3)
        off = rid != cid
        r = np.concatenate([rid, cid[off]])
        c = np.concatenate([cid, rid[off]])
        d = np.concatenate([au, np.swapaxes(au[off], 1, 2)])
        order = np.lexsort((c, r))
        indptr = np.concatenate([[0], np.cumsum(np.bincount(r, minlength=n))])
        self.n = n
        self.A = sp.bsr_matrix((d[order], c[order], indptr), shape=(3 * n, 3 * n), blocksize=(3, 3))

    def __call__(self, x):
        return self.A @ x


def spmv(rid, cid, au, x):
    """y = A x for x of shape (..., V, 3); A given by its stored upper blocks."""
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    rid = np.asarray(rid, dtype=np.int64)
    cid = np.asarray(cid, dtype=np.int64)
    np.add.at(y, (Ellipsis, rid, slice(None)), np.einsum("bij,...bj->...bi", au, x[..., cid, :]))
    off = rid != cid
    np.add.at(
        y,
        (Ellipsis, cid[off], slice(None)),
        np.einsum("bji,...bj->...bi", au[off], x[..., rid[off], :]),
    )
    return y


def pcg(matvec, precond, b, tol=1e-6, max_iter=10_000, fixed_iters=None):
    """PCG on every row of b (shape (K, n)).

    Returns (x, iters, rel_res) with iters the per-RHS matrix-vector product
    count at which ||r|| <= tol ||b|| first held (or max_iter), and rel_res
    the recurrence residual ratio there.  With ``fixed_iters`` every RHS
    runs exactly that many iterations (used to compare two implementations
    along the same Krylov recurrence).
    """
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    K, n = b.shape
    x = np.zeros_like(b)
    iters = np.zeros(K, dtype=np.int64)
    rel = np.zeros(K)
    for k in range(K):
        bn = np.linalg.norm(b[k])
        if bn == 0.0:
            continue
        r = b[k].copy()
        z = precond(r)
        p = z.copy()
        rz = r @ z
        it = 0
        limit = fixed_iters if fixed_iters is not None else max_iter
        while it < limit:
            Ap = matvec(p)
            pAp = p @ Ap
            if pAp <= 0.0:
                raise ValueError("p.Ap <= 0: matrix or preconditioner not SPD")
            alpha = rz / pAp
            x[k] += alpha * p
            r -= alpha * Ap
            it += 1
            if fixed_iters is None and np.linalg.norm(r) <= tol * bn:
                break
            z = precond(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        iters[k] = it
        rel[k] = np.linalg.norm(r) / bn
    return x, iters, rel
