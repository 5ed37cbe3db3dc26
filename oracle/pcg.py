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
