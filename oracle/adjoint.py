"""Gradients through the linear solve x = A^{-1} b (the library's
differentiation form; the paper solves forward only).

With g = dL/dx per right-hand side: lambda = A^{-1} g is dL/db, and since
dx = -A^{-1} dA x, dL/dA = -lambda x^T.  A stored off-diagonal block H = A_rc
also sits transposed at (c, r), so its gradient is -(lambda_r x_c^T +
x_r lambda_c^T); a stored diagonal block appears once: -lambda_r x_r^T.
Right-hand sides add.  Dense solves, for small systems.

Test infrastructure only (see the package docstring).
"""

import numpy as np

from .assembly import to_dense


def solve_dense(n, rid, cid, au, b):
    A = to_dense(n, rid, cid, au)
    return np.linalg.solve(A, np.atleast_2d(b).T).T


def block_gradients(rid, cid, x, lam):
    """dL/dH for every stored block; x, lam of shape (K, n, 3)."""
    x = np.asarray(x).reshape(x.shape[0], -1, 3)
    lam = np.asarray(lam).reshape(lam.shape[0], -1, 3)
    G = -np.einsum("kui,kuj->uij", lam[:, rid], x[:, cid])
    off = rid != cid
    G[off] -= np.einsum("kui,kuj->uij", x[:, rid[off]], lam[:, cid[off]])
    return G


def loss_and_grad(x, x_target):
    """L = sum ||x - x_t||^2 and dL/dx."""
    d = x - x_target
    return float(np.sum(d * d)), 2.0 * d
