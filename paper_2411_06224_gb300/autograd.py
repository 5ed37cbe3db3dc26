"""torch.autograd through the solve x = A^{-1} b (the library's differentiation form).

``solve(blocks, b, system)`` assembles the triplet values ``blocks`` on the
pattern held by ``system``, builds the MAS preconditioner, and solves for
every row of ``b``.  Its backward pass is one call to ``gs_adjoint``: a
second MAS-PCG solve lambda = A^{-1} dL/dx (= dL/db) and the block-sparse
outer products that give dL/d(blocks).  All arithmetic runs in the CUDA
library; this module only passes tensors and handles.
"""

import numpy as np
import torch

from . import binding as B


class System:
    """The parts of a Newton system that do not carry gradients: the block
    pattern (rows, cols), the mesh graph and contacts, the level-0 partition
    and the solver options.  Integer tensors live on the GPU."""

    def __init__(self, ctx, n, rows, cols, X, adj_ptr, adj, contacts=None, domain_size=32, max_levels=3,
                 precision=B.GS_PREC_FP64, tol=1e-10, mixed=False, max_iter=20_000, device="cuda"):
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.int32, device=device)
        self.ctx = ctx
        self.n = int(n)
        self.rows, self.cols = t(rows), t(cols)
        mp, self.n_domains = B.gs_partition(np.asarray(X, dtype=np.float64), domain_size)
        self.map = t(mp)
        self.adj_ptr, self.adj = t(adj_ptr), t(adj)
        self.contacts = None if contacts is None or len(contacts) == 0 else t(np.asarray(contacts).reshape(-1, 2))
        self.domain_size, self.max_levels, self.precision = domain_size, max_levels, precision
        self.tol, self.mixed, self.max_iter = tol, mixed, max_iter


class _Handles:
    """Owns the matrix and preconditioner of one forward pass."""

    def __init__(self, mat, mas):
        self.mat, self.mas = mat, mas

    def free(self):
        if self.mas is not None:
            B.gs_mas_destroy(self.mas)
            self.mas = None
        if self.mat is not None:
            B.gs_mat_destroy(self.mat)
            self.mat = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def _forward(blocks, b, system):
    mat = B.gs_assemble(system.ctx, system.n, system.rows, system.cols, blocks)
    mas = B.gs_build_mas(system.ctx, mat, system.map, system.n_domains, system.adj_ptr, system.adj, system.contacts,
                         domain_size=system.domain_size, max_levels=system.max_levels, precision=system.precision)
    h = _Handles(mat, mas)
    x = torch.empty_like(b)
    nrhs = b.shape[0]
    if system.mixed:
        B.gs_pcg_solve_mixed(system.ctx, mat, mas, b, x, nrhs=nrhs, tol=system.tol, max_iter=system.max_iter)
    else:
        B.gs_pcg_solve(system.ctx, mat, mas, b, x, nrhs=nrhs, tol=system.tol, max_iter=system.max_iter)
    return x, h


class MasPcgSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, blocks, b, system):
        blocks = blocks.contiguous()
        b = b.contiguous()
        x, h = _forward(blocks, b, system)
        ctx.system = system
        ctx.handles = h
        ctx.blocks_shape = blocks.shape
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        system, h = ctx.system, ctx.handles
        nrhs = x.shape[0]
        _, nnzb = B.gs_mat_info(h.mat)
        dH = torch.empty((max(nnzb, 1), 3, 3), dtype=torch.float64, device=x.device)
        dIn = None
        if ctx.needs_input_grad[0]:
            dIn = torch.empty(ctx.blocks_shape, dtype=torch.float64, device=x.device)
        lam, _ = B.gs_adjoint(system.ctx, h.mat, h.mas, x, gx.contiguous(), nrhs=nrhs, tol=system.tol,
                              max_iter=system.max_iter, mixed=system.mixed, dLdH=dH, dLdinput=dIn)
        h.free()
        return dIn, lam, None


def solve(blocks, b, system):
    """x = A(blocks)^{-1} b, differentiable in blocks (K, 3, 3) and b (nrhs, 3n)."""
    return MasPcgSolve.apply(blocks, b, system)
