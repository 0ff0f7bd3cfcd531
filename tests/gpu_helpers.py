"""Helpers that move data between the library's block layout and the oracle's
dense arrays (placement only, no arithmetic of the method)."""
import numpy as np

import paper_1606_06790_gb300 as pkg
from oracle.idmrg import Block


def context(mpo, m, **kw):
    return pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=m, **kw)


def superblock_from_gpu(ctx, mpo, p):
    """The GPU's current superblock p as oracle objects: (L, W1, W2, R)."""
    n = ctx.iteration
    ell = ctx.ell
    qL, _ = ctx.block_basis(p, 0)
    qR, _ = ctx.block_basis(p, 1)
    L = Block(ctx.block_to_host(p, 0), qL.astype(np.int64))
    R = Block(ctx.block_to_host(p, 1), qR.astype(np.int64))
    c1, c2 = (2 * p + n) % ell, (2 * p + n + 1) % ell
    return L, mpo.W[c1], mpo.W[c2], R


def gpu_heff(ctx, p, dense):
    import torch
    desc, N = ctx.psi_layout(p)
    x = torch.tensor(pkg.layout_pack(desc, N, dense), device="cuda", dtype=torch.float64)
    y = torch.zeros(N, device="cuda", dtype=torch.float64)
    ctx.heff_apply(p, x, y)
    torch.cuda.synchronize()
    return pkg.layout_unpack(desc, y.cpu().numpy(), dense.shape)


def gpu_psi_dense(ctx, p, shape):
    desc, N = ctx.psi_layout(p)
    return pkg.layout_unpack(desc, ctx.get_psi(p), shape)
