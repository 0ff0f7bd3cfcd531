"""idmrg_heff_apply_noalloc: H_eff psi for callers that cannot allocate device
memory while they run (memory pools fixed in advance, embedders that forbid
allocator calls).  Its scratch is a fixed array inside the library, so the
check is that it gives what idmrg_heff_apply gives, on two calls in a row
(the second call reuses the array the first one left behind).  Kept in a file
of its own, named to be collected last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_heff_apply_twice():
    import torch

    import paper_1606_06790_gb300 as pkg
    from oracle.idmrg import sector_mask
    from workloads import build_mpo, random_chain_bonds
    from gpu_helpers import superblock_from_gpu

    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 31), 8)
    ctx = pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=48)
    for _ in range(6):
        ctx.unit_cell_step()
    rng = np.random.default_rng(11)
    for call in range(2):
        p = call % ctx.P
        L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
        mask = sector_mask(L.q, mpo.phys_charge, R.q)
        x = np.where(mask, rng.standard_normal(mask.shape), 0.0)
        desc, N = ctx.psi_layout(p)
        xin = torch.tensor(pkg.layout_pack(desc, N, x), device="cuda", dtype=torch.float64)
        ref = torch.zeros(N, device="cuda", dtype=torch.float64)
        out = torch.full((N,), float("nan"), device="cuda", dtype=torch.float64)
        ctx.heff_apply(p, xin, ref)
        s = ctx.lib.idmrg_heff_apply_noalloc(ctx.h, p, C.c_void_p(xin.data_ptr()), C.c_void_p(out.data_ptr()))
        assert s == 0, ctx.lib.idmrg_last_error(ctx.h).decode()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    ctx.close()
