"""idmrg_heff_apply_noalloc: H_eff psi for callers that cannot allocate device
memory while they run (memory pools fixed in advance, embedders that forbid
allocator calls).  Its scratch is a fixed array inside the library, so the
checks are that it gives what the FP64 product gives -- the library's own
idmrg_heff_apply / idmrg_heff_apply_fp64 and the oracle's heff_apply on the
same environments -- on two calls in a row (the second call reuses the array
the first one left behind), in an FP64 and in a TF32x3 context; that a
superblock too large for the array is refused with its sizes; and that a call
between truncation and advance is refused.  Kept in a file of its own, named
to be collected last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative to max |H psi|: FP64 products in a different summation order


def _noalloc(ctx, p, xin, out):
    return ctx.lib.idmrg_heff_apply_noalloc(ctx.h, p, C.c_void_p(xin.data_ptr()), C.c_void_p(out.data_ptr()))


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_noalloc_matches_heff_apply_twice(prec):
    import torch

    import paper_1606_06790_gb300 as pkg
    from oracle.idmrg import heff_apply, sector_mask
    from workloads import build_mpo, random_chain_bonds
    from gpu_helpers import superblock_from_gpu

    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 31), 8)
    ctx = pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=48, prec=prec)
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
        ctx.heff_apply_fp64(p, xin, ref, 0)
        s = _noalloc(ctx, p, xin, out)
        assert s == 0, ctx.lib.idmrg_last_error(ctx.h).decode()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= TOL * np.max(np.abs(b))
        want = heff_apply(L, W1, W2, R, x)
        got = pkg.layout_unpack(desc, a, x.shape)
        assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))
    ctx.close()


def test_noalloc_rejects_oversize_superblock_and_mid_step_call():
    import torch

    import paper_1606_06790_gb300 as pkg
    from workloads import build_mpo, make_config, random_chain_bonds

    # J1-J2 YC4 cylinder at m = 512: T1 + T3 of a saturated superblock (14 to
    # 20 MPO channels times > 1e5 wavefunction entries each, FP64) exceed 16 MiB
    mpo, _ = make_config("yc4_j1j2_l8_m1024")
    ctx = pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=512, prec="tf32x3", lanczos_maxit=120)
    for _ in range(12):
        ctx.unit_cell_step()
    assert int(ctx.psi_layout(0)[1]) > 100000
    _, N = ctx.psi_layout(0)
    xin = torch.ones(N, device="cuda", dtype=torch.float64)
    out = torch.zeros(N, device="cuda", dtype=torch.float64)
    s = _noalloc(ctx, 0, xin, out)
    msg = ctx.lib.idmrg_last_error(ctx.h).decode()
    assert s == 1, (s, msg)  # IDMRG_EINVAL
    assert "the limit is 16777216" in msg and "needs" in msg, msg
    ctx.close()

    mpo = build_mpo(random_chain_bonds(4, 0.5, 1.5, 6), 4)
    ctx = pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=16)
    for _ in range(3):
        ctx.unit_cell_step()
    _, N = ctx.psi_layout(0)
    xin = torch.ones(N, device="cuda", dtype=torch.float64)
    out = torch.zeros(N, device="cuda", dtype=torch.float64)
    ctx.predict_wavefunction(-1)
    ctx.lanczos_solve(-1)
    assert _noalloc(ctx, 0, xin, out) == 0  # solved, not yet truncated: allowed
    ctx.truncate(-1)
    assert _noalloc(ctx, 0, xin, out) == 7  # IDMRG_ESTATE until idmrg_advance
    ctx.update_environments(-1)
    ctx.advance()
    _, N = ctx.psi_layout(0)
    xin = torch.ones(N, device="cuda", dtype=torch.float64)
    out = torch.zeros(N, device="cuda", dtype=torch.float64)
    assert _noalloc(ctx, 0, xin, out) == 0
    torch.cuda.synchronize()
    ctx.close()
