"""FP64-accurate H_eff psi from BF16 digit slices on the tensor cores (the
Ozaki scheme) against the FP64 oracle and against the FP64-GEMM form.

Each operand row is expanded in eight 7-bit digits against a power of two of
its largest element (56 bits), digit products are summed exactly per level
and the levels in FP64, so the product carries the accuracy of an FP64 GEMM:
the bound used here is 1e-13 of max|H psi| (an FP64 GEMM over K <= 768 terms
is within ~K 2^-53 of the sum of |terms|).  The reduced-precision split forms
sit near 1e-7 (TF32 x3) and 1e-5 (BF16 x3) on the same vectors."""
import numpy as np
import pytest

from oracle.idmrg import heff_apply, sector_mask
from workloads import build_mpo, make_config, random_chain_bonds, yc4_j1j2_bonds

from gpu_helpers import context, superblock_from_gpu
import paper_1606_06790_gb300 as pkg

pytestmark = pytest.mark.gpu


def _apply(ctx, p, dense, form):
    import torch
    desc, N = ctx.psi_layout(p)
    x = torch.tensor(pkg.layout_pack(desc, N, dense), device="cuda", dtype=torch.float64)
    y = torch.zeros(N, device="cuda", dtype=torch.float64)
    if form is None:
        ctx.heff_apply(p, x, y)
    else:
        ctx.heff_apply_fp64(p, x, y, form)
    torch.cuda.synchronize()
    return pkg.layout_unpack(desc, y.cpu().numpy(), dense.shape)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("name,bonds,ell,m,steps", [
    ("randchain_l8_m96", random_chain_bonds(8, 0.5, 1.5, 77), 8, 96, 8),
    ("yc4_l8_m40", yc4_j1j2_bonds(1.0, 0.5), 8, 40, 5),
])
def test_digit_form_against_oracle(name, bonds, ell, m, steps, prec):
    mpo = build_mpo(bonds, ell)
    ctx = context(mpo, m, prec=prec)
    for _ in range(steps):
        ctx.unit_cell_step()
    rng = np.random.default_rng(11)
    for p in range(ctx.P):
        L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
        mask = sector_mask(L.q, mpo.phys_charge, R.q)
        # entries over many decades, as in a Schmidt-weighted wavefunction
        x = np.where(mask, rng.standard_normal(mask.shape) * 10.0 ** rng.uniform(-8, 0, mask.shape), 0.0)
        yr = heff_apply(L, W1, W2, R, x)
        scale = np.max(np.abs(yr))
        y1 = _apply(ctx, p, x, 1)
        y0 = _apply(ctx, p, x, 0)
        ym = _apply(ctx, p, x, None)
        e1 = np.max(np.abs(y1 - yr)) / scale
        e0 = np.max(np.abs(y0 - yr)) / scale
        em = np.max(np.abs(ym - yr)) / scale
        assert e1 < 1e-13, (p, e1, e0)
        assert e0 < 1e-13, (p, e0)
        assert em > 100 * e1  # the split form is the reduced-precision one
        assert np.all(y1[~mask] == 0.0)
    ctx.close()


def test_digit_form_at_bench_size():
    """Random-bond chain l = 16, m = 256 (saturated): the digit form is the one
    the restarts use there, and it agrees with the FP64-GEMM form."""
    mpo, opts = make_config("randchain_l16_m256")
    ctx = context(mpo, 256, prec="tf32x3")
    for _ in range(11):
        ctx.unit_cell_step()
    import torch
    rng = np.random.default_rng(5)
    for p in (0, ctx.P - 1):
        desc, N = ctx.psi_layout(p)
        x = torch.tensor(rng.standard_normal(N), device="cuda", dtype=torch.float64)
        y0 = torch.zeros_like(x)
        y1 = torch.zeros_like(x)
        ctx.heff_apply_fp64(p, x, y0, 0)
        ctx.heff_apply_fp64(p, x, y1, 1)
        torch.cuda.synchronize()
        err = (y1 - y0).abs().max().item() / y0.abs().max().item()
        assert err < 1e-13, err
    ctx.close()


def test_digit_form_in_k_chunks():
    """YC4 J1-J2 cylinder (MPO bond dimension up to 20) at m = 256: stage-3 K
    (channels x right-sector dimension) passes the 768 bound of one exact
    digit sum, so those tasks run in K chunks whose FP64 results add up."""
    mpo, _ = make_config("yc4_j1j2_l8_m1024")
    ctx = context(mpo, 256, prec="fp64tc")
    for _ in range(9):
        ctx.unit_cell_step()
    import torch
    rng = np.random.default_rng(9)
    for p in range(ctx.P):
        desc, N = ctx.psi_layout(p)
        x = torch.tensor(rng.standard_normal(N), device="cuda", dtype=torch.float64)
        y0 = torch.zeros_like(x)
        y1 = torch.zeros_like(x)
        ctx.heff_apply_fp64(p, x, y0, 0)
        l0 = ctx.launch_count()
        ctx.heff_apply(p, x, y1)
        chunked = ctx.launch_count() - l0 > 5  # psi digits, 2 W-stage passes, one launch per K chunk
        torch.cuda.synchronize()
        err = (y1 - y0).abs().max().item() / y0.abs().max().item()
        assert err < 1e-13, (p, err)
        assert chunked, p
    ctx.close()


def test_digit_form_unavailable_in_fp64_context():
    mpo = build_mpo(random_chain_bonds(4, 0.5, 1.5, 3), 4)
    ctx = context(mpo, 16, prec="fp64")
    import torch
    desc, N = ctx.psi_layout(0)
    x = torch.ones(N, device="cuda", dtype=torch.float64)
    y = torch.zeros_like(x)
    with pytest.raises(pkg.IdmrgError):
        ctx.heff_apply_fp64(0, x, y, 1)
    ctx.heff_apply_fp64(0, x, y, 0)
    ctx.close()
