"""Mixed-precision path (TF32 x3 or BF16 x3 tensor cores for H_eff psi, FP64
Lanczos with FP64-checked restarts, FP64 SVD) against the FP64 oracle.

Matvec: TF32 split operands (hi + lo, ~21 bits) with FP32 accumulation give a
relative error of a few 1e-7 per product; over K <= a few hundred terms the
bound used here is 3e-5 of max|H psi|.  BF16 splits (hi + lo, ~16 bits) give
a few 1e-6 per product, 5e-4 of max|H psi|.  Energies: the restart scheme ends on
an FP64 residual check, so energies per site, truncation errors and bond
energies must agree with the oracle within 1e-8 (the mixed-mode target).
The centre-bond energy is first order in the eigenvector error (about
2 |h| tol |E| / gap), so these runs use lanczos_tol = 1e-13 on both sides: with
1e-12 a small-gap J1-J2 chain leaves it undetermined at the 1e-8 level in the
oracle itself."""
import numpy as np
import pytest

from oracle.idmrg import ParallelIDMRG, heff_apply, sector_mask
from workloads import build_mpo, chain_bonds, j1j2_chain_bonds, random_chain_bonds

from gpu_helpers import context, gpu_heff, superblock_from_gpu

pytestmark = pytest.mark.gpu


# bound on max|H psi - H psi (oracle)| / max|H psi|: ~3 * 2^-22 (TF32 splits)
# or ~3 * 2^-18 (BF16 splits) per product, times the cancellation over K terms
HEFF_BOUND = {"tf32x3": 3e-5, "bf16x3": 5e-4}


@pytest.mark.parametrize("tiles", [(0, 0), (64, 256), (128, 128), (256, 64)])
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_mixed_heff_against_oracle(prec, tiles):
    """Every N tile of the split-operand GEMMs (the tuner's pick, and each
    width forced on stages 1 and 3)."""
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 77), 8)
    ctx = context(mpo, 96, prec=prec)
    ctx.set_gemm_tile(*tiles)
    for _ in range(8):
        ctx.unit_cell_step()
    rng = np.random.default_rng(4)
    for p in range(ctx.P):
        L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
        mask = sector_mask(L.q, mpo.phys_charge, R.q)
        x = np.where(mask, rng.standard_normal(mask.shape), 0.0)
        y = gpu_heff(ctx, p, x)
        yr = heff_apply(L, W1, W2, R, x)
        err = np.max(np.abs(y - yr)) / np.max(np.abs(yr))
        assert err < HEFF_BOUND[prec], err
        assert err > 0.0  # really the reduced-precision path
        assert np.all(y[~mask] == 0.0)
    for stage, tn in zip((1, 3), tiles):
        t = ctx.gemm_tuning(stage)
        assert t["tn"] == tn if tn else t["tn"] in (64, 128, 256)
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("name,bonds,ell,m,steps", [
    ("chain_l4_m32", chain_bonds(4), 4, 32, 30),
    ("randchain_l8_m64", random_chain_bonds(8, 0.5, 1.5, 1606), 8, 64, 14),
    ("j1j2_l4_m24", j1j2_chain_bonds(4, 1.0, 0.3), 4, 24, 16),
])
def test_mixed_iteration_matches_fp64_oracle(name, bonds, ell, m, steps, prec):
    mpo = build_mpo(bonds, ell)
    ctx = context(mpo, m, prec=prec, lanczos_tol=1e-13)
    ref = ParallelIDMRG.from_mpo(mpo, m=m, lanczos_tol=1e-13)
    for _ in range(steps):
        g = ctx.unit_cell_step()
        r = ref.step()
        N = 2 * r.n + 2
        assert g["converged"]
        assert np.max(np.abs(g["energy"] - r.energies)) / N < 1e-8, (r.n, g["energy"] - r.energies)
        assert np.max(np.abs(g["eps"] - r.eps)) < 1e-8
        assert np.max(np.abs(g["bond"] - r.bond)) < 1e-8
        if r.e_g is not None:
            assert abs(g["e_g"] - r.e_g) < 1e-8
    ctx.close()
