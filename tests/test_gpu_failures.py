"""Failure statuses of the C ABI, made on the host (no device fault is ever
provoked): Lanczos stopped by lanczos_maxit (ENOCONV, with the best estimate
written and equal to the oracle's Ritz value for the same Krylov space), a
start vector with a non-finite or zero norm (ENUMERIC), MPOs that break the
lower-triangular form or charge conservation of Eq. mpo (EINVAL), and a
caller-supplied start vector that is used as given."""
import numpy as np
import pytest

from oracle import ed
from oracle.idmrg import ParallelIDMRG, heff_dense, sector_mask
from workloads import build_mpo, open_chain_bonds, random_chain_bonds

pytestmark = pytest.mark.gpu

from gpu_helpers import context, superblock_from_gpu  # noqa: E402


def _mpo():
    return build_mpo(random_chain_bonds(4, 0.5, 1.5, 77), 4)


def test_enoconv_writes_the_best_estimate():
    """maxit = 2.  At n = 1 both sides start from the same SplitMix64 vector
    in the same (site) basis, so the reported unconverged Ritz values are the
    oracle's.  Later start vectors are drawn in each side's own block basis
    (its singular-vector gauge), so there the estimate is checked against the
    exact ground energy of the open cluster (the run stays in the exact
    regime, D <= m): above it, as a Ritz value must be, and visibly so."""
    bonds = random_chain_bonds(4, 0.5, 1.5, 77)
    mpo = build_mpo(bonds, 4)
    ctx = context(mpo, 16, lanczos_maxit=2)
    ref = ParallelIDMRG.from_mpo(mpo, m=16, lanczos_maxit=2)
    for _ in range(3):
        g = ctx.unit_cell_step()
        r = ref.step()
        n = g["n"]
        assert not g["converged"]
        assert np.all(g["iters"] == 2)
        assert np.all(np.isfinite(g["energy"]))
        if n == 1:
            assert np.max(np.abs(g["energy"] - r.energies)) < 1e-12 * max(1.0, np.max(np.abs(r.energies)))
        for p in range(ctx.P):
            N = 2 * n + 2
            E0 = ed.ground_energy(N, open_chain_bonds(bonds, 4, 2 * p, 2 * p + N - 1))
            assert g["energy"][p] >= E0 - 1e-10 * N and g["energy"][p] - E0 > 1e-6, (n, p, g["energy"][p], E0)
    # stepwise: lanczos_solve returns the estimate with converged = False
    ctx.predict_wavefunction(-1)
    e, it, ok = ctx.lanczos_solve(-1)
    assert not ok and np.all(it == 2) and np.all(np.isfinite(e))
    ctx.close()


@pytest.mark.parametrize("bad", ["nan", "zero"])
def test_enumeric_from_start_vector(bad):
    import torch

    import paper_1606_06790_gb300 as pkg
    mpo = _mpo()
    ctx = context(mpo, 16, lanczos_maxit=20)
    for _ in range(2):
        ctx.unit_cell_step()
    _, N = ctx.psi_layout(0)
    x = torch.full((N,), float("nan") if bad == "nan" else 0.0, device="cuda", dtype=torch.float64)
    ctx.set_start_vector(0, x)
    with pytest.raises(pkg.IdmrgError) as ei:
        ctx.lanczos_solve(0)
    assert ei.value.status == 6  # IDMRG_ENUMERIC
    ctx.close()


def test_start_vector_is_used():
    """The exact ground state of the superblock (dense eigh of the oracle's
    Kronecker matrix on the GPU's own blocks) as start: the solve stops after
    one matvec with that energy."""
    import torch

    import paper_1606_06790_gb300 as pkg
    mpo = _mpo()
    ctx = context(mpo, 16)
    for _ in range(3):
        ctx.unit_cell_step()
    p = 1
    L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
    mask = sector_mask(L.q, mpo.phys_charge, R.q)
    H = heff_dense(L, W1, W2, R)
    idx = np.nonzero(mask.ravel())[0]
    ev, evec = np.linalg.eigh(H[np.ix_(idx, idx)])
    gs = np.zeros(mask.size)
    gs[idx] = evec[:, 0]
    desc, N = ctx.psi_layout(p)
    x = torch.tensor(pkg.layout_pack(desc, N, gs.reshape(mask.shape)), device="cuda", dtype=torch.float64)
    ctx.set_start_vector(p, x)
    e, it, ok = ctx.lanczos_solve(p)
    assert ok and it[0] == 1, (e, it)
    assert abs(e[0] - ev[0]) < 1e-11 * max(1.0, abs(ev[0]))
    ctx.close()


@pytest.mark.parametrize("flaw", ["charge", "triangular"])
def test_einval_invalid_mpo(flaw):
    import paper_1606_06790_gb300 as pkg
    mpo = _mpo()
    W = [w.copy() for w in mpo.W]
    if flaw == "charge":
        # the S+ channel (charge +2) opened with a charge-neutral S^z entry
        W[0][-1, 1] += np.diag([0.5, -0.5])
    else:
        # row 0 ("term completed") must hold nothing but W(0,0) = 1
        W[0][0, 3] = np.diag([0.5, -0.5])
    with pytest.raises(pkg.IdmrgError) as ei:
        pkg.Context(W, mpo.phys_charge, mpo.bond_charge, m=8)
    assert ei.value.status == 1  # IDMRG_EINVAL


def test_settings_and_instrumentation():
    """The restart rule, the tile setting, the Jacobi arithmetic and the SVD
    instrumentation through the C ABI: invalid arguments are EINVAL, the
    reports are consistent."""
    import paper_1606_06790_gb300 as pkg
    mpo = _mpo()
    ctx = context(mpo, 16, prec="bf16x3")
    for bad in ((0.0, 80), (1.0, 80), (1e-2, 1)):
        with pytest.raises(pkg.IdmrgError) as ei:
            ctx.set_mixed_restart(*bad)
        assert ei.value.status == 1
    with pytest.raises(pkg.IdmrgError) as ei:
        ctx.set_gemm_tile(96, 0)
    assert ei.value.status == 1
    for bad in (-1, 3):
        assert ctx.lib.idmrg_set_jacobi_arithmetic(ctx.h, bad) == 1
    ctx.set_mixed_restart(1e-2, 40)
    ctx.profile_enable(True)
    for _ in range(4):
        r = ctx.unit_cell_step()
        assert r["converged"]
    ph = ctx.svd_phase_ms()
    assert set(ph) == set(ctx.SVD_PHASES) and all(v >= 0.0 for v in ph.values())
    assert ph["jacobi64"] > 0.0 and ph["qr"] > 0.0
    st = ctx.svd_stats()
    assert st["max_sweeps32"] >= 1 and 1.0 <= st["mean_sweeps32"] <= st["max_sweeps32"]
    for stage in (1, 3):
        t = ctx.gemm_tuning(stage)
        assert t["tn"] in (64, 128, 256) and t["tunings"] >= 1
        assert t["ms"][t["tn"]] == min(t["ms"].values())
    ctx.close()
