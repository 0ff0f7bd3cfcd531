"""CUDA path against the FP64 oracle, element by element on identical seeded
inputs (FP64 and FP64_TC modes: energies, bond energies and truncation errors
within 1e-10 per site; the matvec within 1e-12 relative)."""
import numpy as np
import pytest

from oracle import ed
from oracle.idmrg import ParallelIDMRG, heff_apply, heff_dense, sector_mask
from workloads import (build_mpo, chain_bonds, dimerized_chain_bonds, j1j2_chain_bonds,
                       open_chain_bonds, random_chain_bonds, xx_chain_bonds)

pytestmark = pytest.mark.gpu

from gpu_helpers import context, gpu_heff, gpu_psi_dense, superblock_from_gpu  # noqa: E402

TOL_SITE = 1e-10


def _run_both(mpo, m, steps, **kw):
    ctx = context(mpo, m, **kw)
    ref = ParallelIDMRG.from_mpo(mpo, m=m, **{k: v for k, v in kw.items() if k in ("predict", "seed")})
    out = []
    for _ in range(steps):
        g = ctx.unit_cell_step()
        r = ref.step()
        out.append((g, r))
    return ctx, ref, out


def _compare(g, r, tol=TOL_SITE):
    N = 2 * r.n + 2
    assert g["n"] == r.n
    assert np.max(np.abs(g["energy"] - r.energies)) / N < tol, (r.n, g["energy"], r.energies)
    assert np.max(np.abs(g["eps"] - r.eps)) < tol, (r.n, g["eps"], r.eps)
    assert np.max(np.abs(g["bond"] - r.bond)) < tol, (r.n, g["bond"], r.bond)
    assert np.array_equal(g["kept"], r.kept), (r.n, g["kept"], r.kept)
    if r.e_g is not None:
        assert abs(g["e_g"] - r.e_g) < tol
    else:
        assert g["e_g"] is None


@pytest.mark.parametrize("prec", ["fp64", "fp64tc"])
@pytest.mark.parametrize("name,bonds,ell,m,steps", [
    ("chain_l4_m32", chain_bonds(4), 4, 32, 40),
    ("randchain_l8_m48", random_chain_bonds(8, 0.5, 1.5, 1606), 8, 48, 16),
    ("j1j2_l4_m24", j1j2_chain_bonds(4, 1.0, 0.3), 4, 24, 20),
    ("xx_l4_m20", xx_chain_bonds(4, 0.5, 1.5, 3), 4, 20, 16),
])
def test_full_iteration_parity(name, bonds, ell, m, steps, prec):
    """FP64 GEMMs (fp64) and FP64-accurate digit slices on the tensor cores
    (fp64tc) against the oracle, step by step."""
    ctx, ref, out = _run_both(build_mpo(bonds, ell), m, steps, prec=prec)
    for g, r in out:
        _compare(g, r)
    ctx.close()


@pytest.mark.parametrize("arith", ["fp64", "pairs"])
def test_large_sector_svd_path(arith):
    """The kernels for sector matrices beyond the shared-memory ones (pivoted
    QR on a cluster with the columns in global memory, the FP32 block
    tournament streamed through shared memory, the final cyclic Jacobi in
    global memory started from the Newton-Schulz-orthogonalised FP32
    rotations, in FP64 or in FP32-pair arithmetic), forced on a small
    problem, against the oracle: the step reports at 1e-10 per site and the
    lambda spectra at 1e-10 every step."""
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 1606), 8)
    ctx = context(mpo, 48)
    ctx.set_svd_path(True)
    ctx.set_jacobi_arithmetic(arith)
    ref = ParallelIDMRG.from_mpo(mpo, m=48)
    for _ in range(14):
        _compare(ctx.unit_cell_step(), ref.step())
        for p in range(ctx.P):
            lg, lr = ctx.get_lambda(p), ref.prev[p].lam_all
            assert len(lg) == len(lr) and np.max(np.abs(lg - lr)) < 1e-10
    assert ctx.svd_stats()["max_sweeps"] <= 6  # FP32-preconditioned final sweeps
    ctx.close()


def test_lambda_spectra_parity():
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 5), 8)
    ctx, ref, out = _run_both(mpo, 40, 8)
    for p in range(ctx.P):
        lg = ctx.get_lambda(p)
        lr = ref.prev[p].lam_all
        k = min(len(lg), len(lr))
        assert abs(len(lg) - len(lr)) == 0
        assert np.max(np.abs(lg[:k] - lr[:k])) < 1e-10
        assert abs(np.sum(lg ** 2) - 1.0) < 1e-12
    ctx.close()


def test_heff_matches_oracle_on_gpu_environments():
    """One H_eff psi per superblock on the GPU's own L, R (several tiles, ragged)."""
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 77), 8)
    ctx = context(mpo, 96)
    for _ in range(8):
        ctx.unit_cell_step()
    rng = np.random.default_rng(3)
    for p in range(ctx.P):
        L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
        mask = sector_mask(L.q, mpo.phys_charge, R.q)
        x = np.where(mask, rng.standard_normal(mask.shape), 0.0)
        y = gpu_heff(ctx, p, x)
        yr = heff_apply(L, W1, W2, R, x)
        assert np.max(np.abs(y - yr)) <= 1e-12 * np.max(np.abs(yr))
        assert np.all(y[~mask] == 0.0)
    ctx.close()


def test_heff_all_superblocks_concatenated():
    import torch
    import paper_1606_06790_gb300 as pkg
    mpo = build_mpo(chain_bonds(4), 4)
    ctx = context(mpo, 16)
    for _ in range(5):
        ctx.unit_cell_step()
    rng = np.random.default_rng(0)
    xs, ys, descs = [], [], []
    for p in range(ctx.P):
        L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
        mask = sector_mask(L.q, mpo.phys_charge, R.q)
        x = np.where(mask, rng.standard_normal(mask.shape), 0.0)
        xs.append(x)
        ys.append(heff_apply(L, W1, W2, R, x))
        descs.append(ctx.psi_layout(p))
    vin = np.concatenate([pkg.layout_pack(d, N, x) for (d, N), x in zip(descs, xs)])
    tin = torch.tensor(vin, device="cuda")
    tout = torch.zeros_like(tin)
    ctx.heff_apply(-1, tin, tout)
    torch.cuda.synchronize()
    vout = tout.cpu().numpy()
    off = 0
    for (d, N), x, yr in zip(descs, xs, ys):
        y = pkg.layout_unpack(d, vout[off:off + N], x.shape)
        off += N
        assert np.max(np.abs(y - yr)) <= 1e-12 * np.max(np.abs(yr))
    ctx.close()


def test_stepwise_api_and_lanczos_against_dense_eigh():
    mpo = build_mpo(random_chain_bonds(4, 0.5, 1.5, 9), 4)
    ctx = context(mpo, 8)
    for _ in range(3):
        ctx.unit_cell_step()
    ctx.predict_wavefunction(-1)
    e, it, conv = ctx.lanczos_solve(-1)
    assert conv
    for p in range(ctx.P):
        L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
        mask = sector_mask(L.q, mpo.phys_charge, R.q)
        H = heff_dense(L, W1, W2, R)[np.ix_(mask.ravel(), mask.ravel())]
        assert abs(e[p] - np.linalg.eigvalsh(H)[0]) < 1e-11 * max(1, abs(e[p]))
        psi = gpu_psi_dense(ctx, p, mask.shape)
        assert abs(np.linalg.norm(psi) - 1) < 1e-13
        r = heff_apply(L, W1, W2, R, psi) - e[p] * psi
        assert np.linalg.norm(r) < 1e-9
    eps, epsb, kept = ctx.truncate(-1)
    assert np.allclose(eps, (2 - epsb) * epsb, atol=1e-14)
    ctx.update_environments(-1)
    ctx.advance()
    for p in range(ctx.P):  # identity channels of the new blocks stay exact
        Lh = ctx.block_to_host(p, 0)
        Rh = ctx.block_to_host(p, 1)
        assert np.allclose(Lh[-1], np.eye(Lh.shape[1]), atol=1e-12)
        assert np.allclose(Rh[0], np.eye(Rh.shape[1]), atol=1e-12)
    ctx.close()


def test_call_order_is_enforced():
    import paper_1606_06790_gb300 as pkg
    mpo = build_mpo(chain_bonds(4), 4)
    ctx = context(mpo, 8)
    with pytest.raises(pkg.IdmrgError) as e:
        ctx.truncate(-1)
    assert e.value.status == 7
    with pytest.raises(pkg.IdmrgError):
        ctx.advance()
    ctx.unit_cell_step()  # still usable
    ctx.close()


def test_exact_regime_against_ed():
    bonds, ell = random_chain_bonds(4, 0.5, 1.5, 21), 4
    ctx = context(build_mpo(bonds, ell), 64)
    for n in range(1, 7):
        g = ctx.unit_cell_step()
        for p in range(ctx.P):
            N = 2 * n + 2
            E = ed.ground_energy(N, open_chain_bonds(bonds, ell, 2 * p, 2 * p + N - 1))
            assert abs(g["energy"][p] - E) < 1e-11 * N
    ctx.close()


def test_degenerate_and_rank_deficient_cases():
    """Majumdar-Ghosh (rank-1 cuts, exact -3/8) and the dimer chain (exact zeros dropped)."""
    for bonds in (j1j2_chain_bonds(4, 1.0, 0.5), dimerized_chain_bonds(4)):
        mpo = build_mpo(bonds, 4)
        ctx, ref, out = _run_both(mpo, 4, 12)
        for g, r in out:
            _compare(g, r)
            if g["e_g"] is not None:
                assert abs(g["e_g"] + 0.375) < 1e-12
        ctx.close()


def test_two_site_cell_and_no_prediction():
    mpo = build_mpo(chain_bonds(2), 2)
    ctx, ref, out = _run_both(mpo, 16, 12, predict=False)
    for g, r in out:
        _compare(g, r)
        assert np.all(np.isnan(g["fidelity"]))
    ctx.close()


def test_seed_changes_start_not_result():
    mpo = build_mpo(chain_bonds(4), 4)
    a = context(mpo, 16, seed=1)
    b = context(mpo, 16, seed=2)
    for _ in range(4):
        ga, gb = a.unit_cell_step(), b.unit_cell_step()
        assert np.max(np.abs(ga["energy"] - gb["energy"])) < 1e-10
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp64tc"])
def test_prediction_parity(prec):
    """Step 3' (Eq. wfprediction, readings R3 and R4) against the oracle: the
    fidelity error of Eq. fid1 per superblock and step, the Lanczos matvec
    counts it buys, and ||psi~|| before each solve (idmrg_predict_wavefunction
    with norm_out) -- quantities the converged energies do not depend on.  A
    wrong lambda^(n-2) or a U taken from the wrong superblock moves the
    fidelity error by orders of magnitude (the CPU test
    test_wrong_prediction_reading_is_visible plants that mistake in the
    oracle)."""
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 1606), 8)
    ctx, ref, out = _run_both(mpo, 48, 14, prec=prec)
    for g, r in out:
        _compare(g, r)
        if r.n < 3:
            assert np.all(np.isnan(g["fidelity"]))
            continue
        fg, fr = g["fidelity"], r.fidelity
        # lambda'' is inverted down to the zero threshold, which magnifies the
        # rounding of the smallest singular values (see test_gpu_fullsize)
        assert np.all(np.abs(fg - fr) <= 1e-9 + 1e-3 * np.abs(fr)), (r.n, fg, fr)
        # the same start vector and operator: matvec counts within the
        # rounding of the two re-orthogonalisation schemes
        assert np.all(np.abs(g["iters"] - r.iters) <= 2), (r.n, g["iters"], r.iters)
    ctx.close()
    # the prediction pays (Sec. 4: ~3x fewer iterations): the oracle without it
    nopred = ParallelIDMRG.from_mpo(mpo, m=48, predict=False)
    its = [nopred.step().iters for _ in range(14)]
    late_gpu = np.mean([np.mean(g["iters"]) for g, r in out if r.n >= 8])
    late_np = np.mean([np.mean(x) for x in its[7:]])
    assert late_gpu < 0.7 * late_np, (late_gpu, late_np)
    # ||psi~|| through the step-by-step calls
    ctx = context(mpo, 48, prec=prec)
    ref = ParallelIDMRG.from_mpo(mpo, m=48)
    for _ in range(12):
        want = np.array([np.linalg.norm(ref.start_vector(p)) for p in range(ref.P)])
        got = ctx.predict_wavefunction(-1)
        assert np.all(np.abs(got - want) <= 1e-9 * want), (ref.n, got, want)
        ctx.lanczos_solve(-1)
        ctx.truncate(-1)
        ctx.update_environments(-1)
        ctx.advance()
        ref.step()
    ctx.close()
