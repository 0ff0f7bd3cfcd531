"""Parity at the cylinder models' large m, where the oracle cannot run from
n = 1 inside a test: the GPU path runs into the saturated regime, saves its
state (idmrg_save), and the oracle reads that file as data
(oracle/checkpoint.py, no code of the library involved) and takes the next
step itself.

* One unit-cell step from a saved FP64 state of the J1-J2 YC4 cylinder and of
  the kagome YC8 cylinder at m = 512 (the oracle steps a sample of the
  superblocks; each is independent within an iteration, Sec. 3): energies,
  truncation errors and bond energies within 1e-10 per site, kept dimensions,
  the lambda spectra and the fidelity error of the prediction (Eq. fid1).
* The benchmark configuration itself (kagome YC8, l = 12, m = 2048, BF16x3,
  as bench.py times it): sampled outputs the oracle computes one by one on
  the GPU's own saturated blocks -- H_eff psi of Step 3 (BF16x3 and the
  FP64-accurate digit form) and the sector SVD of Step 4 applied to the
  GPU's ground state.
"""
import numpy as np
import pytest

from oracle.checkpoint import load_state, read_checkpoint
from oracle.idmrg import Block, heff_apply, sector_mask, truncate
from workloads import make_config

from gpu_helpers import context, superblock_from_gpu

pytestmark = pytest.mark.gpu


def _dense_psi(ctx, p, vec, shape):
    import paper_1606_06790_gb300 as pkg
    desc, _ = ctx.psi_layout(p)
    return pkg.layout_unpack(desc, vec, shape)


@pytest.mark.parametrize("name,m,steps,sample", [
    ("yc4_j1j2_l8_m1024", 512, 12, (0, 3)),
    ("kagome_yc8_l12_m2048", 512, 17, (0, 5)),
])
def test_one_step_from_saved_gpu_state(tmp_path, name, m, steps, sample):
    mpo, _ = make_config(name)
    ctx = context(mpo, m, lanczos_maxit=300)
    for _ in range(steps):
        g = ctx.unit_cell_step()
    assert int(np.min(g["kept"])) >= 0.9 * m  # saturated
    path = str(tmp_path / "state.ck")
    ctx.save(path)
    ck = read_checkpoint(path)
    assert ck["n"] == ctx.iteration and ck["m"] == m
    ref = load_state(path, mpo, m)
    g = ctx.unit_cell_step()
    n = g["n"]
    sites = 2 * n + 2
    for p in sample:
        r = ref.superblock_step(p)
        t = r["trunc"]
        assert abs(g["energy"][p] - r["energy"]) / sites < 1e-10, (p, g["energy"][p], r["energy"])
        assert abs(g["eps"][p] - t.eps) < 1e-10, (p, g["eps"][p], t.eps)
        assert abs(g["bond"][p] - r["bond"]) < 1e-10, (p, g["bond"][p], r["bond"])
        assert abs(int(g["kept"][p]) - len(t.lam)) == 0 or np.all(
            t.lam_all[min(int(g["kept"][p]), len(t.lam)):max(int(g["kept"][p]), len(t.lam))]
            <= 1e-11 * t.lam_all[0]), (p, g["kept"][p], len(t.lam))
        lg = ctx.get_lambda(p)
        k = min(len(lg), len(t.lam_all), m)
        assert np.max(np.abs(lg[:k] - t.lam_all[:k])) < 1e-10
        assert abs(g["fidelity"][p] - r["fidelity"]) <= 1e-10 + 1e-6 * abs(r["fidelity"]), (
            p, g["fidelity"][p], r["fidelity"])
    ctx.close()


def test_bench_configuration_sampled_outputs():
    import torch

    import paper_1606_06790_gb300 as pkg
    mpo, o = make_config("kagome_yc8_l12_m2048")
    m = o["m"]
    ctx = context(mpo, m, prec="bf16x3", lanczos_maxit=160)
    for _ in range(18):
        g = ctx.unit_cell_step()
    assert int(np.min(g["kept"])) >= 0.9 * m  # D = m: the benchmarked regime
    p = 0
    # H_eff psi on the GPU's own blocks against the oracle (Step 3)
    L, W1, W2, R = superblock_from_gpu(ctx, mpo, p)
    mask = sector_mask(L.q, mpo.phys_charge, R.q)
    x = np.where(mask, np.random.default_rng(2048).standard_normal(mask.shape), 0.0)
    want = heff_apply(L, W1, W2, R, x)
    scale = np.max(np.abs(want))
    desc, N = ctx.psi_layout(p)
    xin = torch.tensor(pkg.layout_pack(desc, N, x), device="cuda", dtype=torch.float64)
    for form, tol in ((None, 5e-4), (1, 1e-12)):
        out = torch.zeros_like(xin)
        if form is None:
            ctx.heff_apply(p, xin, out)  # the bench's arithmetic (BF16x3)
        else:
            ctx.heff_apply_fp64(p, xin, out, form)
        torch.cuda.synchronize()
        got = pkg.layout_unpack(desc, out.cpu().numpy(), x.shape)
        assert np.max(np.abs(got - want)) <= tol * scale, (form, np.max(np.abs(got - want)) / scale)
    del L, R, want
    # the sector SVD of Step 4 on the GPU's ground state
    ctx.predict_wavefunction(-1)
    e, it, ok = ctx.lanczos_solve(-1)
    qL, _ = ctx.block_basis(p, 0)
    qR, _ = ctx.block_basis(p, 1)
    psi = _dense_psi(ctx, p, ctx.get_psi(p), (len(qL), mpo.d, mpo.d, len(qR)))
    t = truncate(psi, qL.astype(np.int64), mpo.phys_charge.astype(np.int64), qR.astype(np.int64), m)
    eps, epsb, kept = ctx.truncate(-1)
    lg = ctx.get_lambda(p)
    k = min(len(lg), len(t.lam_all), m)
    assert np.max(np.abs(lg[:k] - t.lam_all[:k])) < 1e-10
    assert abs(eps[p] - t.eps) < 1e-10
    ctx.close()
