"""Independent contexts stepped together (idmrg_batch_step: disorder
realisations of uneven unit cells and m, concurrent on host threads and
streams) give exactly what each context gives alone, and agree with the
oracle."""
import numpy as np
import pytest

import paper_1606_06790_gb300 as pkg
from oracle.idmrg import ParallelIDMRG
from workloads import build_mpo, random_chain_bonds

pytestmark = pytest.mark.gpu


def _realisations():
    # the config-5 recipe at test sizes: l in (4, 8), m in (16, 24), J ~ U[0.2, 1.8]
    out = []
    for r in range(6):
        ell = (4, 8)[r % 2]
        m = (16, 24)[(r // 2) % 2]
        out.append((build_mpo(random_chain_bonds(ell, 0.2, 1.8, 1000 + r), ell), m))
    return out


def _ctx(mpo, m, prec):
    import torch
    return pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=m, prec=prec, stream=torch.cuda.Stream())


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_batch_equals_single(prec):
    work = _realisations()
    batch = [_ctx(mpo, m, prec) for mpo, m in work]
    single = [_ctx(mpo, m, prec) for mpo, m in work]
    for _ in range(10):
        reps = pkg.batch_step(batch, threads=4)
        for ctx, rb in zip(single, reps):
            rs = ctx.unit_cell_step()
            assert rb["n"] == rs["n"]
            assert np.array_equal(rb["energy"], rs["energy"])
            assert np.array_equal(rb["eps"], rs["eps"])
            assert np.array_equal(rb["kept"], rs["kept"])
    for c in batch + single:
        c.close()


def test_batch_against_oracle():
    work = _realisations()[:3]
    batch = [_ctx(mpo, m, "fp64") for mpo, m in work]
    refs = [ParallelIDMRG.from_mpo(mpo, m=m) for mpo, m in work]
    for _ in range(8):
        reps = pkg.batch_step(batch, threads=3)
        for rb, ref in zip(reps, refs):
            r = ref.step()
            assert np.max(np.abs(rb["energy"] - r.energies)) / (2 * r.n + 2) < 1e-10
            assert np.array_equal(rb["kept"], r.kept)
    for c in batch:
        c.close()


def _problems(work):
    return [(mpo.W, mpo.phys_charge, mpo.bond_charge) for mpo, _ in work]


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_ring_context_equals_single(prec):
    """One context over all realisations (idmrg_create_batch: every launch and
    every Lanczos-iteration graph serves the superblocks of all of them, each
    realisation a ring of its own l and m) against each realisation in a
    context of its own.  The FP64 GEMM tiles are tuned on the batched task
    lists, so products may be summed in another order: energies agree to
    rounding, kept dimensions exactly."""
    work = _realisations()
    batch = pkg.Context.batch(_problems(work), [m for _, m in work], prec=prec)
    single = [_ctx(mpo, m, prec) for mpo, m in work]
    assert batch.rings == [(sum(len(w.W) // 2 for w, _ in work[:r]), len(work[r][0].W) // 2)
                           for r in range(len(work))]
    for _ in range(12):
        rb = batch.unit_cell_step()
        for (p0, k), ctx in zip(batch.rings, single):
            rs = ctx.unit_cell_step()
            assert rb["n"] == rs["n"]
            sites = 2 * rs["n"] + 2
            assert np.max(np.abs(rb["energy"][p0:p0 + k] - rs["energy"])) / sites < 1e-12
            assert np.max(np.abs(rb["eps"][p0:p0 + k] - rs["eps"])) < 1e-12
            assert np.array_equal(rb["kept"][p0:p0 + k], rs["kept"])
    for r, ctx in enumerate(single):
        got, want = batch.ring_energy(r), ctx.energy_per_site()
        assert got is not None and got[1] == want[1] and abs(got[0] - want[0]) < 1e-12
    for c in [batch] + single:
        c.close()


def test_ring_context_against_oracle():
    work = _realisations()[:3]
    batch = pkg.Context.batch(_problems(work), [m for _, m in work], prec="fp64")
    refs = [ParallelIDMRG.from_mpo(mpo, m=m) for mpo, m in work]
    for _ in range(8):
        rb = batch.unit_cell_step()
        for (p0, k), ref in zip(batch.rings, refs):
            r = ref.step()
            assert np.max(np.abs(rb["energy"][p0:p0 + k] - r.energies)) / (2 * r.n + 2) < 1e-10
            assert np.array_equal(rb["kept"][p0:p0 + k], r.kept)
    batch.close()


def test_ring_context_argument_errors(tmp_path):
    work = _realisations()[:2]
    batch = pkg.Context.batch(_problems(work), 16)
    batch.unit_cell_step()
    for call in (lambda: batch.save(str(tmp_path / "x.ck")), lambda: batch.spin_dot([(0, 1)]),
                 lambda: batch.step_range(0, 1)):
        with pytest.raises(pkg.IdmrgError) as e:
            call()
        assert e.value.status == 1  # EINVAL: a context of one problem only
    batch.close()
    # another local basis
    mpo = work[0][0]
    with pytest.raises(pkg.IdmrgError) as e:
        pkg.Context.batch([(mpo.W, mpo.phys_charge, mpo.bond_charge),
                           (mpo.W, -np.asarray(mpo.phys_charge), mpo.bond_charge)], 16)
    assert e.value.status == 1
