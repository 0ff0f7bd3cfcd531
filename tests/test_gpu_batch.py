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
