"""idmrg_save / idmrg_load: a context restored from a checkpoint continues
exactly as the saved one (FP64 and TF32x3 modes), and a checkpoint of another
MPO or of a context in the middle of a step is refused."""
import numpy as np
import pytest

import paper_1606_06790_gb300 as pkg
from workloads import build_mpo, chain_bonds, random_chain_bonds

from gpu_helpers import context

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
def test_restored_context_continues_identically(tmp_path, prec):
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 7), 8)
    a = context(mpo, 48, prec=prec)
    for _ in range(9):
        a.unit_cell_step()
    path = str(tmp_path / "state.ck")
    a.save(path)
    b = context(mpo, 48, prec=prec)
    b.load(path)
    assert b.iteration == a.iteration
    seen_eg = False
    for _ in range(7):  # n = 10..16: includes the e_g estimate at n + 1 = 2 l
        ga, gb = a.unit_cell_step(), b.unit_cell_step()
        assert ga["n"] == gb["n"]
        for key in ("energy", "eps", "bond", "kept", "iters"):
            assert np.array_equal(ga[key], gb[key]), (key, ga[key], gb[key])
        assert (ga["e_g"] is None and gb["e_g"] is None) or ga["e_g"] == gb["e_g"]
        seen_eg = seen_eg or ga["e_g"] is not None
    assert seen_eg
    a.close()
    b.close()


def test_checkpoint_of_another_model_is_refused(tmp_path):
    a = context(build_mpo(chain_bonds(4), 4), 16)
    a.unit_cell_step()
    path = str(tmp_path / "chain.ck")
    a.save(path)
    b = context(build_mpo(random_chain_bonds(8, 0.5, 1.5, 7), 8), 16)
    with pytest.raises(pkg.IdmrgError):
        b.load(path)
    with pytest.raises(pkg.IdmrgError):
        b.load(str(tmp_path / "missing.ck"))
    a.predict_wavefunction(-1)  # a step in progress
    with pytest.raises(pkg.IdmrgError):
        a.save(str(tmp_path / "mid.ck"))
    a.close()
    b.close()

