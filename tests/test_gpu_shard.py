"""One problem over two workers on one GPU (Sec. 3, Step 2'): two contexts,
each stepping one half of the pairs (idmrg_set_pair_range), exchange the
boundary pair after every iteration (idmrg_export_pair / idmrg_import_pair,
host bytes) and reproduce a single context stepping all pairs; the exchange
runs through ShardedRun's ring logic with an in-process transport.  The
workers run one after the other on the host: no kernel of one waits on the
other."""
import numpy as np
import pytest

from workloads import build_mpo, make_config, random_chain_bonds

from gpu_helpers import context

pytestmark = pytest.mark.gpu

KEYS = ("energy", "eps", "eps_best", "bond", "kept", "iters")


def _lockstep(mpo, m, prec, steps, halves):
    full = context(mpo, m, prec=prec)
    P = full.P
    ranges = [(0, halves), (halves, P)]
    parts = [context(mpo, m, prec=prec) for _ in ranges]
    out = []
    for _ in range(steps):
        g = full.unit_cell_step()
        reps = [c.step_range(a, b) for c, (a, b) in zip(parts, ranges)]
        # ring shift: worker w sends its first pair to worker w - 1
        msgs = [c.export_pair(a) for c, (a, b) in zip(parts, ranges)]
        for w, (c, (a, b)) in enumerate(zip(parts, ranges)):
            c.import_pair(b % P, msgs[(w + 1) % len(parts)])
        merged = {k: np.concatenate([np.asarray(r[k])[a:b] for r, (a, b) in zip(reps, ranges)]) for k in KEYS}
        merged["fidelity"] = np.concatenate([np.asarray(r["fidelity"])[a:b] for r, (a, b) in zip(reps, ranges)])
        merged["e_g"] = reps[0]["e_g"]
        out.append((g, merged))
    for c in [full] + parts:
        c.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_two_workers_reproduce_one_context(prec):
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 1606), 8)
    for g, h in _lockstep(mpo, 48, prec, 14, 2):
        for k in KEYS:
            assert np.array_equal(np.asarray(g[k]), h[k]), (g["n"], k, g[k], h[k])
        assert np.array_equal(np.asarray(g["fidelity"]), h["fidelity"], equal_nan=True)
        assert g["e_g"] == h["e_g"]


def test_kagome_three_and_three():
    mpo, _ = make_config("kagome_yc8_l12_m2048")
    for g, h in _lockstep(mpo, 32, "fp64", 10, 3):
        assert np.max(np.abs(np.asarray(g["energy"]) - h["energy"])) / (2 * g["n"] + 2) < 1e-12
        assert np.array_equal(np.asarray(g["kept"]), h["kept"])


def test_range_calls_are_checked():
    import paper_1606_06790_gb300 as pkg
    mpo = build_mpo(random_chain_bonds(4, 0.5, 1.5, 3), 4)
    c = context(mpo, 16)
    c.step_range(0, 1)
    with pytest.raises(pkg.IdmrgError) as e:   # the boundary pair is missing
        c.unit_cell_step()
    assert e.value.status == 7
    with pytest.raises(pkg.IdmrgError):        # pair 1 is not stepped here
        c.export_pair(1)
    with pytest.raises(pkg.IdmrgError):        # pair 0 is stepped here
        c.import_pair(0, c.export_pair(0))
    c.close()
