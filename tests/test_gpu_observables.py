"""Uniform-MPS observables (Eq. mps2) through the C ABI against the oracle:
bond strengths and longer-range correlations of the same converged states,
the transfer spectrum and correlation length, the exact dimer values, and
properties that hold at the full bench size (periodicity of the unit, the
bond strengths adding up to e_g, the Cauchy-Schwarz bound)."""
import numpy as np
import pytest

import paper_1606_06790_gb300 as pkg
from oracle import observables as ob
from oracle.idmrg import ParallelIDMRG
from workloads import build_mpo, chain_bonds, dimerized_chain_bonds, j1j2_chain_bonds, random_chain_bonds

pytestmark = pytest.mark.gpu

from gpu_helpers import context  # noqa: E402

SP = np.array([[0.0, 1.0], [0.0, 0.0]])
SZ = np.diag([0.5, -0.5])


def _run_both(mpo, m, steps, prec="fp64"):
    ctx = context(mpo, m, prec=prec)
    ref = ParallelIDMRG.from_mpo(mpo, m=m)
    for _ in range(steps):
        ctx.unit_cell_step()
        ref.step()
    return ctx, ref


def _pairs(ell):
    near = [(i, i + 1) for i in range(2 * ell)]
    far = [(0, 2), (1, ell + 3), (3, 2 * ell + 1), (2, 3 * ell + 2)]
    return near + far


# states whose transfer map has a gap below its leading eigenvalue (in some
# random cells the leading eigenvalue comes as a cluster of four within 1e-7,
# a nearly free effective spin per cell: the fixed point is then ill-conditioned
# and no two implementations need agree on it)
@pytest.mark.parametrize("name,bonds,ell,m,steps", [
    ("chain_l4_m16", chain_bonds(4), 4, 16, 30),
    ("randchain_l8_m20_seed3", random_chain_bonds(8, 0.5, 1.5, 3), 8, 20, 32),
    ("randchain_l16_m16", random_chain_bonds(16, 0.5, 1.5, 1606), 16, 16, 32),
    ("j1j2_l4_m16", j1j2_chain_bonds(4, 1.0, 0.3), 4, 16, 16),
])
def test_against_oracle_fp64(name, bonds, ell, m, steps):
    ctx, ref = _run_both(build_mpo(bonds, ell), m, steps)
    A, s0 = ob.uniform_unit(ref)
    pairs = _pairs(ell)
    got = ctx.spin_dot(pairs)
    want = np.array([ob.spin_dot(A, s0, i, j) for i, j in pairs])
    assert np.max(np.abs(got - want)) < 1e-9, (got, want)
    # a charge-changing mixture: <(S+ + S-)_i Sz_j> + 0.3 <Sz_i Sz_j>
    X = SP + SP.T
    terms = [(X, SZ, 1.0), (SZ, SZ, 0.3)]
    got2 = ctx.correlation(terms, pairs[:6])
    want2 = np.array([ob.correlation(A, s0, X, SZ, i, j) + 0.3 * ob.correlation(A, s0, SZ, SZ, i, j)
                      for i, j in pairs[:6]])
    assert np.max(np.abs(got2 - want2)) < 1e-9, (got2, want2)
    t1, t2, xi, it, conv = ctx.transfer_spectrum(tol=1e-11, maxit=5000)
    ev = np.abs(ob.spectrum(A))
    assert conv
    assert t1 == pytest.approx(ev[0], rel=1e-10)
    assert t2 == pytest.approx(ev[1], rel=1e-6)
    assert xi == pytest.approx(ob.correlation_length(A), rel=1e-6)
    ctx.close()


@pytest.mark.parametrize("bonds", [dimerized_chain_bonds(4), j1j2_chain_bonds(4, 1.0, 0.5)])
def test_exact_dimer_states(bonds):
    ctx = context(build_mpo(bonds, 4), 4)
    for _ in range(12):
        ctx.unit_cell_step()
    vals = ctx.spin_dot([(i, i + 1) for i in range(8)] + [(0, 3), (1, 6)])
    expect = [-0.75 if i % 2 == 0 else 0.0 for i in range(8)] + [0.0, 0.0]
    assert np.max(np.abs(vals - expect)) < 1e-12, vals
    t1, t2, xi, _, _ = ctx.transfer_spectrum()
    assert t1 == pytest.approx(1.0, abs=1e-12)
    assert t2 < 1e-10 and xi < 0.1
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp64tc"])
def test_other_precisions(prec):
    ctx, ref = _run_both(build_mpo(chain_bonds(4), 4), 16, 30, prec=prec)
    A, s0 = ob.uniform_unit(ref)
    pairs = _pairs(4)
    got = ctx.spin_dot(pairs)
    want = np.array([ob.spin_dot(A, s0, i, j) for i, j in pairs])
    tol = 1e-9 if prec == "fp64tc" else 1e-6
    assert np.max(np.abs(got - want)) < tol, (got, want)
    ctx.close()


def test_state_and_argument_errors():
    ctx = context(build_mpo(chain_bonds(4), 4), 8)
    ctx.unit_cell_step()     # n = 2 afterwards: the unit needs two completed iterations
    with pytest.raises(pkg.IdmrgError) as e:
        ctx.spin_dot([(1, 1)])
    assert e.value.status == 1
    with pytest.raises(pkg.IdmrgError) as e:
        ctx.spin_dot([(3, 2)])
    assert e.value.status == 1
    with pytest.raises(pkg.IdmrgError) as e:
        ctx.spin_dot([(0, 1)])
    assert e.value.status == 7
    fresh = context(build_mpo(chain_bonds(4), 4), 8)
    with pytest.raises(pkg.IdmrgError) as e:
        fresh.transfer_spectrum()
    assert e.value.status == 7
    # values are cached per iteration and recomputed after the next step
    for _ in range(3):
        ctx.unit_cell_step()
    a = ctx.spin_dot([(0, 1)])
    ctx.unit_cell_step()
    b = ctx.spin_dot([(0, 1)])
    assert a.shape == b.shape == (1,)
    ctx.close()
    fresh.close()


def test_full_size_properties():
    """Random-bond chain l = 16, m = 256 (the bench workload), TF32x3 after
    32 iterations: the unit repeats, the bond energies J <s.s> of one unit add
    up to l e_g, every |<s.s>| <= 3/4."""
    from workloads import make_config
    mpo, opts = make_config("randchain_l16_m256")
    ctx = context(mpo, opts["m"], prec="tf32x3")
    e_g = None
    for _ in range(32):
        r = ctx.unit_cell_step()
        e_g = r["e_g"] if r["e_g"] is not None else e_g
    ell = 16
    near = [(i, i + 1) for i in range(ell)]
    shifted = [(i + ell, i + ell + 1) for i in range(ell)]
    v = ctx.spin_dot(near + shifted + [(0, 40), (5, 100)])
    assert np.max(np.abs(v[:ell] - v[ell:2 * ell])) < 1e-10
    assert np.all(np.abs(v) <= 0.75 + 1e-12)
    J = {b.i % ell: b.jz for b in mpo.bonds if b.j == b.i + 1 and b.jxy == b.jz}
    assert len(J) == ell
    e_unit = sum(J[i] * v[i] for i in range(ell)) / ell
    assert e_unit == pytest.approx(e_g, abs=1e-5)
    t1, t2, xi, _, conv = ctx.transfer_spectrum()
    assert conv and abs(t1 - 1.0) < 1e-2 and 0.0 < xi < 1e3
    ctx.close()


def test_checkpoint_restores_observables(tmp_path):
    """A context restored from a checkpoint rebuilds the same unit: the
    observables come out bit for bit (seeded start vectors, fixed-order
    reductions, fixed tile shape)."""
    mpo = build_mpo(chain_bonds(4), 4)
    ctx = context(mpo, 16)
    for _ in range(20):
        ctx.unit_cell_step()
    pairs = _pairs(4)
    a = ctx.spin_dot(pairs)
    sa = ctx.transfer_spectrum()
    path = str(tmp_path / "obs.ck")
    ctx.save(path)
    other = context(mpo, 16)
    other.load(path)
    b = other.spin_dot(pairs)
    sb = other.transfer_spectrum()
    assert np.array_equal(a, b)
    assert sa == sb
    ctx.close()
    other.close()
