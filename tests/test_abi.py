"""The C-ABI library builds for sm_103a, loads, and exports every function
include/idmrg.h declares (no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_1606_06790_gb300 as pkg
    if not os.path.exists(os.path.join(ROOT, "paper_1606_06790_gb300", "libidmrg.so")):
        from paper_1606_06790_gb300.build import build
        build()
    return pkg.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "idmrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(idmrg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_header(lib):
    import paper_1606_06790_gb300 as pkg
    assert sorted(pkg.EXPORTED_SYMBOLS) == declared_functions()


def test_default_opts_without_gpu(lib):
    import ctypes as C
    import paper_1606_06790_gb300 as pkg
    o = pkg._Opts()
    lib.idmrg_default_opts(C.byref(o))
    assert (o.m, o.lanczos_maxit, o.predict) == (64, 300, 1)
    assert o.lanczos_tol == 1e-12 and o.tie_rel == 1e-7


def test_no_cpu_fallback():
    import torch
    import paper_1606_06790_gb300 as pkg
    from workloads import build_mpo, chain_bonds
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    mpo = build_mpo(chain_bonds(4), 4)
    with pytest.raises(RuntimeError):
        pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=8)


def test_observable_helpers_match_the_oracle_conventions():
    # host-side marshalling of the observables (no GPU): the spin-1/2 terms of
    # s_i . s_j in the MPO's basis (2Sz = +1 is state 0) and Eqs. diff1, diff2
    import numpy as np
    import paper_1606_06790_gb300 as pkg
    from oracle import observables as ob
    terms = pkg.spin_half_dot_terms([1, -1])
    assert [t[2] for t in terms] == [1.0, 0.5, 0.5]
    assert np.array_equal(terms[0][0], ob.SZ) and np.array_equal(terms[0][1], ob.SZ)
    assert np.array_equal(terms[1][0], ob.SP) and np.array_equal(terms[1][1], ob.SM)
    assert np.array_equal(terms[2][0], ob.SM) and np.array_equal(terms[2][1], ob.SP)
    # a basis ordered the other way round gives the same operators relabelled
    flip = pkg.spin_half_dot_terms([-1, 1])
    P = np.array([[0.0, 1.0], [1.0, 0.0]])
    for (a, b, c), (a2, b2, c2) in zip(terms, flip):
        assert np.array_equal(P @ a @ P, a2) and np.array_equal(P @ b @ P, b2) and c == c2
    with pytest.raises(ValueError):
        pkg.spin_half_dot_terms([2, 0, -2])
    vals = [-0.2158, -0.2208, -0.2171, -0.2190]
    assert np.allclose(pkg.delta_pm(vals), ob.delta_pm(vals), rtol=0, atol=1e-15)
