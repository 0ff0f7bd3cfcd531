"""Device memory: the library allocates only through the caller's allocator
callback (torch's caching allocator in the binding) and only while its
buffers grow; in the saturated regime a unit-cell step allocates nothing."""
import pytest

from workloads import build_mpo, random_chain_bonds

from gpu_helpers import context

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_no_allocation_in_the_saturated_regime(prec):
    """Device memory comes from the caller's allocator (torch's caching
    allocator here) and only while buffers grow: once every block holds m
    states, a unit-cell step calls the allocator no more."""
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 1606), 8)
    ctx = context(mpo, 48, prec=prec)
    for _ in range(12):
        r = ctx.unit_cell_step()
    assert min(r["kept"]) >= 40
    before = ctx.alloc_calls
    for _ in range(8):
        ctx.unit_cell_step()
    assert ctx.alloc_calls == before, ctx.alloc_calls - before
    ctx.close()
