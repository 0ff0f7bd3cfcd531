"""The ring-shift sharding of one problem (Sec. 3, Step 2') on
CPU processes with gloo: each rank steps its contiguous range of pairs with
the FP64 oracle, exchanges the boundary pair's R^(n), U^(n), lambda^(n) with
its ring neighbours, and the gathered step reports equal a single-process
run bit for bit (every superblock computes the same operations on the same
numbers in both)."""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1606_06790_gb300.shard import ShardedRun, partition


class OracleStepper:
    """The oracle behind the stepper interface of ShardedRun (test only)."""

    def __init__(self, ref):
        self.ref = ref
        self.P = ref.P

    def step_range(self, p0, p1):
        r = self.ref.step_range(p0, p1)
        return dict(n=r.n, e_g=r.e_g, energy=r.energies, iters=r.iters, eps=r.eps, eps_best=r.eps_best,
                    fidelity=r.fidelity, bond=r.bond, kept=r.kept)

    def export_pair(self, q):
        return pickle.dumps((self.ref.R[q], self.ref.prev[q]))

    def import_pair(self, q, data):
        self.ref.R[q], self.ref.prev[q] = pickle.loads(data)


def _mpo(ell):
    from workloads import build_mpo, random_chain_bonds
    return build_mpo(random_chain_bonds(ell, 0.5, 1.5, 42), ell)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ell, m, steps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.idmrg import ParallelIDMRG
        run = ShardedRun(OracleStepper(ParallelIDMRG.from_mpo(_mpo(ell), m=m)), dist)
        reps = [run.step() for _ in range(steps)]
        if rank == 0:
            out["reps"] = pickle.dumps(reps)
        out[f"sent{rank}"] = run.bytes_sent
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ell", [(2, 8), (3, 6)])
def test_sharded_equals_single_process(world, ell):
    m, steps = 24, 12
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, ell, m, steps, out), nprocs=world, join=True,
                       start_method="spawn")
    reps = pickle.loads(out["reps"])
    from oracle.idmrg import ParallelIDMRG
    ref = ParallelIDMRG.from_mpo(_mpo(ell), m=m)
    for g in reps:
        r = ref.step()
        assert g["n"] == r.n
        for key, want in (("energy", r.energies), ("eps", r.eps), ("eps_best", r.eps_best), ("bond", r.bond),
                          ("iters", r.iters), ("kept", r.kept)):
            assert np.array_equal(np.asarray(g[key]), np.asarray(want)), (key, r.n, g[key], want)
        assert np.array_equal(np.asarray(g["fidelity"]), r.fidelity, equal_nan=True)
        assert (g["e_g"] is None) == (r.e_g is None) and (r.e_g is None or g["e_g"] == r.e_g)
    assert all(out[f"sent{r}"] > 0 for r in range(world))


def test_partition():
    assert partition(6, 1) == [(0, 6)]
    assert partition(6, 4) == [(0, 2), (2, 4), (4, 5), (5, 6)]
    assert partition(8, 3) == [(0, 3), (3, 6), (6, 8)]
    with pytest.raises(ValueError):
        partition(3, 4)
