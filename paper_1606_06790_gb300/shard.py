"""One parallel-iDMRG problem sharded over processes (Sec. 3, Step 2').

The l/2 superblocks of an iteration are independent; what couples two
iterations is the rotation of Step 2': superblock p at n + 1 takes the right
block R^(n) of pair p + 1, and the prediction of Step 3' (Eq. wfprediction)
takes U^(n)_{p+1}, lambda^(n)_{p+1} and lambda^(n-1)_{p+1}.  With contiguous
ranges of pairs per rank, only the first pair of each range crosses a rank
boundary, so one ring shift per iteration suffices: every rank sends the data
of its first pair to the rank before it (rank 0 to the last) and receives
that of the pair after its range.  lambda^(n-1) of that pair is the one the
receiver got in the previous shift, so a message carries R^(n), U^(n) and
lambda^(n) of one pair.  The energies of superblock 1 (Step 5') stay on rank
0; the step reports are gathered there.

This module is the host logic only: the partition, the exchange (point-to-
point sends over torch.distributed, any backend) and the gather.  A `stepper`
does the arithmetic: the library's Context (Context.step_range,
Context.export_pair, Context.import_pair) on a GPU per rank.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def partition(P: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous pair ranges [p0, p1) per rank, sizes differing by at most
    one, larger ranges first.  Needs 1 <= world <= P (every rank owns a pair,
    so every ring neighbour holds the pair the shift asks for)."""
    if not 1 <= world <= P:
        raise ValueError(f"{world} ranks for {P} superblocks: need 1 <= ranks <= l/2")
    base, extra = divmod(P, world)
    out, p = [], 0
    for r in range(world):
        k = base + (1 if r < extra else 0)
        out.append((p, p + k))
        p += k
    return out


def _send_bytes(dist, payload: bytes, dst: int, dev):
    import torch
    n = torch.tensor([len(payload)], dtype=torch.int64, device=dev)
    reqs = [dist.isend(n, dst)]
    if payload:
        buf = torch.frombuffer(bytearray(payload), dtype=torch.uint8).to(dev)
        reqs.append(dist.isend(buf, dst))
    return reqs


def _recv_bytes(dist, src: int, dev) -> bytes:
    import torch
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    dist.recv(n, src)
    k = int(n.item())
    if k == 0:
        return b""
    buf = torch.empty(k, dtype=torch.uint8, device=dev)
    dist.recv(buf, src)
    return bytes(buf.cpu().numpy().tobytes())


class ShardedRun:
    """Rank `rank` of `world` steps the superblocks of its range of pairs.

    ``stepper`` provides:
      * ``P`` -- superblocks per iteration;
      * ``step_range(p0, p1)`` -- one iteration on superblocks p0..p1-1, a
        report dict with per-superblock arrays (entries outside the range
        unspecified) and ``n``, ``e_g``;
      * ``export_pair(q)`` -> bytes and ``import_pair(q, bytes)`` -- the
        boundary data of pair q after an iteration (R^(n), U^(n), lambda^(n))."""

    KEYS = ("energy", "iters", "eps", "eps_best", "fidelity", "bond", "kept")

    def __init__(self, stepper, dist=None):
        self.s = stepper
        self.dist = dist
        self.world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
        self.rank = dist.get_rank() if self.world > 1 else 0
        self.P = stepper.P
        self.ranges = partition(self.P, self.world)
        self.p0, self.p1 = self.ranges[self.rank]
        self.bytes_sent = 0
        # NCCL moves device tensors, gloo host tensors
        import torch
        nccl = self.world > 1 and dist.get_backend() == "nccl"
        self.dev = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")

    def _ring_shift(self):
        """Send the first pair of this range to the previous rank, receive the
        pair after this range (the next rank's first) from the next rank."""
        if self.world == 1:
            return
        left, right = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        payload = self.s.export_pair(self.p0)
        reqs = _send_bytes(self.dist, payload, left, self.dev)
        got = _recv_bytes(self.dist, right, self.dev)
        for q in reqs:
            q.wait()
        self.bytes_sent += len(payload)
        self.s.import_pair(self.p1 % self.P, got)

    def step(self) -> Dict[str, object]:
        """One unit-cell step of the whole problem; every rank returns the
        gathered report (per-superblock arrays of all P superblocks, e_g from
        the owner of pair 0)."""
        rep = self.s.step_range(self.p0, self.p1)
        self._ring_shift()
        if self.world == 1:
            return rep
        return self._gather(rep)

    def _gather(self, rep):
        import torch
        P = self.P
        mine = np.zeros((len(self.KEYS), P))
        for k, key in enumerate(self.KEYS):
            v = np.asarray(rep[key], dtype=np.float64)
            mine[k, self.p0:self.p1] = v[self.p0:self.p1]
        t = torch.tensor(mine, dtype=torch.float64, device=self.dev)
        parts = [torch.zeros_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t)
        eg = torch.tensor([np.nan if rep.get("e_g") is None else float(rep["e_g"])], dtype=torch.float64,
                          device=self.dev)
        self.dist.broadcast(eg, src=0)
        out = dict(rep)
        full = np.zeros((len(self.KEYS), P))
        for r, (a, b) in enumerate(self.ranges):
            full[:, a:b] = parts[r].cpu().numpy()[:, a:b]
        for k, key in enumerate(self.KEYS):
            out[key] = full[k].astype(np.int64) if key in ("iters", "kept") else full[k]
        out["e_g"] = None if np.isnan(eg.item()) else float(eg.item())
        return out
