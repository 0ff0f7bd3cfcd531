"""The oracle's checkpoint reader (oracle/checkpoint.py) on CPU, against a
writer of the file layout its docstring documents: an oracle state written in
that layout and read back is the same state (every block entry, every kept
vector and singular value, the e^(n)_1 and eps^(n)_1 histories), and the
restored oracle steps on exactly as the original does.  Damaged files and a
state of another m are refused.  The library's own writer is checked against
the same reader on the GPU (one step from a saved state)."""
import struct

import numpy as np
import pytest

from oracle.checkpoint import MAGIC, load_state, read_checkpoint
from oracle.idmrg import ParallelIDMRG
from workloads import build_mpo, random_chain_bonds


def _pack(fmt, *v):
    return struct.pack("<" + fmt, *v)


def _vec(a, code, width=1):
    a = np.asarray(a).ravel()
    assert len(a) % width == 0
    return _pack("q", len(a) // width) + a.astype("<" + code).tobytes()


def _sectors(q):
    """Runs of equal charge in basis order; every charge forms one run."""
    qs, dims = [], []
    for x in np.asarray(q).tolist():
        if qs and qs[-1] == x:
            dims[-1] += 1
        else:
            qs.append(int(x))
            dims.append(1)
    assert len(set(qs)) == len(qs), "basis not ordered by sector"
    return qs, dims


def _basis(q):
    qs, dims = _sectors(q)
    return _vec(qs, "i4") + _vec(dims, "i4")


def _offsets(dims):
    return np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(int) if dims else np.zeros(0, int)


def _block(B):
    """Basis, channel charges (from the non-zero entries: every channel moves
    the charge by one amount), then the sector blocks channel by channel."""
    qs, dims = _sectors(B.q)
    off = _offsets(dims)
    where = {c: i for i, c in enumerate(qs)}
    chq = []
    for a in range(B.op.shape[0]):
        x, y = np.nonzero(B.op[a])
        moves = set((B.q[x] - B.q[y]).tolist())
        assert len(moves) <= 1, "channel does not conserve charge"
        chq.append(moves.pop() if moves else 0)
    data = []
    for a, ch in enumerate(chq):
        for si in range(len(qs)):
            so = where.get(qs[si] + ch)
            if so is None:
                continue
            data.append(B.op[a, off[so]:off[so] + dims[so], off[si]:off[si] + dims[si]].ravel())
    flat = np.concatenate(data) if data else np.zeros(0)
    return _basis(B.q) + _vec(chq, "i4") + _vec(flat, "f8")


def _truncation(t, qL, qR, qp, target):
    if t is None:
        empty = _vec([], "i4") + _vec([], "i4")
        return (_pack("i", 0) + empty * 4 + _pack("q", 0) + _vec([], "f8") * 2 + _pack("dd", 0.0, 0.0)
                + _pack("qq", 0, 0) + _vec([], "f8") * 2)
    Ls, dL = _sectors(qL)
    Rs, dR = _sectors(qR)
    offL, offR = _offsets(dL), _offsets(dR)
    Us, dU = _sectors(t.q)
    offU = _offsets(dU)
    d = len(qp)
    head, Ublk, Vblk = b"", [], []
    u_off = v_off = 0
    for g, (Q, k) in enumerate(zip(Us, dU)):
        cols = slice(offU[g], offU[g] + k)
        rg, rows, first = [], [], 0
        for i in range(len(Ls)):
            for s in range(d):
                if Ls[i] + qp[s] == Q:
                    rg.append((i, s, first))
                    rows.append(t.U[offL[i]:offL[i] + dL[i], s, cols])
                    first += dL[i]
        cg, crow, cfirst = [], [], 0
        for s in range(d):
            for j in range(len(Rs)):
                if qp[s] + Rs[j] == target - Q:
                    cg.append((s, j, cfirst))
                    crow.append(t.V[s, offR[j]:offR[j] + dR[j], cols])
                    cfirst += dR[j]
        bu, bv = np.vstack(rows), np.vstack(crow)
        head += _pack("iiiii", Q, k, first, cfirst, g) + _pack("qq", u_off, v_off) + _pack("i", int(offU[g]))
        head += _vec(np.array(rg), "i4", 3) + _vec(np.array(cg), "i4", 3)
        Ublk.append(bu.ravel())
        Vblk.append(bv.ravel())
        u_off += bu.size
        v_off += bv.size
    U, V = np.concatenate(Ublk), np.concatenate(Vblk)
    return (_pack("i", 1) + _basis(qL) + _basis(qR) + _vec(Us, "i4") + _vec(dU, "i4")
            + _vec([target - Q for Q in Us], "i4") + _vec(dU, "i4") + _pack("q", len(Us)) + head
            + _vec(t.lam, "f8") + _vec(t.lam_all, "f8") + _pack("dd", t.eps, t.eps_best)
            + _pack("qq", U.size, V.size) + _vec(U, "f8") + _vec(V, "f8"))


class _Recorded(ParallelIDMRG):
    """The oracle, remembering the block bases each truncation was made in."""

    def step_range(self, p0, p1):
        bases = {p: (self.L[p].q.copy(), self.R[(p + 1) % self.P].q.copy()) for p in range(p0, p1)}
        self.__dict__.setdefault("bases", {})[self.n] = bases
        return super().step_range(p0, p1)


def _write(ref, mpo, path):
    n = ref.n
    egs = [k for k in ref.e1 if k >= 0 and (k + 1) % ref.ell == 0]
    eg_n = max(egs) if egs else -1
    eg = ref.energy_per_site(eg_n) if egs else 0.0
    dims = [w.shape[0] for w in mpo.W] + [mpo.W[0].shape[0]]
    out = MAGIC + _pack("iiiiii", ref.ell, len(ref.qp), ref.P, ref.m, 0, ref.target) + _vec(dims, "i4")
    out += _pack("ii", n, eg_n) + _pack("d", eg)
    e1 = sorted(k for k in ref.e1 if k >= 0)
    out += _vec(e1, "i4") + _vec([ref.e1[k] for k in e1], "f8")
    ep = sorted(ref.eps1)
    out += _vec(ep, "i4") + _vec([ref.eps1[k] for k in ep], "f8")
    for p in range(ref.P):
        out += _block(ref.L[p]) + _block(ref.R[p])
        for t, at in ((ref.prev[p], n - 1), (ref.prev2[p], n - 2)):
            qL, qR = ref.bases[at][p] if t is not None else (None, None)
            out += _truncation(t, qL, qR, ref.qp, ref.target)
    with open(path, "wb") as f:
        f.write(out)
    return out


def _same_state(a, b):
    assert a.n == b.n
    for p in range(a.P):
        for x, y in ((a.L[p], b.L[p]), (a.R[p], b.R[p])):
            assert np.array_equal(x.q, y.q) and np.array_equal(x.op, y.op)
        for s, t in ((a.prev[p], b.prev[p]), (a.prev2[p], b.prev2[p])):
            assert (s is None) == (t is None)
            if s is None:
                continue
            for f in ("U", "V", "lam", "q", "lam_all"):
                assert np.array_equal(getattr(s, f), getattr(t, f)), f
            assert s.eps == t.eps and s.eps_best == t.eps_best
    assert {k: v for k, v in a.e1.items()} == {k: v for k, v in b.e1.items()}
    assert a.eps1 == b.eps1


@pytest.mark.parametrize("steps", [2, 6])
def test_written_state_reads_back_and_steps_on_identically(tmp_path, steps):
    """steps = 2: the truncation at n-2 is absent (an invalid record); 6: the
    blocks are saturated at m (several charge sectors per basis)."""
    mpo = build_mpo(random_chain_bonds(4, 0.5, 1.5, 7), 4)
    ref = _Recorded.from_mpo(mpo, m=10)
    for _ in range(steps):
        ref.step()
    path = str(tmp_path / "state.ck")
    _write(ref, mpo, path)
    ck = read_checkpoint(path)
    assert (ck["ell"], ck["P"], ck["m"], ck["n"]) == (4, 2, 10, steps + 1)
    back = load_state(path, mpo, m=10)
    _same_state(ref, back)
    if steps == 6:
        assert max(len(t.lam) for t in ref.prev) == 10
        assert len(np.unique(ref.L[0].q)) >= 3
    for _ in range(3):
        r1, r2 = ref.step(), back.step()
        for f in ("energies", "iters", "eps", "eps_best", "bond", "kept"):
            assert np.array_equal(getattr(r1, f), getattr(r2, f)), f
        assert np.array_equal(np.nan_to_num(r1.fidelity, nan=-1.0), np.nan_to_num(r2.fidelity, nan=-1.0))
        assert r1.e_g == r2.e_g


def test_damaged_files_and_other_m_are_refused(tmp_path):
    mpo = build_mpo(random_chain_bonds(4, 0.5, 1.5, 7), 4)
    ref = _Recorded.from_mpo(mpo, m=8)
    for _ in range(4):
        ref.step()
    good = _write(ref, mpo, str(tmp_path / "good.ck"))
    for name, data in (("short", good[:-9]), ("long", good + b"\0"), ("magic", b"IDMRGCK0" + good[8:])):
        path = str(tmp_path / name)
        with open(path, "wb") as f:
            f.write(data)
        with pytest.raises(ValueError):
            read_checkpoint(path)
    with pytest.raises(ValueError):
        load_state(str(tmp_path / "good.ck"), mpo, m=9)
    other = build_mpo(random_chain_bonds(6, 0.5, 1.5, 7), 6)
    with pytest.raises(ValueError):
        load_state(str(tmp_path / "good.ck"), other, m=8)
