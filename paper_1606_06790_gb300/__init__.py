"""Python binding of libidmrg (include/idmrg.h): argument marshalling only.

Every step of the iDMRG hot path runs in the CUDA kernels of the shared
library; this module converts Python/torch objects to the C ABI's pointers and
sizes.  PyTorch provides device memory (through the caching allocator, handed
to the library as an ``idmrg_allocator``) and the CUDA stream.  There is no CPU
fallback: if libidmrg.so is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

__all__ = ["load_library", "Context", "STATUS", "PREC", "EXPORTED_SYMBOLS", "IdmrgError", "batch_step"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libidmrg.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ETIMEOUT", 6: "ENUMERIC",
          7: "ESTATE"}
PREC = {"fp64": 0, "tf32x3": 1, "bf16x3": 2, "fp64tc": 3}

EXPORTED_SYMBOLS = [
    "idmrg_default_opts", "idmrg_create", "idmrg_destroy", "idmrg_last_error", "idmrg_set_stream",
    "idmrg_iteration", "idmrg_psi_layout", "idmrg_block_basis", "idmrg_block_to_host",
    "idmrg_heff_apply", "idmrg_heff_apply_fp64", "idmrg_predict_wavefunction", "idmrg_set_start_vector",
    "idmrg_lanczos_solve", "idmrg_get_psi",
    "idmrg_truncate", "idmrg_get_lambda", "idmrg_update_environments", "idmrg_advance",
    "idmrg_unit_cell_step", "idmrg_batch_step", "idmrg_run", "idmrg_truncation_error", "idmrg_energy_per_site", "idmrg_heff_cost", "idmrg_launch_count",
    "idmrg_profile_enable", "idmrg_profile_read", "idmrg_transfer_bytes", "idmrg_heff_apply_noalloc",
    "idmrg_svd_stats", "idmrg_set_svd_path", "idmrg_set_jacobi_arithmetic", "idmrg_gemm_tuning", "idmrg_set_gemm_tile", "idmrg_create_batch", "idmrg_ring_energy", "idmrg_set_mixed_restart", "idmrg_svd_phase_ms", "idmrg_svd_sweeps32", "idmrg_save", "idmrg_load",
    "idmrg_correlation", "idmrg_transfer_spectrum", "idmrg_delta_pm", "idmrg_extrapolate",
    "idmrg_fit_correlation_length", "idmrg_set_pair_range", "idmrg_export_pair", "idmrg_import_pair",
]

KERNEL_CLASSES = {"heff_gemm": 0, "heff_wstage": 1, "lanczos_vec": 2, "lanczos_tri": 3, "svd": 4, "env": 5,
                  "predict": 6, "heff_f64": 7}


class IdmrgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _MPO(C.Structure):
    _fields_ = [("ell", C.c_int), ("d", C.c_int), ("bond_dim", C.POINTER(C.c_int)),
                ("W", C.POINTER(C.c_double)), ("phys_charge", C.POINTER(C.c_int)),
                ("bond_charge", C.POINTER(C.c_int))]


class _Opts(C.Structure):
    _fields_ = [("m", C.c_int), ("target_charge", C.c_int), ("lanczos_tol", C.c_double),
                ("lanczos_maxit", C.c_int), ("prec", C.c_int), ("predict", C.c_int),
                ("seed", C.c_uint64), ("lambda_zero_rel", C.c_double), ("tie_rel", C.c_double)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class _Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC), ("free", _FREE), ("user", C.c_void_p)]


class _Report(C.Structure):
    _fields_ = [("n", C.c_int), ("energy", C.POINTER(C.c_double)), ("iters", C.POINTER(C.c_int)),
                ("eps", C.POINTER(C.c_double)), ("eps_best", C.POINTER(C.c_double)),
                ("fidelity", C.POINTER(C.c_double)), ("bond", C.POINTER(C.c_double)),
                ("kept", C.POINTER(C.c_int)), ("e_g", C.c_double)]


_lib_handle = None


def load_library(path: Optional[str] = None) -> C.CDLL:
    """Load libidmrg.so (built by ``paper_1606_06790_gb300.build``); raises if absent."""
    global _lib_handle
    if _lib_handle is not None and path is None:
        return _lib_handle
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libidmrg.so not found at {p}: run __graft_entry__.build() first "
                          "(the iDMRG path has no CPU fallback)")
    lib = C.CDLL(p)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    P = C.POINTER
    sig = {
        "idmrg_default_opts": (None, [P(_Opts)]),
        "idmrg_create": (i, [P(_MPO), P(_Opts), vp, P(_Allocator), P(vp)]),
        "idmrg_destroy": (None, [vp]),
        "idmrg_last_error": (C.c_char_p, [vp]),
        "idmrg_set_stream": (i, [vp, vp]),
        "idmrg_iteration": (i, [vp, P(i)]),
        "idmrg_psi_layout": (i, [vp, i, P(i), i, P(i), P(sz)]),
        "idmrg_block_basis": (i, [vp, i, i, P(i), i, P(i), P(i)]),
        "idmrg_block_to_host": (i, [vp, i, i, P(d), sz]),
        "idmrg_heff_apply": (i, [vp, i, vp, vp]),
        "idmrg_heff_apply_fp64": (i, [vp, i, vp, vp, i]),
        "idmrg_predict_wavefunction": (i, [vp, i, P(d)]),
        "idmrg_set_start_vector": (i, [vp, i, vp]),
        "idmrg_lanczos_solve": (i, [vp, i, P(d), P(i)]),
        "idmrg_get_psi": (i, [vp, i, P(d), sz]),
        "idmrg_truncate": (i, [vp, i, P(d), P(d), P(i)]),
        "idmrg_get_lambda": (i, [vp, i, P(d), i, P(i)]),
        "idmrg_update_environments": (i, [vp, i]),
        "idmrg_advance": (i, [vp]),
        "idmrg_unit_cell_step": (i, [vp, P(_Report)]),
        "idmrg_batch_step": (i, [vp, i, i, vp]),
        "idmrg_run": (i, [vp, i, d, P(d), P(d), P(i)]),
        "idmrg_truncation_error": (i, [vp, P(d)]),
        "idmrg_energy_per_site": (i, [vp, P(d), P(i)]),
        "idmrg_heff_cost": (i, [vp, i, P(d), P(d)]),
        "idmrg_launch_count": (i, [vp, P(C.c_uint64)]),
        "idmrg_profile_enable": (i, [vp, i]),
        "idmrg_profile_read": (i, [vp, i, P(d), P(C.c_uint64), P(d), P(d)]),
        "idmrg_transfer_bytes": (i, [vp, P(C.c_uint64), P(C.c_uint64)]),
        "idmrg_heff_apply_noalloc": (i, [vp, i, vp, vp]),
        "idmrg_save": (i, [vp, C.c_char_p]),
        "idmrg_load": (i, [vp, C.c_char_p]),
        "idmrg_svd_stats": (i, [vp, P(i), P(i), P(i), P(i), P(d)]),
        "idmrg_set_svd_path": (i, [vp, i]),
        "idmrg_set_jacobi_arithmetic": (i, [vp, i]),
        "idmrg_gemm_tuning": (i, [vp, i, P(i), P(C.c_float), P(i)]),
        "idmrg_set_gemm_tile": (i, [vp, i, i]),
        "idmrg_create_batch": (i, [P(_MPO), i, P(i), P(_Opts), vp, P(_Allocator), P(vp)]),
        "idmrg_ring_energy": (i, [vp, i, P(d), P(i)]),
        "idmrg_set_mixed_restart": (i, [vp, d, i]),
        "idmrg_svd_phase_ms": (i, [vp, P(d)]),
        "idmrg_svd_sweeps32": (i, [vp, P(i), P(d)]),
        "idmrg_correlation": (i, [vp, i, P(d), P(d), P(d), i, P(C.c_int64), P(C.c_int64), P(d)]),
        "idmrg_transfer_spectrum": (i, [vp, d, i, P(d), P(d), P(d), P(i)]),
        "idmrg_delta_pm": (i, [P(d), i, P(d), P(d), P(d)]),
        "idmrg_extrapolate": (i, [P(d), P(d), i, i, P(d), P(d)]),
        "idmrg_fit_correlation_length": (i, [P(d), P(d), i, d, P(d), P(d)]),
        "idmrg_set_pair_range": (i, [vp, i, i]),
        "idmrg_export_pair": (i, [vp, i, vp, sz, P(sz)]),
        "idmrg_import_pair": (i, [vp, i, vp, sz]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib_handle = lib
    return lib


def _dptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def spin_half_dot_terms(phys_charge):
    """The terms of s_i . s_j = Sz Sz + (S+ S- + S- S+) / 2 for a spin-1/2 basis
    whose states carry 2 Sz = phys_charge (one +1, one -1)."""
    qp = np.asarray(phys_charge).ravel()
    if sorted(qp.tolist()) != [-1, 1]:
        raise ValueError("spin 1/2 needs local charges {+1, -1}")
    up, dn = int(np.argmax(qp)), int(np.argmin(qp))
    sz = np.diag(qp.astype(np.float64) / 2.0)
    sp = np.zeros((2, 2))
    sp[up, dn] = 1.0
    return [(sz, sz, 1.0), (sp, sp.T.copy(), 0.5), (sp.T.copy(), sp, 0.5)]


def delta_pm(values):
    """Eqs. diff1, diff2 over bond strengths that translational symmetry makes
    equal: (average, max - average, min - average), by idmrg_delta_pm."""
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).ravel())
    a, dp, dm = C.c_double(), C.c_double(), C.c_double()
    s = load_library().idmrg_delta_pm(_dptr(v, C.c_double), len(v), C.byref(a), C.byref(dp), C.byref(dm))
    if s != 0:
        raise ValueError("delta_pm needs at least one finite value")
    return a.value, dp.value, dm.value


class Context:
    """One parallel-iDMRG problem on the current CUDA device (see include/idmrg.h).

    ``W`` are the site tensors of one period ([a_k, a_{k+1}, d, d] each),
    ``phys_charge`` the 2Sz of the local states, ``bond_charge`` one int array
    per bond (bond k = left of site k)."""

    def __init__(self, W: Sequence[np.ndarray], phys_charge, bond_charge: Sequence[np.ndarray], m: int,
                 prec: str = "fp64", lanczos_tol: float = 1e-12, lanczos_maxit: int = 300,
                 predict: bool = True, seed: int = 0, lambda_zero_rel: float = 1e-12,
                 tie_rel: float = 1e-7, target_charge: int = 0, stream=None):
        self._create([(W, phys_charge, bond_charge)], [m], prec, lanczos_tol, lanczos_maxit, predict, seed,
                     lambda_zero_rel, tie_rel, target_charge, stream)

    @classmethod
    def batch(cls, problems, m, **kw) -> "Context":
        """One context over several independent problems (idmrg_create_batch):
        ``problems`` a list of (W, phys_charge, bond_charge) with the same
        local basis, ``m`` one int or one per problem.  Superblocks are
        numbered problem after problem (``rings``: first superblock and count
        of each); every call steps all of them together."""
        self = cls.__new__(cls)
        ms = list(m) if hasattr(m, "__len__") else [int(m)] * len(problems)
        self._create(list(problems), ms, **kw)
        return self

    def _create(self, problems, ms, prec: str = "fp64", lanczos_tol: float = 1e-12, lanczos_maxit: int = 300,
                predict: bool = True, seed: int = 0, lambda_zero_rel: float = 1e-12, tie_rel: float = 1e-7,
                target_charge: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        if len(problems) < 1 or len(ms) != len(problems):
            raise ValueError("one m per problem")
        self._torch = torch
        self.lib = load_library()
        self.ell = len(problems[0][0])
        self.d = int(np.asarray(problems[0][0][0]).shape[2])
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = []
        mpos = (_MPO * len(problems))()
        self.rings, p0 = [], 0
        for r, (W, phys_charge, bond_charge) in enumerate(problems):
            dims = np.array([w.shape[0] for w in W] + [W[0].shape[0]], dtype=np.int32)
            Wf = np.ascontiguousarray(np.concatenate([np.asarray(w, dtype=np.float64).ravel() for w in W]))
            qp = np.ascontiguousarray(np.asarray(phys_charge, dtype=np.int32))
            bq = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.int32) for b in bond_charge]))
            self._keep += [dims, Wf, qp, bq]
            mpos[r] = _MPO(len(W), int(np.asarray(W[0]).shape[2]), _dptr(dims, C.c_int), _dptr(Wf, C.c_double),
                           _dptr(qp, C.c_int), _dptr(bq, C.c_int))
            self.rings.append((p0, len(W) // 2))
            p0 += len(W) // 2
        self.P = p0
        self._qp = self._keep[2]
        self._ms = np.ascontiguousarray(np.asarray(ms, dtype=np.int32))
        o = _Opts()
        self.lib.idmrg_default_opts(C.byref(o))
        o.m, o.target_charge, o.lanczos_tol, o.lanczos_maxit = int(max(ms)), target_charge, lanczos_tol, lanczos_maxit
        o.prec, o.predict, o.seed = PREC[prec], int(bool(predict)), seed
        o.lambda_zero_rel, o.tie_rel = lambda_zero_rel, tie_rel
        self.opts = o
        self.prec = prec
        # torch caching allocator as the library's device memory provider
        dev, st = self.device, self.stream

        self.alloc_calls = 0

        def _alloc(nbytes, user):
            self.alloc_calls += 1
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=st)
            except Exception:  # out of memory -> NULL -> IDMRG_ENOMEM
                return None

        def _free(ptr, nbytes, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (_ALLOC(_alloc), _FREE(_free))
        self._alloc = _Allocator(self._cb[0], self._cb[1], None)
        h = C.c_void_p()
        if len(problems) == 1:
            s = self.lib.idmrg_create(C.byref(mpos[0]), C.byref(o), C.c_void_p(self.stream.cuda_stream),
                                      C.byref(self._alloc), C.byref(h))
        else:
            s = self.lib.idmrg_create_batch(mpos, len(problems), _dptr(self._ms, C.c_int), C.byref(o),
                                            C.c_void_p(self.stream.cuda_stream), C.byref(self._alloc), C.byref(h))
        if s != 0:
            raise IdmrgError(s, "idmrg_create failed (invalid MPO or options, or no device memory)")
        self.h = h

    def ring_energy(self, r: int):
        """Problem r's latest Step 5' estimate (e_g, n), or None before the first."""
        e, n = C.c_double(), C.c_int()
        s = self._check(self.lib.idmrg_ring_energy(self.h, int(r), C.byref(e), C.byref(n)), "ring_energy", ok=(0, 7))
        return None if s != 0 else (e.value, n.value)

    # ------------------------------------------------------------ helpers
    def _check(self, s: int, what: str, ok=(0,)):
        if s not in ok:
            raise IdmrgError(s, f"{what}: {self.lib.idmrg_last_error(self.h).decode()}")
        return s

    def close(self):
        if getattr(self, "h", None):
            self.lib.idmrg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _n_of(self, p: int) -> int:
        return self.P if p < 0 else 1

    # ------------------------------------------------------------ queries
    @property
    def iteration(self) -> int:
        n = C.c_int()
        self._check(self.lib.idmrg_iteration(self.h, C.byref(n)), "iteration")
        return n.value

    def psi_layout(self, p: int):
        """(descriptor array [nblocks, 8], vector length); see idmrg_psi_layout."""
        nb, ne = C.c_int(), C.c_size_t()
        self._check(self.lib.idmrg_psi_layout(self.h, p, None, 0, C.byref(nb), C.byref(ne)), "psi_layout")
        desc = np.zeros((max(nb.value, 1), 8), dtype=np.int32)
        self._check(self.lib.idmrg_psi_layout(self.h, p, _dptr(desc, C.c_int), nb.value, C.byref(nb),
                                              C.byref(ne)), "psi_layout")
        return desc[: nb.value], ne.value

    def block_basis(self, p: int, side: int):
        D, w = C.c_int(), C.c_int()
        self._check(self.lib.idmrg_block_basis(self.h, p, side, None, 0, C.byref(D), C.byref(w)), "block_basis")
        q = np.zeros(max(D.value, 1), dtype=np.int32)
        self._check(self.lib.idmrg_block_basis(self.h, p, side, _dptr(q, C.c_int), D.value, C.byref(D),
                                               C.byref(w)), "block_basis")
        return q[: D.value], w.value

    def block_to_host(self, p: int, side: int) -> np.ndarray:
        q, w = self.block_basis(p, side)
        D = len(q)
        out = np.zeros((w, D, D))
        self._check(self.lib.idmrg_block_to_host(self.h, p, side, _dptr(out, C.c_double), out.size),
                    "block_to_host")
        return out

    # ------------------------------------------------------------ steps
    def heff_apply(self, p: int, psi, out) -> None:
        """out = H_eff psi; psi/out are float64 CUDA tensors in the layout of p."""
        self._check(self.lib.idmrg_heff_apply(self.h, p, C.c_void_p(psi.data_ptr()), C.c_void_p(out.data_ptr())),
                    "heff_apply")

    def heff_apply_fp64(self, p: int, psi, out, form: int) -> None:
        """out = H_eff psi in an FP64-accurate form: 0 = FP64 GEMMs, 1 = BF16
        digit slices on the tensor cores (mixed-precision contexts)."""
        self._check(self.lib.idmrg_heff_apply_fp64(self.h, p, C.c_void_p(psi.data_ptr()),
                                                   C.c_void_p(out.data_ptr()), form), "heff_apply_fp64")

    def predict_wavefunction(self, p: int = -1) -> np.ndarray:
        out = np.zeros(self._n_of(p))
        self._check(self.lib.idmrg_predict_wavefunction(self.h, p, _dptr(out, C.c_double)), "predict_wavefunction")
        return out

    def set_start_vector(self, p: int, psi) -> None:
        """Start vector of the next solve (float64 CUDA tensor in the layout of
        p, or all superblocks' vectors concatenated for p = -1)."""
        self._check(self.lib.idmrg_set_start_vector(self.h, p, C.c_void_p(psi.data_ptr())), "set_start_vector")

    def lanczos_solve(self, p: int = -1):
        e = np.zeros(self._n_of(p))
        it = np.zeros(self._n_of(p), dtype=np.int32)
        s = self._check(self.lib.idmrg_lanczos_solve(self.h, p, _dptr(e, C.c_double), _dptr(it, C.c_int)),
                        "lanczos_solve", ok=(0, 4))
        return e, it, s == 0

    def get_psi(self, p: int) -> np.ndarray:
        _, N = self.psi_layout(p)
        out = np.zeros(N)
        self._check(self.lib.idmrg_get_psi(self.h, p, _dptr(out, C.c_double), N), "get_psi")
        return out

    def truncate(self, p: int = -1):
        k = self._n_of(p)
        eps, epsb, kept = np.zeros(k), np.zeros(k), np.zeros(k, dtype=np.int32)
        self._check(self.lib.idmrg_truncate(self.h, p, _dptr(eps, C.c_double), _dptr(epsb, C.c_double),
                                            _dptr(kept, C.c_int)), "truncate")
        return eps, epsb, kept

    def get_lambda(self, p: int) -> np.ndarray:
        n = C.c_int()
        self._check(self.lib.idmrg_get_lambda(self.h, p, None, 0, C.byref(n)), "get_lambda")
        out = np.zeros(max(n.value, 1))
        self._check(self.lib.idmrg_get_lambda(self.h, p, _dptr(out, C.c_double), n.value, C.byref(n)),
                    "get_lambda")
        return out[: n.value]

    def update_environments(self, p: int = -1) -> None:
        self._check(self.lib.idmrg_update_environments(self.h, p), "update_environments")

    def advance(self) -> None:
        self._check(self.lib.idmrg_advance(self.h), "advance")

    def run(self, max_steps: int, de_tol: float = 1e-8):
        """Unit-cell steps until successive e_g estimates differ by less than
        de_tol (or max_steps): (e_g, eps, steps, converged)."""
        eg, eps, k = C.c_double(), C.c_double(), C.c_int()
        s = self._check(self.lib.idmrg_run(self.h, int(max_steps), float(de_tol), C.byref(eg), C.byref(eps),
                                           C.byref(k)), "run", ok=(0, 4))
        return eg.value, eps.value, k.value, s == 0

    def truncation_error(self) -> float:
        """Largest eps^(n)_1 over the last l iterations (Eq. tru)."""
        e = C.c_double()
        self._check(self.lib.idmrg_truncation_error(self.h, C.byref(e)), "truncation_error")
        return e.value

    # ---- uniform-MPS observables (Eq. mps2)
    def correlation(self, terms, pairs) -> np.ndarray:
        """sum_t coef_t <(A_t)_i (B_t)_j> for each (i, j) in pairs (lattice
        sites, i < j); terms is a list of (A, B, coef) with d x d operators
        <s|O|t> in the MPO's physical basis."""
        d = self.d
        opa = np.ascontiguousarray(np.array([np.asarray(t[0], dtype=np.float64).reshape(d, d) for t in terms]))
        opb = np.ascontiguousarray(np.array([np.asarray(t[1], dtype=np.float64).reshape(d, d) for t in terms]))
        coef = np.ascontiguousarray(np.array([float(t[2]) for t in terms]))
        pr = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
        si = np.ascontiguousarray(pr[:, 0])
        sj = np.ascontiguousarray(pr[:, 1])
        out = np.zeros(len(pr))
        self._check(self.lib.idmrg_correlation(self.h, len(terms), _dptr(opa, C.c_double), _dptr(opb, C.c_double),
                                               _dptr(coef, C.c_double), len(pr), _dptr(si, C.c_int64),
                                               _dptr(sj, C.c_int64), _dptr(out, C.c_double)), "correlation")
        return out

    def spin_dot(self, pairs) -> np.ndarray:
        """<s_i . s_j> for spin 1/2 (bond strengths, spin-spin correlations)."""
        return self.correlation(spin_half_dot_terms(self._qp), pairs)

    def transfer_spectrum(self, tol: float = 1e-10, maxit: int = 2000):
        """(t1, |t2|, xi in unit cells, iterations, converged) of the unit's transfer map."""
        t1, t2, xi, it = C.c_double(), C.c_double(), C.c_double(), C.c_int()
        s = self._check(self.lib.idmrg_transfer_spectrum(self.h, float(tol), int(maxit), C.byref(t1), C.byref(t2),
                                                         C.byref(xi), C.byref(it)), "transfer_spectrum", ok=(0, 4))
        return t1.value, t2.value, xi.value, it.value, s == 0

    def _report(self):
        P = self.P
        arr = {k: np.zeros(P) for k in ("energy", "eps", "eps_best", "fidelity", "bond")}
        iarr = {k: np.zeros(P, dtype=np.int32) for k in ("iters", "kept")}
        rep = _Report(0, _dptr(arr["energy"], C.c_double), _dptr(iarr["iters"], C.c_int),
                      _dptr(arr["eps"], C.c_double), _dptr(arr["eps_best"], C.c_double),
                      _dptr(arr["fidelity"], C.c_double), _dptr(arr["bond"], C.c_double),
                      _dptr(iarr["kept"], C.c_int), float("nan"))
        return rep, arr, iarr

    @staticmethod
    def _report_dict(rep, arr, iarr, converged: bool) -> Dict[str, object]:
        out: Dict[str, object] = dict(n=rep.n, converged=converged, **arr, **iarr)
        out["e_g"] = None if math.isnan(rep.e_g) else rep.e_g
        return out

    def unit_cell_step(self) -> Dict[str, object]:
        rep, arr, iarr = self._report()
        s = self._check(self.lib.idmrg_unit_cell_step(self.h, C.byref(rep)), "unit_cell_step", ok=(0, 4))
        return self._report_dict(rep, arr, iarr, s == 0)

    # ---- one problem over several workers (shard.ShardedRun)
    def step_range(self, p0: int, p1: int) -> Dict[str, object]:
        """One unit-cell step of superblocks p0..p1-1 (idmrg_set_pair_range
        when the range changes, then idmrg_unit_cell_step)."""
        if getattr(self, "_range", (0, self.P)) != (p0, p1):
            self._check(self.lib.idmrg_set_pair_range(self.h, int(p0), int(p1)), "set_pair_range")
            self._range = (p0, p1)
        return self.unit_cell_step()

    def export_pair(self, q: int) -> bytes:
        """Pair q's R^(n) and truncation after a step (idmrg_export_pair)."""
        n = C.c_size_t()
        self._check(self.lib.idmrg_export_pair(self.h, int(q), None, 0, C.byref(n)), "export_pair")
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.idmrg_export_pair(self.h, int(q), buf, n.value, C.byref(n)), "export_pair")
        return buf.raw[: n.value]

    def import_pair(self, q: int, data: bytes) -> None:
        """The next worker's first pair after the same step (idmrg_import_pair)."""
        buf = C.create_string_buffer(bytes(data), len(data))
        self._check(self.lib.idmrg_import_pair(self.h, int(q), buf, len(data)), "import_pair")

    def save(self, path: str) -> None:
        """Checkpoint between steps (idmrg_save)."""
        self._check(self.lib.idmrg_save(self.h, os.fsencode(path)), "save")

    def load(self, path: str) -> None:
        """Restore a checkpoint of the same MPO and options (idmrg_load)."""
        self._check(self.lib.idmrg_load(self.h, os.fsencode(path)), "load")

    def energy_per_site(self):
        e, n = C.c_double(), C.c_int()
        s = self.lib.idmrg_energy_per_site(self.h, C.byref(e), C.byref(n))
        return (e.value, n.value) if s == 0 else (None, None)

    def heff_cost(self, p: int = -1):
        f, b = C.c_double(), C.c_double()
        self._check(self.lib.idmrg_heff_cost(self.h, p, C.byref(f), C.byref(b)), "heff_cost")
        return f.value, b.value

    def launch_count(self) -> int:
        n = C.c_uint64()
        self._check(self.lib.idmrg_launch_count(self.h, C.byref(n)), "launch_count")
        return int(n.value)

    def profile_enable(self, on: bool = True) -> None:
        self._check(self.lib.idmrg_profile_enable(self.h, int(on)), "profile_enable")

    def profile_read(self) -> Dict[str, Dict[str, float]]:
        """Per kernel class: device ms, launches, algorithmic flops and bytes."""
        out = {}
        for name, k in KERNEL_CLASSES.items():
            ms, n, f, b = C.c_double(), C.c_uint64(), C.c_double(), C.c_double()
            self._check(self.lib.idmrg_profile_read(self.h, k, C.byref(ms), C.byref(n), C.byref(f), C.byref(b)),
                        "profile_read")
            out[name] = dict(ms=ms.value, launches=int(n.value), flops=f.value, bytes=b.value)
        return out

    def set_svd_path(self, global_only: bool) -> None:
        """Sector SVDs on the large-sector (global-memory) kernels only."""
        self._check(self.lib.idmrg_set_svd_path(self.h, int(bool(global_only))), "set_svd_path")

    JACOBI_ARITHMETIC = {"auto": 0, "fp64": 1, "pairs": 2}

    def set_jacobi_arithmetic(self, mode: str) -> None:
        """Arithmetic of the final Jacobi of large sectors: "fp64", "pairs"
        (FP32 pairs) or "auto" (pairs for the mixed precisions)."""
        self._check(self.lib.idmrg_set_jacobi_arithmetic(self.h, self.JACOBI_ARITHMETIC[mode]),
                    "set_jacobi_arithmetic")

    def svd_stats(self) -> Dict[str, float]:
        j, mc, mr, ms, me = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_double()
        self._check(self.lib.idmrg_svd_stats(self.h, C.byref(j), C.byref(mc), C.byref(mr), C.byref(ms), C.byref(me)),
                    "svd_stats")
        m32, e32 = C.c_int(), C.c_double()
        self._check(self.lib.idmrg_svd_sweeps32(self.h, C.byref(m32), C.byref(e32)), "svd_sweeps32")
        return dict(jobs=j.value, max_cols=mc.value, max_rank=mr.value, max_sweeps=ms.value, mean_sweeps=me.value,
                    max_sweeps32=m32.value, mean_sweeps32=e32.value)

    SVD_PHASES = ("qr", "jacobi32", "newton_schulz_xbv", "jacobi64", "select", "compact")

    def svd_phase_ms(self) -> Dict[str, float]:
        """Event-timed milliseconds of the SVD's phases since profiling was enabled."""
        ms = (C.c_double * len(self.SVD_PHASES))()
        self._check(self.lib.idmrg_svd_phase_ms(self.h, ms), "svd_phase_ms")
        return {k: ms[i] for i, k in enumerate(self.SVD_PHASES)}

    def set_mixed_restart(self, inner_factor: float, inner_cap: int) -> None:
        """Restart rule of the mixed-precision Lanczos (idmrg_set_mixed_restart)."""
        self._check(self.lib.idmrg_set_mixed_restart(self.h, float(inner_factor), int(inner_cap)),
                    "set_mixed_restart")

    def set_gemm_tile(self, tn1: int, tn3: int) -> None:
        """Fix the N tiles of H_eff stages 1 and 3 (0 = tuned) from the next plan on."""
        self._check(self.lib.idmrg_set_gemm_tile(self.h, tn1, tn3), "set_gemm_tile")

    def gemm_tuning(self, stage: int) -> Dict[str, object]:
        """The tuner's N tile for H_eff stage 1 or 3 and its candidates' times."""
        tn, nt = C.c_int(), C.c_int()
        ms = (C.c_float * 3)()
        self._check(self.lib.idmrg_gemm_tuning(self.h, stage, C.byref(tn), ms, C.byref(nt)), "gemm_tuning")
        return dict(tn=tn.value, ms={64: ms[0], 128: ms[1], 256: ms[2]}, tunings=nt.value)

    def transfer_bytes(self):
        a, b = C.c_uint64(), C.c_uint64()
        self._check(self.lib.idmrg_transfer_bytes(self.h, C.byref(a), C.byref(b)), "transfer_bytes")
        return int(a.value), int(b.value)


def batch_step(contexts: Sequence["Context"], threads: int = 16) -> List[Dict[str, object]]:
    """One unit-cell step of every context (independent problems, e.g. disorder
    realisations), run concurrently on `threads` host threads; each context
    must have its own CUDA stream.  Returns the step reports in order."""
    if not contexts:
        return []
    lib = contexts[0].lib
    reps = [c._report() for c in contexts]
    arr = (_Report * len(contexts))(*[r[0] for r in reps])
    hs = (C.c_void_p * len(contexts))(*[c.h for c in contexts])
    s = lib.idmrg_batch_step(C.cast(hs, C.c_void_p), len(contexts), int(threads), C.cast(arr, C.c_void_p))
    if s not in (0, 4):
        raise IdmrgError(s, "batch_step: " + "; ".join(
            c.lib.idmrg_last_error(c.h).decode() for c in contexts if c.lib.idmrg_last_error(c.h)))
    out = []
    for i, (_, a, ia) in enumerate(reps):
        out.append(Context._report_dict(arr[i], a, ia, True))
    return out


def layout_pack(desc: np.ndarray, N: int, dense: np.ndarray) -> np.ndarray:
    """Copy a dense psi[x, s, t, y] into the library's block layout (data movement only)."""
    out = np.zeros(N)
    for x0, Dx, s, t, y0, Dy, off, ld in desc:
        blk = dense[x0:x0 + Dx, s, t, y0:y0 + Dy]
        for i in range(Dx):
            out[off + i * ld: off + i * ld + Dy] = blk[i]
    return out


def layout_unpack(desc: np.ndarray, vec: np.ndarray, shape) -> np.ndarray:
    """Inverse of ``layout_pack`` (zeros outside the charge-allowed blocks)."""
    dense = np.zeros(shape)
    for x0, Dx, s, t, y0, Dy, off, ld in desc:
        for i in range(Dx):
            dense[x0 + i, s, t, y0:y0 + Dy] = vec[off + i * ld: off + i * ld + Dy]
    return dense
