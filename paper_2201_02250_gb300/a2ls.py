"""Thin Python binding of libA2LS (include/a2ls.h) over ctypes.

Argument marshalling only: every step of setup, apply and solve runs in the
CUDA library.  PyTorch provides device memory and the current stream.  The
binding fails loudly when the library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import _build

A2LS_OK, A2LS_ERR_ARG, A2LS_ERR_SINGULAR, A2LS_ERR_NOT_CONVERGED = 0, 1, 2, 3
A2LS_ERR_EIGEN, A2LS_ERR_TIMEOUT, A2LS_ERR_CUDA, A2LS_ERR_OOM, A2LS_ERR_STATE = 4, 5, 6, 7, 8
FP64, FP32, FP32X2, BF16 = 0, 1, 2, 3
VARIANTS = {"deflated_ras": 0, "deflated_asm": 1, "additive_ras": 2, "additive_asm": 3, "ras": 4, "asm": 5}
POU = {"boolean": 0, "multiplicity": 1}
(Q_SIZES, Q_SUBDOMAINS, Q_LUMP, Q_FACTORS, Q_COARSE, Q_EIGVALS, Q_TIMES, Q_EINV, Q_EIGSTATS, Q_LAUNCHES,
 Q_KERNEL_TIMES, Q_TUNING, Q_EIG_UNCONVERGED, Q_ENVELOPE, Q_EIGRES, Q_PIVOT_BOOSTS) = range(16)
TRACKED_KERNELS = ["lu_local", "lu_splitting", "eig_triangular_solves", "eig_orthogonalisation",
                   "eig_rayleigh_ritz", "coarse_lu", "coarse_inverse", "apply_local_solves"]
PHASES = ["graph", "extract", "lu", "eig_coarse", "coarse", "setup_total", "solve_total", "apply", "apply_prep"]


class A2lsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"a2ls error {code}: {msg}")
        self.code = code


class CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("rowptr", ctypes.c_void_p),
                ("colind", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("variant", ctypes.c_int32), ("pou", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("max_it", ctypes.c_int32), ("flexible", ctypes.c_int32),
                ("tau", ctypes.c_double), ("eig_block_steps", ctypes.c_int32),
                ("eig_max_cycles", ctypes.c_int32), ("eig_tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("timing", ctypes.c_int32),
                ("eig_precision", ctypes.c_int32), ("graphs", ctypes.c_int32), ("warm_start", ctypes.c_void_p),
                ("eig_strict", ctypes.c_int32), ("eig_stall_cycles", ctypes.c_int32),
                ("tensor_cores", ctypes.c_int32), ("eig_thick_restart", ctypes.c_int32),
                ("local_solve_kernel", ctypes.c_int32), ("eig_block_size", ctypes.c_int32),
                ("static_pivoting", ctypes.c_int32)]


_LIB = None


def header_functions() -> list:
    """Names of the functions declared in include/a2ls.h."""
    path = os.path.join(_build.ROOT, "include", "a2ls.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(a2ls_\w+)\s*\(", text)))


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libA2LS.so (building it first if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libA2LS.so not found at {path}; run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    L.a2ls_default_options.argtypes = [ctypes.POINTER(Options)]
    L.a2ls_default_options.restype = None
    L.a2ls_setup.argtypes = [ctypes.POINTER(CSR), vp, i32, i32, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    L.a2ls_apply.argtypes = [vp, vp, vp]
    L.a2ls_solve.argtypes = [vp, vp, vp, f64, ctypes.POINTER(i32), ctypes.POINTER(f64)]
    L.a2ls_destroy.argtypes = [vp]
    L.a2ls_destroy.restype = None
    L.a2ls_last_error.argtypes = []
    L.a2ls_last_error.restype = ctypes.c_char_p
    L.a2ls_query.argtypes = [vp, i32, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.a2ls_set_coarse_basis.argtypes = [vp, vp, vp]
    L.a2ls_spmv.argtypes = [vp, vp, vp]
    L.a2ls_apply_static.argtypes = [vp, vp, vp]
    L.a2ls_solve_multi.argtypes = [vp, i32, vp, vp, f64, vp, vp]
    L.a2ls_setup_batch.argtypes = [i32, vp, vp, vp, vp, ctypes.POINTER(Options), vp]
    L.a2ls_trim_memory.argtypes = []
    L.a2ls_partition.argtypes = [i32, vp, vp, i32, ctypes.c_uint64, vp]
    for f in ("a2ls_setup", "a2ls_apply", "a2ls_solve", "a2ls_query", "a2ls_set_coarse_basis", "a2ls_spmv",
              "a2ls_apply_static", "a2ls_solve_multi", "a2ls_setup_batch", "a2ls_trim_memory", "a2ls_partition"):
        getattr(L, f).restype = ctypes.c_int
    # learned warm start
    i64 = ctypes.c_int64
    L.a2ls_gnn_num_params.argtypes = []
    L.a2ls_gnn_num_params.restype = i64
    L.a2ls_gnn_launches.argtypes = [vp]
    L.a2ls_gnn_launches.restype = i64
    L.a2ls_gnn_create.argtypes = [ctypes.c_uint64, vp, ctypes.POINTER(vp)]
    L.a2ls_gnn_destroy.argtypes = [vp]
    L.a2ls_gnn_get_params.argtypes = [vp, vp, i64]
    L.a2ls_gnn_set_params.argtypes = [vp, vp, i64]
    L.a2ls_gnn_get_grads.argtypes = [vp, vp, i64]
    L.a2ls_gnn_sample_create.argtypes = [vp, ctypes.POINTER(vp)]
    L.a2ls_gnn_sample_set_target.argtypes = [vp, vp, vp]
    L.a2ls_gnn_sample_destroy.argtypes = [vp]
    L.a2ls_gnn_sample_query.argtypes = [vp, i32, vp, i64, ctypes.POINTER(i64)]
    L.a2ls_gnn_forward.argtypes = [vp, vp, vp]
    L.a2ls_gnn_loss_grad.argtypes = [vp, vp, ctypes.POINTER(f64)]
    L.a2ls_gnn_adam_step.argtypes = [vp, f64]
    for f in ("a2ls_gnn_create", "a2ls_gnn_destroy", "a2ls_gnn_get_params", "a2ls_gnn_set_params",
              "a2ls_gnn_get_grads", "a2ls_gnn_sample_create", "a2ls_gnn_sample_set_target",
              "a2ls_gnn_sample_destroy", "a2ls_gnn_sample_query", "a2ls_gnn_forward", "a2ls_gnn_loss_grad",
              "a2ls_gnn_adam_step"):
        getattr(L, f).restype = ctypes.c_int
    _LIB = L
    return L


def _check(rc: int, allow=()):
    if rc != A2LS_OK and rc not in allow:
        raise A2lsError(rc, lib().a2ls_last_error().decode())
    return rc


def default_options(**kw) -> Options:
    o = Options()
    lib().a2ls_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        if k == "pou" and isinstance(v, str):
            v = POU[v]
        if k in ("precision", "eig_precision") and isinstance(v, str):
            v = {"fp64": FP64, "fp32": FP32, "fp32x2": FP32X2, "bf16": BF16}[v]
        if k == "warm_start":
            v = None if v is None else v._g.value
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    return int(t.data_ptr())


class Preconditioner:
    """Handle on a set-up two-level Schwarz preconditioner (device data owned by the library).

    rowptr, colind (int32), val (float64) and part (int32) are CUDA tensors.
    """

    def __init__(self, rowptr, colind, val, part, overlap: int, nev: int, stream=None, **opts):
        import torch
        for t, dt in ((rowptr, torch.int32), (colind, torch.int32), (val, torch.float64), (part, torch.int32)):
            if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
                raise ValueError("CSR and partition must be contiguous CUDA tensors (int32 / float64)")
        self.n = int(rowptr.numel() - 1)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o = default_options(**opts)
        o.stream = ctypes.c_void_p(int(stream.cuda_stream))
        self.options = o
        self._warm = opts.get("warm_start")  # the network must outlive the setup call
        csr = CSR(self.n, int(colind.numel()), _ptr(rowptr), _ptr(colind), _ptr(val))
        h = ctypes.c_void_p()
        _check(lib().a2ls_setup(ctypes.byref(csr), ctypes.c_void_p(_ptr(part)), int(overlap), int(nev),
                                ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().a2ls_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, r, z):
        _check(lib().a2ls_apply(self._h, ctypes.c_void_p(_ptr(r)), ctypes.c_void_p(_ptr(z))))

    def apply_static(self, r, z):
        """Same as apply, with scratch from the library's fixed static device array (no allocation)."""
        _check(lib().a2ls_apply_static(self._h, ctypes.c_void_p(_ptr(r)), ctypes.c_void_p(_ptr(z))))

    def spmv(self, x, y):
        _check(lib().a2ls_spmv(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(y))))

    def solve(self, b, x, rtol: float = 1e-8, allow_not_converged: bool = False):
        it = ctypes.c_int32()
        rr = ctypes.c_double()
        rc = lib().a2ls_solve(self._h, ctypes.c_void_p(_ptr(b)), ctypes.c_void_p(_ptr(x)), float(rtol),
                              ctypes.byref(it), ctypes.byref(rr))
        _check(rc, allow=(A2LS_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return int(it.value), float(rr.value), rc == A2LS_OK

    def solve_multi(self, B, X, rtol: float = 1e-8, allow_not_converged: bool = False):
        """B, X: CUDA float64 tensors of shape (nrhs, n), one right-hand side per row."""
        nrhs = int(B.shape[0])
        it = np.zeros(nrhs, dtype=np.int32)
        rr = np.zeros(nrhs, dtype=np.float64)
        rc = lib().a2ls_solve_multi(self._h, nrhs, ctypes.c_void_p(_ptr(B)), ctypes.c_void_p(_ptr(X)), float(rtol),
                                    it.ctypes.data, rr.ctypes.data)
        _check(rc, allow=(A2LS_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return it, rr, rc == A2LS_OK

    # --- queries ------------------------------------------------------------------
    def _query(self, what: int) -> bytes:
        need = ctypes.c_int64()
        _check(lib().a2ls_query(self._h, what, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(max(int(need.value), 1))
        _check(lib().a2ls_query(self._h, what, buf, int(need.value), None))
        return buf.raw[:int(need.value)]

    def sizes(self) -> dict:
        s = np.frombuffer(self._query(Q_SIZES), dtype=np.int64)
        return {"n": int(s[0]), "N": int(s[1]), "n0": int(s[2]), "sum_ni": int(s[3]), "max_ni": int(s[4]),
                "w_elems": int(s[5]), "precision": int(s[6]), "variant": int(s[7])}

    def subdomains(self) -> list:
        """[(interior indices, overlap indices)] per subdomain, in the library's local order."""
        N = self.sizes()["N"]
        raw = np.frombuffer(self._query(Q_SUBDOMAINS), dtype=np.int32)
        off, nI, idx = raw[:N + 1], raw[N + 1:2 * N + 1], raw[2 * N + 1:]
        return [(idx[off[i]:off[i] + nI[i]].copy(), idx[off[i] + nI[i]:off[i + 1]].copy()) for i in range(N)]

    def lump(self) -> list:
        N = self.sizes()["N"]
        raw = np.frombuffer(self._query(Q_SUBDOMAINS), dtype=np.int32)
        off = raw[:N + 1]
        s = np.frombuffer(self._query(Q_LUMP), dtype=np.float64)
        return [s[off[i]:off[i + 1]].copy() for i in range(N)]

    def factors(self) -> list:
        """Per subdomain the stored block-inverted LU (n_i x n_i, float64 view)."""
        sz = self.sizes()
        N = sz["N"]
        raw = self._query(Q_FACTORS)
        tail = (N + 1) * 8 + N * 4
        if sz["precision"] == BF16:   # bfloat16: the upper half of an FP32 value
            bits = np.frombuffer(raw[:len(raw) - tail], dtype=np.uint16).astype(np.uint32) << 16
            vals = bits.view(np.float32)
        else:
            vals = np.frombuffer(raw[:len(raw) - tail], dtype=np.float64 if sz["precision"] == FP64 else np.float32)
        foff = np.frombuffer(raw[len(raw) - tail:len(raw) - N * 4], dtype=np.int64)
        ld = np.frombuffer(raw[len(raw) - N * 4:], dtype=np.int32)
        subs = self.subdomains()
        out = []
        for i in range(N):
            n_i = len(subs[i][0]) + len(subs[i][1])
            F = vals[foff[i]:foff[i] + n_i * ld[i]].reshape(n_i, ld[i])[:, :n_i].astype(np.float64)
            out.append(F)
        return out

    def coarse_basis(self) -> list:
        N = self.sizes()["N"]
        raw = self._query(Q_COARSE)
        m = np.frombuffer(raw[:4 * N], dtype=np.int32)
        W = np.frombuffer(raw[4 * N:], dtype=np.float64)
        subs = self.subdomains()
        out, o = [], 0
        for i in range(N):
            n_i = len(subs[i][0]) + len(subs[i][1])
            out.append(W[o:o + n_i * m[i]].reshape(n_i, m[i]).copy())
            o += n_i * m[i]
        return out

    def eigenvalues(self) -> np.ndarray:
        N = self.sizes()["N"]
        ev = np.frombuffer(self._query(Q_EIGVALS), dtype=np.float64)
        if ev.size == 0:
            return np.zeros((N, 0), dtype=complex)
        ev = ev.reshape(N, -1, 2)
        return ev[..., 0] + 1j * ev[..., 1]

    def eig_stats(self) -> np.ndarray:
        N = self.sizes()["N"]
        s = np.frombuffer(self._query(Q_EIGSTATS), dtype=np.int32)
        return s.reshape(N, 2) if s.size else np.zeros((N, 2), dtype=np.int32)

    def times(self) -> dict:
        t = np.frombuffer(self._query(Q_TIMES), dtype=np.float64)
        return {k: float(t[i]) for i, k in enumerate(PHASES)}

    def tuning(self) -> dict:
        v = np.frombuffer(self._query(Q_TUNING), dtype=np.int32)
        return {"local_solve_threads": int(v[0]), "apply_graphs": int(v[1])}

    def envelope(self) -> np.ndarray:
        """(N, 4): envelope LU flops (all pivots, overlap pivots), L row-envelope and U column-envelope entries."""
        return np.frombuffer(self._query(Q_ENVELOPE), dtype=np.float64).reshape(-1, 4).copy()

    def eig_unconverged(self) -> int:
        """Subdomains whose local eigensolve stopped without reaching eig_tol."""
        return int(np.frombuffer(self._query(Q_EIG_UNCONVERGED), dtype=np.int32)[0])

    def eig_stalled(self) -> int:
        """Subdomains of eig_unconverged() that the stagnation stop ended."""
        return int(np.frombuffer(self._query(Q_EIG_UNCONVERGED), dtype=np.int32)[1])

    def pivot_boosts(self) -> int:
        """Local LU pivots replaced under static pivoting (0 without the option)."""
        return int(np.frombuffer(self._query(Q_PIVOT_BOOSTS), dtype=np.int32)[0])

    def eig_residuals(self) -> np.ndarray:
        """(N,): largest relative residual of the wanted Ritz pairs at each subdomain's last cycle."""
        return np.frombuffer(self._query(Q_EIGRES), dtype=np.float64).copy()

    def launches(self) -> int:
        return int(np.frombuffer(self._query(Q_LAUNCHES), dtype=np.int64)[0])

    def kernel_times(self) -> dict:
        """{kernel: (launches, total ms, algorithmic work)} for the tracked kernels (needs timing=1);
        work is flops, or bytes moved for the apply local solves."""
        v = np.frombuffer(self._query(Q_KERNEL_TIMES), dtype=np.float64).reshape(-1, 3)
        return {k: (int(v[i, 0]), float(v[i, 1]), float(v[i, 2])) for i, k in enumerate(TRACKED_KERNELS)}

    def coarse_inverse(self) -> np.ndarray:
        n0 = self.sizes()["n0"]
        return np.frombuffer(self._query(Q_EINV), dtype=np.float64).reshape(n0, n0).copy()

    def set_coarse_basis(self, W: list):
        m = np.array([w.shape[1] for w in W], dtype=np.int32)
        flat = np.concatenate([np.ascontiguousarray(w, dtype=np.float64).ravel() for w in W]) if len(W) else \
            np.zeros(1)
        flat = np.ascontiguousarray(flat)
        _check(lib().a2ls_set_coarse_basis(self._h, m.ctypes.data_as(ctypes.c_void_p),
                                           flat.ctypes.data_as(ctypes.c_void_p)))


def trim_memory() -> None:
    """Return the unused blocks of the library's device memory pools to the system (a2ls_trim_memory)."""
    _check(lib().a2ls_trim_memory())


def partition(rowptr, colind, nparts: int, seed: int = 0) -> np.ndarray:
    """k-way partition of the graph of A + A^T (a2ls_partition, host side, no GPU needed).

    rowptr, colind: the CSR pattern of A as host arrays; returns part (int32, n values in [0, nparts)).
    """
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    n = int(rp.size - 1)
    part = np.empty(max(n, 0), dtype=np.int32)
    _check(lib().a2ls_partition(n, ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.ctypes.data if ci.size else 0),
                                int(nparts), ctypes.c_uint64(seed), ctypes.c_void_p(part.ctypes.data)))
    return part


def resolve_partition(A, part, seed: int = 0) -> np.ndarray:
    """The partition array for A: `part` itself (n part ids), or, when `part` is an int N, the
    partition of the graph of A + A^T into N parts by a2ls_partition."""
    if isinstance(part, (int, np.integer)):
        return partition(A.indptr, A.indices, int(part), seed=seed)
    p = np.asarray(part, dtype=np.int32)
    if p.shape != (A.shape[0],):
        raise ValueError(f"partition has shape {p.shape}, expected ({A.shape[0]},)")
    return p


def from_scipy(A, part, overlap: int, nev: int, device: str = "cuda", **opts):
    """Upload a scipy CSR matrix and partition, then set up; returns (Preconditioner, device tensors).

    part: n part ids, or an int N to partition the graph of A + A^T into N parts (a2ls_partition)."""
    import torch
    rowptr = torch.as_tensor(np.asarray(A.indptr, dtype=np.int32), device=device)
    colind = torch.as_tensor(np.asarray(A.indices, dtype=np.int32), device=device)
    val = torch.as_tensor(np.asarray(A.data, dtype=np.float64), device=device)
    p = torch.as_tensor(resolve_partition(A, part), device=device)
    P = Preconditioner(rowptr, colind, val, p, overlap, nev, **opts)
    return P, (rowptr, colind, val, p)


# ---------------------------------------------------------------------------------------------
# learned warm start of the local eigensolves
# ---------------------------------------------------------------------------------------------
GQ_FEATURES, GQ_ROWPTR, GQ_COLS, GQ_WEIGHTS, GQ_SWEIGHTS, GQ_TARGET_COLS = range(6)
GNN_OUT = 16


class WarmStartNet:
    """The warm-start network (weights, Adam state) of the library; see a2ls_gnn_* in include/a2ls.h."""

    def __init__(self, seed: int = 0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        g = ctypes.c_void_p()
        _check(lib().a2ls_gnn_create(ctypes.c_uint64(seed), ctypes.c_void_p(int(stream.cuda_stream)),
                                     ctypes.byref(g)))
        self._g = g

    @staticmethod
    def num_params() -> int:
        return int(lib().a2ls_gnn_num_params())

    def close(self):
        if getattr(self, "_g", None):
            lib().a2ls_gnn_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().a2ls_gnn_get_params(self._g, out.ctypes.data, out.size))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().a2ls_gnn_set_params(self._g, p.ctypes.data, p.size))

    def grads(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().a2ls_gnn_get_grads(self._g, out.ctypes.data, out.size))
        return out

    def forward(self, sample: "GnnSample") -> np.ndarray:
        out = np.empty((sample.rows, GNN_OUT), dtype=np.float32)
        _check(lib().a2ls_gnn_forward(self._g, sample._s, out.ctypes.data))
        return out

    def loss_grad(self, sample: "GnnSample") -> float:
        L = ctypes.c_double()
        _check(lib().a2ls_gnn_loss_grad(self._g, sample._s, ctypes.byref(L)))
        return float(L.value)

    def adam_step(self, lr: float):
        _check(lib().a2ls_gnn_adam_step(self._g, float(lr)))

    def launches(self) -> int:
        return int(lib().a2ls_gnn_launches(self._g))


class GnnSample:
    """Local graphs, features and target eigenvectors of a set-up Preconditioner's subdomains."""

    def __init__(self, pre: Preconditioner):
        s = ctypes.c_void_p()
        _check(lib().a2ls_gnn_sample_create(pre._h, ctypes.byref(s)))
        self._s = s
        sz = pre.sizes()
        self.N, self.rows = sz["N"], sz["sum_ni"]

    def close(self):
        if getattr(self, "_s", None):
            lib().a2ls_gnn_sample_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _query(self, what: int, dtype) -> np.ndarray:
        need = ctypes.c_int64()
        _check(lib().a2ls_gnn_sample_query(self._s, what, None, 0, ctypes.byref(need)))
        out = np.empty(int(need.value) // np.dtype(dtype).itemsize, dtype=dtype)
        _check(lib().a2ls_gnn_sample_query(self._s, what, out.ctypes.data, int(need.value), None))
        return out

    def features(self) -> np.ndarray:
        return self._query(GQ_FEATURES, np.float32).reshape(self.rows, 8)[:, :6]

    def graph(self) -> dict:
        return {"rowptr": self._query(GQ_ROWPTR, np.int64), "cols": self._query(GQ_COLS, np.int32),
                "w": self._query(GQ_WEIGHTS, np.float32), "s": self._query(GQ_SWEIGHTS, np.float32)}

    def target_cols(self) -> np.ndarray:
        return self._query(GQ_TARGET_COLS, np.int32)

    def set_target(self, Z: list):
        """Z: one (n_i x m_i) array per subdomain, in the local order of Preconditioner.subdomains()."""
        m = np.array([z.shape[1] for z in Z], dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(z, dtype=np.float64).ravel() for z in Z]))
        _check(lib().a2ls_gnn_sample_set_target(self._s, m.ctypes.data, flat.ctypes.data))


def setup_batch(systems: list, stream=None, **opts) -> list:
    """a2ls_setup_batch over [(rowptr, colind, val, part, overlap, nev)] CUDA tensors; returns Preconditioners."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    nsys = len(systems)
    csrs = (CSR * max(nsys, 1))()
    parts = (ctypes.c_void_p * max(nsys, 1))()
    ov = np.zeros(max(nsys, 1), dtype=np.int32)
    nv = np.zeros(max(nsys, 1), dtype=np.int32)
    for k, (rowptr, colind, val, part, overlap, nev) in enumerate(systems):
        csrs[k] = CSR(int(rowptr.numel() - 1), int(colind.numel()), _ptr(rowptr), _ptr(colind), _ptr(val))
        parts[k] = _ptr(part)
        ov[k], nv[k] = overlap, nev
    o = default_options(**opts)
    o.stream = ctypes.c_void_p(int(stream.cuda_stream))
    out = (ctypes.c_void_p * max(nsys, 1))()
    _check(lib().a2ls_setup_batch(nsys, csrs, parts, ov.ctypes.data, nv.ctypes.data, ctypes.byref(o), out))
    handles = []
    for k in range(nsys):
        P = Preconditioner.__new__(Preconditioner)
        P.n = int(systems[k][0].numel() - 1)
        P.stream, P.options, P._warm = stream, o, opts.get("warm_start")
        P._h = ctypes.c_void_p(out[k])
        P._keep = systems[k]
        handles.append(P)
    return handles
