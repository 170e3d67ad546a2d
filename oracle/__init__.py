"""FP64 CPU oracle for the PSLR preconditioner (arXiv 2002.00917).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2002_00917_gb300``) never imports it and has no CPU fallback.

The arithmetic lives in ``pslr_oracle.c`` (plain C, single-threaded, FP64);
this module compiles it with gcc on first use and wraps it with ctypes.
Vectors are numpy float64 arrays.  ``apply``/``apply_T``/``fgmres`` take and
return vectors in the original ordering; the block operators
(``solve_B``, ``Es``, ``series``, ``Err``...) work in the reordered numbering
(interior 0..p-1, interface 0..q-1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pslr_oracle.c")
_HDR = os.path.join(_HERE, "pslr_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_ZERO_PIVOT, ERR_BREAKDOWN, ERR_SINGULAR_IMH, ERR_NOT_CONVERGED = 0, 1, 3, 4, 5, 6
BLOCKS = {"B": 0, "E": 1, "F": 2, "C": 3, "C0": 4, "Cg": 5, "LU_B": 6, "LU_C0": 7}


def build(force=False):
    """Compile liboracle.so next to its source (gcc, -O2, no host-specific flags)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, I32, D, U64 = C.c_void_p, C.c_int32, C.c_double, C.c_uint64
            sig = {
                "orc_setup": (P, [I32, P, P, P, P, P, P, I32, D, P]),
                "orc_destroy": (None, [P]),
                "orc_sizes": (None, [P, P, P, P, P]),
                "orc_maps": (None, [P, P, P, P]),
                "orc_offsets": (None, [P, P, P]),
                "orc_block_nnz": (I32, [P, I32]),
                "orc_get_block": (None, [P, I32, P, P, P]),
                "orc_solve_B": (None, [P, P, P]),
                "orc_solve_BT": (None, [P, P, P]),
                "orc_solve_C0": (None, [P, P, P]),
                "orc_solve_C0T": (None, [P, P, P]),
                "orc_Es": (None, [P, P, P]),
                "orc_EsT": (None, [P, P, P]),
                "orc_series": (None, [P, I32, P, P]),
                "orc_seriesT": (None, [P, I32, P, P]),
                "orc_Err": (None, [P, I32, P, P]),
                "orc_build_lowrank": (I32, [P, I32, I32, U64, I32, P]),
                "orc_get_lowrank": (None, [P, P, P, P]),
                "orc_set_lowrank": (I32, [P, I32, I32, P, P]),
                "orc_apply": (None, [P, P, P]),
                "orc_apply_T": (None, [P, P, P]),
                "orc_fgmres": (I32, [P, I32, P, P, D, I32, I32, P, P]),
                "orc_splitmix_uniform": (D, [U64, U64]),
                "orc_neumann_series": (None, [P, I32, D, I32, P, P]),
                "orc_neumann_apply": (None, [P, I32, D, I32, P, P]),
                "orc_set_neumann": (None, [P, I32, D]),
                "orc_graph_partition": (I32, [I32, P, P, I32, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


class Oracle:
    """One PSLR set-up (reordering + blocks + local factors) on the CPU."""

    def __init__(self, A, dims=None, splits=None, part=None, factor=0, drop_tol=0.0):
        lib = _load()
        self._lib = lib
        self.A = A
        st = C.c_int32(0)
        d = np.ascontiguousarray(dims if dims is not None else (0, 0, 0), dtype=np.int32)
        s = np.ascontiguousarray(splits if splits is not None else (0, 0, 0), dtype=np.int32)
        pa = None if part is None else np.ascontiguousarray(part, dtype=np.int32)
        self._keep = (A.rowptr, A.col, A.val, d, s, pa)
        h = lib.orc_setup(A.n, _p(A.rowptr), _p(A.col), _p(A.val), _p(d), _p(s), _p(pa), factor,
                          float(drop_tol), C.byref(st))
        if not h:
            raise OracleError(st.value, "orc_setup")
        self.h = C.c_void_p(h)
        n, ns, p, q = (C.c_int32() for _ in range(4))
        lib.orc_sizes(self.h, C.byref(n), C.byref(ns), C.byref(p), C.byref(q))
        self.n, self.s, self.p, self.q = n.value, ns.value, p.value, q.value
        self.m, self.r = 0, 0

    def __del__(self):
        if getattr(self, "h", None) and self._lib is not None:
            self._lib.orc_destroy(self.h)
            self.h = None

    # -- reordering (Section 2)
    def maps(self):
        part = np.empty(self.n, np.int32)
        iface = np.empty(self.n, np.int32)
        perm = np.empty(self.n, np.int32)
        self._lib.orc_maps(self.h, _p(part), _p(iface), _p(perm))
        return part, iface, perm

    def offsets(self):
        io = np.empty(self.s + 1, np.int32)
        go = np.empty(self.s + 1, np.int32)
        self._lib.orc_offsets(self.h, _p(io), _p(go))
        return io, go

    def block_nnz(self, name):
        """Stored entries of a block (-1 if not stored for this factor kind)."""
        return int(self._lib.orc_block_nnz(self.h, BLOCKS[name]))

    def block(self, name):
        """(rowptr, col, val, shape) of a block in the reordered numbering."""
        w = BLOCKS[name]
        nnz = self._lib.orc_block_nnz(self.h, w)
        if nnz < 0:
            raise ValueError(f"block {name} not stored for this factor kind")
        nr = {"B": self.p, "E": self.p, "F": self.q, "C": self.q, "C0": self.q, "Cg": self.q,
              "LU_B": self.p, "LU_C0": self.q}[name]
        nc = {"B": self.p, "E": self.q, "F": self.p, "C": self.q, "C0": self.q, "Cg": self.q,
              "LU_B": self.p, "LU_C0": self.q}[name]
        rp = np.empty(nr + 1, np.int32)
        ci = np.empty(max(nnz, 1), np.int32)
        v = np.empty(max(nnz, 1), np.float64)
        self._lib.orc_get_block(self.h, w, _p(rp), _p(ci), _p(v))
        return rp, ci[:nnz], v[:nnz], (nr, nc)

    def dense_block(self, name):
        rp, ci, v, (nr, nc) = self.block(name)
        D = np.zeros((nr, nc))
        rows = np.repeat(np.arange(nr), np.diff(rp))
        D[rows, ci] = v
        return D

    # -- operators (reordered numbering)
    def _unary(self, fn, x, nout, *extra):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty(max(nout, 1), np.float64)
        fn(self.h, *extra, _p(x), _p(out))
        return out[:nout]

    def solve_B(self, x):
        return self._unary(self._lib.orc_solve_B, x, self.p)

    def solve_BT(self, x):
        return self._unary(self._lib.orc_solve_BT, x, self.p)

    def solve_C0(self, x):
        return self._unary(self._lib.orc_solve_C0, x, self.q)

    def solve_C0T(self, x):
        return self._unary(self._lib.orc_solve_C0T, x, self.q)

    def Es(self, x):
        return self._unary(self._lib.orc_Es, x, self.q)

    def EsT(self, x):
        return self._unary(self._lib.orc_EsT, x, self.q)

    def series(self, m, x):
        return self._unary(self._lib.orc_series, x, self.q, m)

    def seriesT(self, m, x):
        return self._unary(self._lib.orc_seriesT, x, self.q, m)

    def Err(self, m, x):
        return self._unary(self._lib.orc_Err, x, self.q, m)

    # -- low rank (Algorithm 1, steps 6-8)
    def build_lowrank(self, m, rank, seed=0, full_rank=False):
        kept = C.c_int32(0)
        st = self._lib.orc_build_lowrank(self.h, m, rank, seed, int(bool(full_rank)), C.byref(kept))
        if st not in (OK, ERR_BREAKDOWN):
            raise OracleError(st, "orc_build_lowrank")
        self.m, self.r = m, kept.value
        return kept.value, st

    def lowrank(self):
        r, q = self.r, self.q
        if r == 0:
            return np.zeros((q, 0)), np.zeros((0, 0)), np.zeros((0, 0))
        V = np.empty(q * r)
        H = np.empty(r * r)
        G = np.empty(r * r)
        self._lib.orc_get_lowrank(self.h, _p(V), _p(H), _p(G))
        return V.reshape(r, q).T.copy(), H.reshape(r, r).T.copy(), G.reshape(r, r).T.copy()

    def set_lowrank(self, m, V, G):
        r = 0 if V is None else V.shape[1]
        Vc = np.ascontiguousarray(V.T, dtype=np.float64) if r else None
        Gc = np.ascontiguousarray(G.T, dtype=np.float64) if r else None
        self._lib.orc_set_lowrank(self.h, m, r, _p(Vc), _p(Gc))
        self.m, self.r = m, r

    # -- Algorithm 3
    def apply(self, b):
        return self._unary(self._lib.orc_apply, b, self.n)

    def apply_T(self, b):
        return self._unary(self._lib.orc_apply_T, b, self.n)

    def neumann_series(self, m, omega, t, transpose=False):
        """Sec. 1 Neumann polynomial of the Schur complement applied to t
        (interface numbering)."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        out = np.empty(self.q + 1)
        self._lib.orc_neumann_series(self.h, int(m), float(omega), int(bool(transpose)), _p(t), _p(out))
        return out[: self.q]

    def neumann_apply(self, m, omega, b, transpose=False):
        """Algorithm 3's block elimination with the Neumann polynomial in place
        of the PSLR Schur approximation (original ordering)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        z = np.empty(self.n)
        self._lib.orc_neumann_apply(self.h, int(m), float(omega), int(bool(transpose)), _p(b), _p(z))
        return z

    def set_neumann(self, m, omega):
        """FGMRES preconditioned by the Neumann polynomial (omega > 0), or by
        PSLR again (omega <= 0)."""
        self._lib.orc_set_neumann(self.h, int(m), float(omega))

    def fgmres(self, b, rtol=1e-8, restart=40, maxit=500, precond=True, transpose=False):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(self.n)
        its = C.c_int32(0)
        rel = C.c_double(0.0)
        flags = (1 if precond else 0) | (2 if transpose else 0)
        st = self._lib.orc_fgmres(self.h, flags, _p(b), _p(x), rtol, restart, maxit, C.byref(its),
                                  C.byref(rel))
        return x, its.value, rel.value, st


def splitmix_uniform(seed, j):
    return _load().orc_splitmix_uniform(seed, j)


def graph_partition(A, nparts):
    """Recursive breadth-first bisection of the graph of A + A^T into
    ``nparts`` parts (the oracle's own implementation)."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    part = np.empty(A.n, dtype=np.int32)
    st = _load().orc_graph_partition(A.n, _p(rp), _p(ci), int(nparts), _p(part))
    if st != OK:
        raise OracleError(st, "orc_graph_partition")
    return part


def from_workload(w):
    """Oracle set-up for a workload dict from ``pslr_inputs.configs``; a
    workload with ``nparts`` is partitioned by :func:`graph_partition`."""
    if w.get("nparts"):
        return Oracle(w["A"], part=graph_partition(w["A"], w["nparts"]), factor=w["factor"],
                      drop_tol=w.get("drop_tol", 0.0))
    return Oracle(w["A"], dims=w["dims"], splits=w["splits"], factor=w["factor"], drop_tol=w.get("drop_tol", 0.0))
