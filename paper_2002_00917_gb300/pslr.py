"""Thin Python binding of libpslr (include/pslr.h): argument marshalling only.

Every step of the preconditioner and of the solver runs in the library's CUDA
kernels; this module turns torch tensors into device pointers and the current
torch stream into a cudaStream_t.  There is no CPU fallback: when libpslr.so
cannot be loaded, every call raises.

The function names mirror the C ABI (``pslr_setup``, ``pslr_apply``, ...).  The
class :class:`Pslr` owns one context.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpslr.so")

PSLR_OK = 0
PSLR_ERR_ARG = 1
PSLR_ERR_CUDA = 2
PSLR_ERR_ZERO_PIVOT = 3
PSLR_ERR_BREAKDOWN = 4
PSLR_ERR_SINGULAR_IMH = 5
PSLR_ERR_NOT_CONVERGED = 6
PSLR_ERR_NAN = 7
PSLR_ERR_TIMEOUT = 8
PSLR_ERR_STATE = 9
PSLR_ERR_TOO_LARGE = 10
PSLR_FP64 = 0
PSLR_FP32 = 1


class pslr_opts(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("splits", C.c_int32 * 3), ("part", C.c_void_p),
                ("factor", C.c_int32), ("seed", C.c_uint64), ("drop_tol", C.c_double),
                ("setup_threads", C.c_int32), ("nparts", C.c_int32), ("merge_levels", C.c_int32),
                ("device_factor", C.c_int32)]


class pslr_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("s", C.c_int32), ("p", C.c_int32), ("q", C.c_int32),
                ("m", C.c_int32), ("rank", C.c_int32), ("nnz_A", C.c_int64), ("nnz_ilu", C.c_int64),
                ("nnz_lr", C.c_int64), ("fill_ilu", C.c_double), ("fill_lr", C.c_double),
                ("fill_total", C.c_double), ("max_interior", C.c_int32),
                ("max_interface", C.c_int32), ("levels_B", C.c_int32), ("levels_C0", C.c_int32),
                ("apply_bytes_fp64", C.c_int64), ("apply_bytes_fp32", C.c_int64),
                ("layout_hash", C.c_uint64), ("setup_threads", C.c_int32), ("layout_errors", C.c_int64),
                ("grid", C.c_int32 * 2), ("ring", C.c_int32 * 2), ("ctas_per_sm", C.c_int32 * 2),
                ("nnz_fact_B", C.c_int64), ("nnz_fact_C0", C.c_int64), ("nnz_E", C.c_int64),
                ("nnz_F", C.c_int64), ("nnz_Cg", C.c_int64), ("omega", C.c_double),
                ("merged", C.c_int32 * 2), ("unit_sweeps", C.c_int32), ("device_factor", C.c_int32),
                ("factor_ms", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        for k in ("grid", "ring", "ctas_per_sm", "merged"):
            d[k] = list(getattr(self, k))
        return d


class pslr_batch_info(C.Structure):
    _fields_ = [("nsys", C.c_int32), ("nrhs", C.c_int32), ("nprob", C.c_int32), ("n_total", C.c_int64),
                ("items", C.c_int32), ("grid", C.c_int32), ("ring", C.c_int32 * 2),
                ("group", C.c_int32 * 2), ("groups", C.c_int32 * 2), ("max_m", C.c_int32),
                ("max_p", C.c_int32), ("max_q", C.c_int32), ("apply_bytes_fp64", C.c_int64),
                ("apply_bytes_fp32", C.c_int64), ("graph", C.c_int32), ("handoff", C.c_int32),
                ("krylov_chunk", C.c_int32), ("pair_rhs", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        for k in ("ring", "group", "groups"):
            d[k] = list(getattr(self, k))
        return d


class pslr_batch_opts(C.Structure):
    _fields_ = [("group", C.c_int32 * 2), ("ring_max", C.c_int32 * 2), ("krylov_chunk", C.c_int32),
                ("pair_rhs", C.c_int32)]


_P, _I32, _I64, _D, _U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
SIGNATURES = {
    "pslr_setup": (_I32, [_I32, _P, _P, _P, C.POINTER(pslr_opts), _P, C.POINTER(_P)]),
    "pslr_plan": (_I32, [_I32, _P, _P, _P, C.POINTER(pslr_opts), _I32, _I32, C.POINTER(pslr_info),
                         _P, _P, _P]),
    "pslr_build_lowrank": (_I32, [_P, _I32, _I32, _I32, _P]),
    "pslr_set_lowrank": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "pslr_set_neumann": (_I32, [_P, _I32, _D, _P]),
    "pslr_apply": (_I32, [_P, _P, _P, _I32, _I32, _P]),
    "pslr_apply_T": (_I32, [_P, _P, _P, _I32, _I32, _P]),
    "pslr_apply_host": (_I32, [_P, _P, _P, _I32, _I32, _I32, _P]),
    "pslr_apply_noalloc": (_I32, [_P, _P, _P, _I32, _I32, _P]),
    "pslr_solve": (_I32, [_P, _P, _P, _D, _I32, _I32, _I32, _I32, C.POINTER(_I32),
                          C.POINTER(_D), _P]),
    "pslr_matvec": (_I32, [_P, _P, _P, _I32, _P]),
    "pslr_grad_values": (_I32, [_P, _P, _P, _P, _P]),
    "pslr_get_maps": (_I32, [_P, _P, _P, _P]),
    "pslr_ilu0_device": (_I32, [_I32, _I32, _P, _P, _P, _P, _P]),
    "pslr_get_lowrank": (_I32, [_P, _P, _P, _P]),
    "pslr_get_info": (_I32, [_P, C.POINTER(pslr_info)]),
    "pslr_sync": (_I32, [_P, _P]),
    "pslr_set_wait_limit": (_I64, [_P, _I64]),
    "pslr_last_error": (C.c_char_p, [_P]),
    "pslr_status_string": (C.c_char_p, [_I32]),
    "pslr_destroy": (None, [_P]),
    "pslr_batch_create": (_I32, [_I32, _P, _I32, _I32, C.POINTER(_P)]),
    "pslr_batch_create_opts": (_I32, [_I32, _P, _I32, _P, C.POINTER(_P)]),
    "pslr_batch_apply": (_I32, [_P, _P, _P, _I32, _P]),
    "pslr_batch_solve": (_I32, [_P, _P, _P, _D, _I32, _I32, _I32, _P, _P, _P]),
    "pslr_batch_get_info": (_I32, [_P, C.POINTER(pslr_batch_info)]),
    "pslr_batch_sync": (_I32, [_P, _P]),
    "pslr_batch_set_wait_limit": (_I64, [_P, _I64]),
    "pslr_batch_last_error": (C.c_char_p, [_P]),
    "pslr_batch_destroy": (None, [_P]),
}

_lib = None


def load():
    """Load libpslr.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2002_00917_gb300.build.build() "
                               "(the PSLR path has no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class PslrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Pslr:
    """One PSLR context on the current CUDA device.

    ``A`` is host CSR (``rowptr``, ``col``, ``val`` numpy arrays, or any object
    with those attributes and ``n``).  ``dims``/``splits`` select the geometric
    split; ``part`` (length n) overrides it.  ``factor``: 0 ILU(0), 1 exact LU,
    2 ILUT(``drop_tol``).  ``setup_threads``: host threads of the set-up (0 =
    all hardware threads); the context is the same for every value.
    ``nparts`` > 0 with ``dims`` all zero and no ``part``: the library's graph
    partition (recursive breadth-first bisection) into that many subdomains.
    ``merge_levels``: sweep segment layout, 0 automatic, 1 one level per
    segment, 2 several levels per segment (same result, bit for bit).
    ``device_factor``: compute the ILU(0) local factors (``factor`` 0) on
    the GPU instead of on the host.
    """

    def __init__(self, A, dims=(0, 0, 0), splits=(1, 1, 1), part=None, factor=0, seed=0,
                 stream=None, drop_tol=0.0, setup_threads=0, nparts=0, merge_levels=0, device_factor=False):
        lib = load()
        self.lib = lib
        self.n = int(A.n)
        self._rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
        self._ci = np.ascontiguousarray(A.col, dtype=np.int32)
        self._av = np.ascontiguousarray(A.val, dtype=np.float64)
        o = pslr_opts()
        for d in range(3):
            o.dims[d] = int(dims[d])
            o.splits[d] = int(splits[d])
        self._part = None if part is None else np.ascontiguousarray(part, dtype=np.int32)
        o.part = None if self._part is None else self._part.ctypes.data
        o.factor = int(factor)
        o.seed = int(seed)
        o.drop_tol = float(drop_tol)
        o.setup_threads = int(setup_threads)
        o.nparts = int(nparts)
        o.merge_levels = int(merge_levels)
        o.device_factor = int(bool(device_factor))
        self.factor, self.drop_tol = int(factor), float(drop_tol)
        h = C.c_void_p()
        st = lib.pslr_setup(self.n, self._rp.ctypes.data, self._ci.ctypes.data, self._av.ctypes.data,
                            C.byref(o), _stream(stream), C.byref(h))
        if st != PSLR_OK:
            raise PslrError(st, f"pslr_setup: {lib.pslr_status_string(st).decode()}")
        self.h = h
        self.info = self.get_info()

    def close(self):
        if getattr(self, "h", None):
            self.lib.pslr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what, ok=(PSLR_OK,)):
        if st not in ok:
            msg = self.lib.pslr_last_error(self.h).decode()
            raise PslrError(st, f"{what}: {msg}")
        return st

    # -- set-up products
    def get_info(self):
        info = pslr_info()
        self._check(self.lib.pslr_get_info(self.h, C.byref(info)), "pslr_get_info")
        return info.as_dict()

    def get_maps(self):
        part = np.empty(self.n, np.int32)
        iface = np.empty(self.n, np.int32)
        perm = np.empty(self.n, np.int32)
        self._check(self.lib.pslr_get_maps(self.h, part.ctypes.data, iface.ctypes.data,
                                           perm.ctypes.data), "pslr_get_maps")
        return part, iface, perm

    # -- low-rank term (Algorithm 1, steps 6-8)
    def build_lowrank(self, m, rank, full_rank=False, stream=None):
        st = self.lib.pslr_build_lowrank(self.h, int(m), int(rank), int(bool(full_rank)),
                                         _stream(stream))
        self._check(st, "pslr_build_lowrank", ok=(PSLR_OK, PSLR_ERR_BREAKDOWN))
        self.info = self.get_info()
        return self.info["rank"], st

    def set_lowrank(self, m, V=None, G=None, stream=None):
        r = 0 if V is None else V.shape[1]
        Vc = np.asfortranarray(V, dtype=np.float64) if r else None
        Gc = np.asfortranarray(G, dtype=np.float64) if r else None
        st = self.lib.pslr_set_lowrank(self.h, int(m), r, None if Vc is None else Vc.ctypes.data,
                                       None if Gc is None else Gc.ctypes.data, _stream(stream))
        self._check(st, "pslr_set_lowrank")
        self.info = self.get_info()

    def set_neumann(self, m, omega, stream=None):
        """Apply the classical Neumann polynomial of Sec. 1 (scaling omega, m+1
        terms, no low-rank term) instead of PSLR; build_lowrank/set_lowrank
        return to PSLR."""
        self._check(self.lib.pslr_set_neumann(self.h, int(m), float(omega), _stream(stream)), "pslr_set_neumann")
        self.info = self.get_info()

    def get_lowrank(self):
        q, r = self.info["q"], self.info["rank"]
        V = np.zeros((q, r), order="F")
        H = np.zeros((r, r), order="F")
        G = np.zeros((r, r), order="F")
        self._check(self.lib.pslr_get_lowrank(self.h, V.ctypes.data if r else None,
                                              H.ctypes.data if r else None,
                                              G.ctypes.data if r else None), "pslr_get_lowrank")
        return V, H, G

    # -- checkpoint of the low-rank term
    def fingerprint(self):
        """Hex digest of what the low-rank term depends on: the matrix, the
        local factor kind and threshold, and the reordering (Section 2)."""
        h = hashlib.sha256()
        for a in (self._rp, self._ci, self._av, *self.get_maps()):
            h.update(np.ascontiguousarray(a).tobytes())
        h.update(np.array([self.factor], np.int64).tobytes())
        h.update(np.array([self.drop_tol], np.float64).tobytes())
        return h.hexdigest()

    def save_lowrank(self, path):
        """Write the low-rank term (m, V, H, G of Algorithm 1, steps 6-8) with
        this context's fingerprint to ``path`` (numpy .npz).  The local factors
        are not saved: setting up the same matrix with the same options
        rebuilds them bit for bit, so only the Arnoldi work is kept."""
        V, H, G = self.get_lowrank()
        np.savez(path, m=np.int64(self.info["m"]), V=V, H=H, G=G, fingerprint=np.array(self.fingerprint()))

    def load_lowrank(self, path, stream=None):
        """Install a term written by :meth:`save_lowrank` for the same matrix,
        factor kind and reordering (ValueError otherwise); returns its rank."""
        with np.load(path) as f:
            if str(f["fingerprint"]) != self.fingerprint():
                raise ValueError(f"{path}: low-rank term of another matrix, factor kind or reordering")
            m, V, G = int(f["m"]), f["V"], f["G"]
        self.set_lowrank(m, V if V.shape[1] else None, G if V.shape[1] else None, stream=stream)
        return V.shape[1]

    # -- Algorithm 3 and its transpose
    def apply(self, b, z, transpose=False, stream=None):
        """z = M^{-1} b (or M^{-T} b) on device tensors, float64 or float32,
        shape (n,) or (n, nrhs) column-major."""
        prec = PSLR_FP64 if b.dtype.itemsize == 8 else PSLR_FP32
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        if b.dim() == 2 and nrhs > 1 and b.stride(0) != 1:
            raise ValueError("multi-rhs tensors must be column-major (stride(0) == 1)")
        f = self.lib.pslr_apply_T if transpose else self.lib.pslr_apply
        return self._check(f(self.h, _ptr(b), _ptr(z), nrhs, prec, _stream(stream)), "pslr_apply")

    def apply_host(self, b, z, transpose=False, stream=None):
        """End-to-end apply on host numpy arrays (copies in, applies, copies out)."""
        prec = PSLR_FP64 if b.dtype.itemsize == 8 else PSLR_FP32
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        return self._check(self.lib.pslr_apply_host(self.h, C.c_void_p(b.ctypes.data),
                                                    C.c_void_p(z.ctypes.data), nrhs, prec,
                                                    int(bool(transpose)), _stream(stream)),
                           "pslr_apply_host")

    def solve(self, b, x, rtol=1e-8, restart=40, maxit=500, prec=PSLR_FP64, transpose=False,
              stream=None, check=True):
        its = C.c_int32(0)
        rel = C.c_double(0.0)
        st = self.lib.pslr_solve(self.h, _ptr(b), _ptr(x), float(rtol), int(restart), int(maxit),
                                 int(prec), int(bool(transpose)), C.byref(its), C.byref(rel),
                                 _stream(stream))
        if check:
            self._check(st, "pslr_solve", ok=(PSLR_OK, PSLR_ERR_NOT_CONVERGED))
        return its.value, rel.value, st

    def grad_values(self, lam, u, grad, stream=None):
        """grad[k] = -lam[row_k] * u[col_k] over the stored entries of A."""
        return self._check(self.lib.pslr_grad_values(self.h, _ptr(lam), _ptr(u), _ptr(grad),
                                                     _stream(stream)), "pslr_grad_values")

    def matvec(self, x, y, transpose=False, stream=None):
        return self._check(self.lib.pslr_matvec(self.h, _ptr(x), _ptr(y), int(bool(transpose)),
                                                _stream(stream)), "pslr_matvec")

    def sync(self, stream=None, check=True):
        st = self.lib.pslr_sync(self.h, _stream(stream))
        if check:
            self._check(st, "pslr_sync")
        return st

    def set_wait_limit(self, polls):
        return self.lib.pslr_set_wait_limit(self.h, int(polls))


class Batch:
    """Many set-up contexts (:class:`Pslr`, low-rank term built) applied and
    solved together, ``nrhs`` right-hand sides each (pslr_batch_*).

    Batched vectors are 1-D device tensors of ``info["n_total"]`` elements:
    the systems in order, each an n_k x nrhs column-major block;
    :meth:`offsets` gives the blocks' starts.  The contexts must outlive the
    batch; the batch keeps references to them.  ``group``: subdomains of one
    system a CTA sweeps in lockstep (0: the largest that fits; an int, or a
    pair (FP64, FP32)); ``ring_max``
    (FP64, FP32) caps the apply's ring slots (0: as many as fit);
    ``krylov_chunk``: rows per chunk of the batched FGMRES kernels (0: 1024);
    ``pair_rhs``: in the FP64 apply with several right-hand sides, one thread
    per (row, rhs) pair (1) or per row (0).  None changes a result; see
    :func:`paper_2002_00917_gb300.autotune.tune_batch`."""

    def __init__(self, systems, nrhs, group=0, ring_max=(0, 0), krylov_chunk=0, pair_rhs=1):
        lib = load()
        self.lib = lib
        self.systems = list(systems)
        self.nrhs = int(nrhs)
        arr = (C.c_void_p * len(self.systems))(*[p.h for p in self.systems])
        o = pslr_batch_opts()
        g = (group, group) if isinstance(group, int) else tuple(group)
        o.group[0], o.group[1] = int(g[0]), int(g[1])
        o.ring_max[0], o.ring_max[1] = int(ring_max[0]), int(ring_max[1])
        o.krylov_chunk = int(krylov_chunk)
        o.pair_rhs = int(pair_rhs)
        h = C.c_void_p()
        st = lib.pslr_batch_create_opts(len(self.systems), arr, self.nrhs, C.byref(o), C.byref(h))
        if st != PSLR_OK:
            raise PslrError(st, f"pslr_batch_create: {lib.pslr_batch_last_error(None).decode()}")
        self.h = h
        self.info = self.get_info()

    def close(self):
        if getattr(self, "h", None):
            self.lib.pslr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what, ok=(PSLR_OK,)):
        if st not in ok:
            msg = self.lib.pslr_batch_last_error(self.h).decode()
            raise PslrError(st, f"{what}: {msg}")
        return st

    def get_info(self):
        info = pslr_batch_info()
        self._check(self.lib.pslr_batch_get_info(self.h, C.byref(info)), "pslr_batch_get_info")
        return info.as_dict()

    def offsets(self):
        """Start of each system's n_k x nrhs block in a batched vector."""
        out, o = [], 0
        for p in self.systems:
            out.append(o)
            o += p.n * self.nrhs
        return out

    def apply(self, b, z, stream=None):
        """z = M_k^{-1} b for every system and right-hand side, one launch;
        float64 (FP64 form) or float32 (FP32 form, BF16 V) batched vectors."""
        prec = PSLR_FP64 if b.dtype.itemsize == 8 else PSLR_FP32
        return self._check(self.lib.pslr_batch_apply(self.h, _ptr(b), _ptr(z), prec, _stream(stream)),
                           "pslr_batch_apply")

    def solve(self, b, x, rtol=1e-8, restart=40, maxit=500, prec=PSLR_FP64, stream=None, check=True):
        """Batched FGMRES; returns (iters, relres, status), per problem
        ((system, rhs) pairs in system-major order)."""
        P = self.info["nprob"]
        its = np.zeros(P, np.int32)
        rel = np.zeros(P, np.float64)
        st = self.lib.pslr_batch_solve(self.h, _ptr(b), _ptr(x), float(rtol), int(restart), int(maxit),
                                       int(prec), its.ctypes.data, rel.ctypes.data, _stream(stream))
        if check:
            self._check(st, "pslr_batch_solve", ok=(PSLR_OK, PSLR_ERR_NOT_CONVERGED))
        self.info = self.get_info()
        return its, rel, st

    def sync(self, stream=None, check=True):
        st = self.lib.pslr_batch_sync(self.h, _stream(stream))
        if check:
            self._check(st, "pslr_batch_sync")
        return st

    def set_wait_limit(self, polls):
        return self.lib.pslr_batch_set_wait_limit(self.h, int(polls))


def _opts(dims, splits, part, factor, seed, drop_tol=0.0, setup_threads=0, nparts=0, merge_levels=0,
          device_factor=0):
    o = pslr_opts()
    for d in range(3):
        o.dims[d] = int(dims[d])
        o.splits[d] = int(splits[d])
    o.part = None if part is None else part.ctypes.data
    o.factor = int(factor)
    o.seed = int(seed)
    o.drop_tol = float(drop_tol)
    o.setup_threads = int(setup_threads)
    o.nparts = int(nparts)
    o.merge_levels = int(merge_levels)
    o.device_factor = int(device_factor)
    return o


def plan(A, dims=(0, 0, 0), splits=(1, 1, 1), part=None, factor=0, m=0, rank=0, drop_tol=0.0, setup_threads=0,
         nparts=0, merge_levels=0, device_factor=0):
    """Host-only dry run of the set-up (no GPU needed): returns (info dict,
    part, is_interface, perm) exactly as a device context would report them."""
    lib = load()
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    av = np.ascontiguousarray(A.val, dtype=np.float64)
    pa = None if part is None else np.ascontiguousarray(part, dtype=np.int32)
    o = _opts(dims, splits, pa, factor, 0, drop_tol, setup_threads, nparts, merge_levels, device_factor)
    info = pslr_info()
    n = int(A.n)
    mp = [np.empty(n, np.int32) for _ in range(3)]
    st = lib.pslr_plan(n, rp.ctypes.data, ci.ctypes.data, av.ctypes.data, C.byref(o), int(m), int(rank),
                       C.byref(info), *[a.ctypes.data for a in mp])
    if st != PSLR_OK:
        raise PslrError(st, f"pslr_plan: {lib.pslr_status_string(st).decode()}")
    return (info.as_dict(), *mp)


def from_workload(w, seed=0, stream=None, merge_levels=0, device_factor=False):
    """Context for a workload dict of ``pslr_inputs.configs``."""
    return Pslr(w["A"], dims=w.get("dims", (0, 0, 0)), splits=w.get("splits", (1, 1, 1)), factor=w["factor"],
                seed=seed, stream=stream, drop_tol=w.get("drop_tol", 0.0), nparts=w.get("nparts", 0),
                merge_levels=merge_levels, device_factor=device_factor)


def ilu0_device(block_ptr, rowptr, col, val, stream=None):
    """ILU(0) on the device of the block-diagonal CSR matrix (``block_ptr``
    the first row of each diagonal block, plus n; ``rowptr``/``col`` the
    host pattern); ``val`` is a CUDA float64 tensor, factored in place (L
    strictly lower with unit diagonal, U the rest).  See pslr_ilu0_device."""
    lib = load()
    bp = np.ascontiguousarray(block_ptr, dtype=np.int32)
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    n = len(rp) - 1
    import torch
    if val.dtype != torch.float64 or not val.is_cuda or not val.is_contiguous() or val.numel() != int(rp[-1]):
        raise ValueError("val must be a contiguous CUDA float64 tensor with rowptr[-1] entries")
    st = lib.pslr_ilu0_device(n, len(bp) - 1, bp.ctypes.data, rp.ctypes.data, ci.ctypes.data, _ptr(val),
                              _stream(stream))
    if st != PSLR_OK:
        raise PslrError(st, f"pslr_ilu0_device: {lib.pslr_status_string(st).decode()}")
    return val
