"""Python binding of the GB300 structured-matrix-approximation library.

Argument marshalling only: every step of the path runs in the CUDA kernels of
libsma.so (see include/sma.h).  The binding exposes the C ABI under the same
names (sma_create, sma_compress, sma_get_result, sma_get_ranks,
sma_reconstruct, sma_apply, sma_export, sma_destroy) and a small ``Handle``
convenience wrapper.  There is no fallback: importing works without a GPU,
but every call that needs the library raises if libsma.so is missing, and the
library itself returns an error status without a CUDA device.

Arrays are column-major, as in the C ABI.  A torch tensor passed as a matrix
must have strides (1, ld) (``colmajor(t)`` makes one); numpy arrays are
treated as host memory and must be Fortran-ordered.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsma.so")

# enums (include/sma.h)
SMA_OK, SMA_ERR_ARG, SMA_ERR_STRUCT, SMA_ERR_CUDA, SMA_ERR_ALLOC = 0, 1, 2, 3, 4
SMA_ERR_NOCONVERGE, SMA_ERR_TIMEOUT, SMA_ERR_NONFINITE, SMA_ERR_STATE, SMA_ERR_UNSUPPORTED = 5, 6, 7, 8, 9
SMA_ERR_NOT_SPD = 10
SMA_FP64, SMA_MIXED = 0, 1
SMA_TSVDM, SMA_TUCKER_BLOCKMODE, SMA_TUCKER_SHARED_U, SMA_TUCKER_ROWCOL, SMA_HOSVD_MULTILEVEL = 0, 1, 2, 3, 4
SMA_TUCKER_SPD = 5
SMA_CP_ALS = 6
SMA_M_DCT2, SMA_M_IDENTITY, SMA_M_USER = 0, 1, 2
SMA_INPUT_DENSE, SMA_INPUT_BLOCKS = 0, 1
SMA_PRECOND_AUTO, SMA_PRECOND_NONE, SMA_PRECOND_QRCP, SMA_PRECOND_QRCP2 = 0, 1, 2, 3
EXPORT_X, EXPORT_XHAT, EXPORT_SIGMA, EXPORT_T, EXPORT_FACTOR, EXPORT_CHOL = 0, 1, 2, 3, 4, 5
EXPORT_CP_X, EXPORT_CP_Z = 6, 7

EXPORTED = ("sma_create", "sma_compress", "sma_get_result", "sma_get_ranks", "sma_reconstruct",
            "sma_apply", "sma_export", "sma_profile", "sma_slice_svd_noalloc", "sma_destroy",
            "sma_status_string", "sma_version")
STAGES = ("gather", "transform", "svd", "truncate", "factors", "report", "apply", "precond")


class sma_problem(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int32), ("q", ctypes.c_int32), ("m", ctypes.c_int32),
                ("n", ctypes.c_int32), ("p", ctypes.c_int32),
                ("block_map", ctypes.POINTER(ctypes.c_int32)),
                ("levels", ctypes.c_int32),
                ("level_ell", ctypes.POINTER(ctypes.c_int32)),
                ("level_q", ctypes.POINTER(ctypes.c_int32)),
                ("level_p", ctypes.POINTER(ctypes.c_int32)),
                ("level_maps", ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)))]


class sma_options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("decomp", ctypes.c_int), ("mkind", ctypes.c_int),
                ("layout", ctypes.c_int), ("M_user", ctypes.POINTER(ctypes.c_double)),
                ("fixed_rank", ctypes.c_int32), ("rel_tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("profile", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("precondition", ctypes.c_int), ("autotune", ctypes.c_int32),
                ("sketch_cols", ctypes.c_int32),
                ("sketch_omega", ctypes.POINTER(ctypes.c_double)),
                ("sketch_psi", ctypes.POINTER(ctypes.c_double)),
                ("cp_iters", ctypes.c_int32),
                ("cp_init_x", ctypes.POINTER(ctypes.c_double)),
                ("cp_init_z", ctypes.POINTER(ctypes.c_double))]


class sma_result(ctypes.Structure):
    _fields_ = [("total_rank", ctypes.c_int32), ("n_kron_terms", ctypes.c_int32),
                ("ranks", ctypes.c_int32 * 4), ("sweeps_max", ctypes.c_int32),
                ("device_status", ctypes.c_int32), ("norm", ctypes.c_double),
                ("tensor_err", ctypes.c_double), ("rel_err", ctypes.c_double),
                ("orth_defect", ctypes.c_double), ("trace_relerr", ctypes.c_double),
                ("storage_ratio", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: (list(getattr(self, k)) if k == "ranks" else getattr(self, k))
                for k, _ in self._fields_}


class SmaError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {sma_status_string(status)} (status {status})")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsma.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "or python -m paper_2105_01170_gb300._build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.sma_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(sma_problem), i32,
                                 ctypes.POINTER(sma_options)]
        L.sma_compress.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                   ctypes.POINTER(sma_result)]
        L.sma_get_result.argtypes = [vp, i32, ctypes.POINTER(sma_result)]
        L.sma_get_ranks.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.sma_reconstruct.argtypes = [vp, i32, vp, i64]
        L.sma_apply.argtypes = [vp, i32, vp, i64, vp, i64, i32]
        L.sma_export.argtypes = [vp, i32, i32, vp, i64, ctypes.POINTER(i64)]
        L.sma_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                  ctypes.POINTER(i64), i32]
        L.sma_slice_svd_noalloc.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp, i32, vp]
        L.sma_destroy.argtypes = [vp]
        L.sma_status_string.argtypes = [ctypes.c_int]
        L.sma_status_string.restype = ctypes.c_char_p
        L.sma_version.restype = ctypes.c_char_p
        for name in ("sma_create", "sma_compress", "sma_get_result", "sma_get_ranks",
                     "sma_reconstruct", "sma_apply", "sma_export", "sma_profile",
                     "sma_slice_svd_noalloc", "sma_destroy"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int, where: str) -> int:
    if status != SMA_OK:
        raise SmaError(status, where)
    return status


# ---- the C ABI under its own names ------------------------------------------

def sma_status_string(status: int) -> str:
    return lib().sma_status_string(int(status)).decode()


def sma_version() -> str:
    return lib().sma_version().decode()


def sma_create(problems, options: sma_options):
    arr = (sma_problem * len(problems))(*problems)
    h = ctypes.c_void_p()
    st = lib().sma_create(ctypes.byref(h), arr, len(problems), ctypes.byref(options))
    return st, h


def sma_compress(h, ptrs, ldas, results=None):
    n = len(ptrs)
    P = (ctypes.c_void_p * n)(*[ctypes.c_void_p(int(x)) for x in ptrs])
    L = (ctypes.c_int64 * n)(*[int(x) for x in ldas])
    return lib().sma_compress(h, P, L, results)


def sma_get_result(h, i, res: sma_result):
    return lib().sma_get_result(h, int(i), ctypes.byref(res))


def sma_get_ranks(h, i, out, count):
    return lib().sma_get_ranks(h, int(i), out, ctypes.byref(count))


def sma_reconstruct(h, i, ptr, ld):
    return lib().sma_reconstruct(h, int(i), ctypes.c_void_p(int(ptr)), int(ld))


def sma_apply(h, i, xptr, ldx, yptr, ldy, nrhs):
    return lib().sma_apply(h, int(i), ctypes.c_void_p(int(xptr)), int(ldx),
                           ctypes.c_void_p(int(yptr)), int(ldy), int(nrhs))


def sma_export(h, i, which, ptr, count, avail):
    return lib().sma_export(h, int(i), int(which), ctypes.c_void_p(int(ptr)), int(count),
                            ctypes.byref(avail))


def sma_profile(h, ms, calls, launches, reset):
    return lib().sma_profile(h, ms, calls, ctypes.byref(launches), int(reset))


def sma_slice_svd_noalloc(x_ptr, m, n, p, w_ptr, v_ptr, sigma_ptr, sweeps_ptr, status_ptr,
                          max_sweeps=0, stream=None):
    """Allocation-free batched slice SVD (device pointers; see include/sma.h)."""
    c = ctypes.c_void_p
    return lib().sma_slice_svd_noalloc(c(int(x_ptr)), int(m), int(n), int(p), c(int(w_ptr)),
                                       c(int(v_ptr)), c(int(sigma_ptr)), c(int(sweeps_ptr or 0)),
                                       c(int(status_ptr or 0)), int(max_sweeps),
                                       c(int(stream or 0)))


def sma_destroy(h):
    return lib().sma_destroy(h)


# ---- marshalling helpers ------------------------------------------------------

def colmajor(t):
    """Column-major copy of a 2-D torch tensor (strides (1, rows))."""
    return t.t().contiguous().t()


def _ptr_ld(a):
    """(address, leading dimension) of a column-major torch tensor or
    Fortran-ordered numpy array (host)."""
    if isinstance(a, np.ndarray):
        if a.ndim == 1:
            return a.ctypes.data, a.shape[0]
        if not a.flags.f_contiguous:
            raise ValueError("numpy matrices must be Fortran-ordered (np.asfortranarray)")
        return a.ctypes.data, a.shape[0]
    if a.dim() == 1:
        return a.data_ptr(), a.shape[0]
    if a.stride(0) != 1:
        raise ValueError("torch matrices must be column-major (use colmajor())")
    return a.data_ptr(), max(a.stride(1), a.shape[0])


@dataclass
class MultilevelProblem:
    """Multilevel structured matrix (Section 7): level t has an ell_t x q_t map
    with p_t distinct indices, level 1 outermost.  Three levels with scalar
    blocks (m = n = 1, Section 7.2) or two levels with m x n blocks."""
    level_maps: list       # (ell_t, q_t) int arrays, one per level
    level_p: list          # p_t per level
    m: int = 1
    n: int = 1


@dataclass
class Problem:
    ell: int
    q: int
    m: int
    n: int
    p: int
    block_map: np.ndarray    # (ell, q) int


class Handle:
    """Owns one sma handle; methods mirror the ABI calls."""

    def __init__(self, problems, prec=SMA_MIXED, decomp=SMA_TSVDM, mkind=SMA_M_DCT2,
                 layout=SMA_INPUT_DENSE, M_user=None, fixed_rank=0, rel_tol=0.0,
                 max_sweeps=0, stream=None, profile=False, graph=False,
                 precondition=None, autotune=False, sketch=None, cp_init=None, cp_iters=0):
        self._keep = []
        structs = []
        for pr in problems:
            if hasattr(pr, "level_maps"):
                structs.append(self._multilevel_struct(pr))
                continue
            bm = np.ascontiguousarray(np.asarray(pr.block_map, dtype=np.int32).ravel(order="F"))
            self._keep.append(bm)
            s = sma_problem(int(pr.ell), int(pr.q), int(pr.m), int(pr.n), int(pr.p),
                            bm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1,
                            None, None, None, None)
            structs.append(s)
        mu = None
        if M_user is not None:
            Mf = np.asfortranarray(np.asarray(M_user, dtype=np.float64))
            self._keep.append(Mf)
            mu = Mf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        sptr = None
        if stream is not None:
            sptr = ctypes.c_void_p(int(stream))
        # sketch = (Omega, Psi): the Gaussian maps of the randomized block-index
        # factor, m x s and n x s
        sk_cols, sk_om, sk_ps = 0, None, None
        if sketch is not None:
            Om = np.asfortranarray(np.asarray(sketch[0], dtype=np.float64))
            Ps = np.asfortranarray(np.asarray(sketch[1], dtype=np.float64))
            if Om.ndim != 2 or Ps.ndim != 2 or Om.shape[1] != Ps.shape[1]:
                raise ValueError("sketch maps must be m x s and n x s")
            self._keep += [Om, Ps]
            sk_cols = Om.shape[1]
            sk_om = Om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            sk_ps = Ps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        # cp_init = (Xf0, Zf0): the initial CP factors, m x r and n x r
        cp_x = cp_z = None
        if cp_init is not None:
            X0 = np.asfortranarray(np.asarray(cp_init[0], dtype=np.float64))
            Z0 = np.asfortranarray(np.asarray(cp_init[1], dtype=np.float64))
            self._keep += [X0, Z0]
            cp_x = X0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            cp_z = Z0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.opt = sma_options(prec, decomp, mkind, layout, mu, int(fixed_rank), float(rel_tol),
                               int(max_sweeps), sptr, 1 if profile else 0, 1 if graph else 0,
                               SMA_PRECOND_AUTO if precondition is None else int(precondition),
                               1 if autotune else 0, sk_cols, sk_om, sk_ps, int(cp_iters), cp_x,
                               cp_z)
        self.nprob = len(structs)
        self.prec = prec
        st, self.h = sma_create(structs, self.opt)
        _check(st, "sma_create")

    def _multilevel_struct(self, pr):
        I32 = ctypes.c_int32
        maps = [np.ascontiguousarray(np.asarray(m, dtype=np.int32).ravel(order="F"))
                for m in pr.level_maps]
        L = len(maps)
        ells = (I32 * L)(*[np.asarray(m).shape[0] for m in pr.level_maps])
        qs = (I32 * L)(*[np.asarray(m).shape[1] for m in pr.level_maps])
        ps = (I32 * L)(*[int(p) for p in pr.level_p])
        mptrs = (ctypes.POINTER(I32) * L)(*[m.ctypes.data_as(ctypes.POINTER(I32)) for m in maps])
        self._keep += [maps, ells, qs, ps, mptrs]
        return sma_problem(1, 1, int(pr.m), int(pr.n), 1, None, L, ells, qs, ps, mptrs)

    def compress(self, As, want_result=True, check=True):
        ptrs, ldas = zip(*[_ptr_ld(a) for a in As])
        res = (sma_result * self.nprob)() if want_result else None
        st = sma_compress(self.h, ptrs, ldas, res)
        if check and st not in (SMA_OK,):
            raise SmaError(st, "sma_compress")
        self.last_status = st
        return [r.as_dict() for r in res] if want_result else None

    def result(self, i=0) -> dict:
        r = sma_result()
        _check(sma_get_result(self.h, i, r), "sma_get_result")
        return r.as_dict()

    def ranks(self, i=0) -> np.ndarray:
        out = (ctypes.c_int32 * 65536)()
        cnt = ctypes.c_int32(0)
        _check(sma_get_ranks(self.h, i, out, cnt), "sma_get_ranks")
        return np.array(out[:cnt.value], dtype=np.int64)

    def apply(self, i, X, Y, nrhs=None):
        xp, ldx = _ptr_ld(X)
        yp, ldy = _ptr_ld(Y)
        if nrhs is None:
            nrhs = 1 if X.ndim == 1 else X.shape[1]
        _check(sma_apply(self.h, i, xp, ldx, yp, ldy, nrhs), "sma_apply")

    def reconstruct(self, i, Ahat):
        p, ld = _ptr_ld(Ahat)
        _check(sma_reconstruct(self.h, i, p, ld), "sma_reconstruct")

    def export_size(self, i, which) -> int:
        avail = ctypes.c_int64(0)
        _check(sma_export(self.h, i, which, 0, 0, avail), "sma_export")
        return avail.value

    def export(self, i, which, dst, count=None):
        avail = ctypes.c_int64(0)
        if count is None:
            count = dst.numel() if hasattr(dst, "numel") else dst.size
        ptr = dst.data_ptr() if hasattr(dst, "data_ptr") else dst.ctypes.data
        _check(sma_export(self.h, i, which, ptr, count, avail), "sma_export")

    def profile(self, reset=False) -> dict:
        """Per-stage device ms and call counts, and the kernel-launch count."""
        ms = (ctypes.c_double * len(STAGES))()
        calls = (ctypes.c_int64 * len(STAGES))()
        launches = ctypes.c_int64(0)
        _check(sma_profile(self.h, ms, calls, launches, reset), "sma_profile")
        return {"ms": dict(zip(STAGES, list(ms))), "calls": dict(zip(STAGES, list(calls))),
                "launches": launches.value}

    def close(self):
        if getattr(self, "h", None):
            sma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
