"""GB300 H^2 matrix-vector product: thin ctypes binding of libh2gb300.so.

The binding only marshals arguments: every step of the product runs in the
library's CUDA kernels (include/h2.h documents the ABI). PyTorch supplies
device memory and streams. There is no CPU fallback: if the shared library is
missing, importing ``paper_1902_01829_gb300`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libh2gb300.so")

H2_OK, H2_ERR_INVALID, H2_ERR_OOM, H2_ERR_CUDA, H2_ERR_UNSUPPORTED, H2_ERR_TIMEOUT = range(6)
STORAGE = {"fp64": 0, "fp16": 2, "bf16": 3, "int16": 4}
STATUS_NAMES = {0: "H2_OK", 1: "H2_ERR_INVALID", 2: "H2_ERR_OOM", 3: "H2_ERR_CUDA", 4: "H2_ERR_UNSUPPORTED",
                5: "H2_ERR_TIMEOUT"}

# every symbol include/h2.h declares
EXPORTS = ["h2_create", "h2_create_kernel_coupling", "h2_matvec", "h2_matvec_f32", "h2_matvec_host", "h2_check", "h2_debug_withhold_copy", "h2_info", "h2_profile",
           "h2_profile_read", "h2_matvec_static", "h2_matvec_static_check", "h2_create_generated", "h2_tune", "h2_destroy", "h2_batch_create", "h2_batch_matvec", "h2_batch_check",
           "h2_batch_info", "h2_batch_profile", "h2_batch_profile_read", "h2_batch_tune", "h2_batch_destroy",
           "h2_compress_create", "h2_compress_run", "h2_compress_result", "h2_compress_read", "h2_compress_profile",
           "h2_compress_profile_read", "h2_compress_info", "h2_compress_destroy", "h2_build", "h2_built_info",
           "h2_built_times", "h2_built_read", "h2_create_built", "h2_built_destroy", "h2_last_error"]
PHASES = ["upsweep", "coupling", "downsweep", "dense_expand"]
COMPRESS_PHASES = ["orthogonalize", "project", "basis_generation", "truncate", "project_truncated"]
COMPRESS_ARRAYS = {"U": 0, "V": 1, "E": 2, "F": 3, "S": 4, "T_ortho_U": 5, "T_ortho_V": 6, "R_U": 7, "R_V": 8,
                   "sigma_U": 9, "sigma_V": 10}


class H2Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class h2_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("depth", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("symmetric", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("leaf_offset", ctypes.c_void_p), ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("E", ctypes.c_void_p), ("F", ctypes.c_void_p),
                ("S_rowptr", ctypes.c_void_p), ("S_colidx", ctypes.c_void_p), ("S_val", ctypes.c_void_p),
                ("D_rowptr", ctypes.c_void_p), ("D_colidx", ctypes.c_void_p), ("D_val", ctypes.c_void_p),
                ("check_cover", ctypes.c_int32), ("bases_fp32", ctypes.c_int32)]


class h2_build_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int32), ("m", ctypes.c_int32), ("p", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("eta", ctypes.c_double), ("ell", ctypes.c_double),
                ("values", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class h2_coupling_kernel(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("dim", ctypes.c_int32), ("p", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ell", ctypes.c_double), ("cheb", ctypes.c_void_p)]


KERNELS = {"exp": 0, "matern32": 1}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.h2_create.argtypes = [ctypes.POINTER(h2_desc), ctypes.POINTER(vp)]
    lib.h2_create_kernel_coupling.argtypes = [ctypes.POINTER(h2_desc), ctypes.POINTER(h2_coupling_kernel), ctypes.POINTER(vp)]
    lib.h2_create_generated.argtypes = [ctypes.POINTER(h2_desc), ctypes.POINTER(h2_coupling_kernel), vp, ctypes.POINTER(vp)]
    lib.h2_matvec.argtypes = [vp, i32, vp, i64, vp, i64, vp]
    lib.h2_matvec_host.argtypes = [vp, i32, vp, i64, vp, i64, vp]
    lib.h2_matvec_f32.argtypes = [vp, i32, vp, i64, vp, i64, vp]
    lib.h2_info.argtypes = [vp, vp]
    lib.h2_destroy.argtypes = [vp]
    lib.h2_profile.argtypes = [vp, i32]
    lib.h2_check.argtypes = [vp, vp]
    lib.h2_matvec_static.argtypes = [ctypes.POINTER(h2_desc), i64, i32, vp, i64, vp, i64, vp]
    lib.h2_matvec_static_check.argtypes = [vp]
    lib.h2_debug_withhold_copy.argtypes = [vp, i32, i64]
    lib.h2_profile_read.argtypes = [vp, vp, vp]
    lib.h2_batch_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
    lib.h2_batch_matvec.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.h2_batch_check.argtypes = [vp, vp]
    lib.h2_batch_info.argtypes = [vp, vp]
    lib.h2_batch_destroy.argtypes = [vp]
    lib.h2_batch_profile.argtypes = [vp, i32]
    lib.h2_batch_profile_read.argtypes = [vp, vp, vp]
    lib.h2_tune.argtypes = [vp, i32, vp, i64, vp, i64, vp, vp]
    lib.h2_batch_tune.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.h2_compress_create.argtypes = [ctypes.POINTER(h2_desc), ctypes.POINTER(vp)]
    lib.h2_compress_run.argtypes = [vp, ctypes.c_double, vp]
    lib.h2_compress_result.argtypes = [vp, vp, vp, vp, vp]
    lib.h2_compress_read.argtypes = [vp, i32, vp, i64, vp]
    lib.h2_compress_profile.argtypes = [vp, i32]
    lib.h2_compress_profile_read.argtypes = [vp, vp, vp]
    lib.h2_compress_destroy.argtypes = [vp]
    lib.h2_compress_info.argtypes = [vp, vp]
    lib.h2_build.argtypes = [ctypes.POINTER(h2_build_desc), vp, ctypes.POINTER(vp)]
    lib.h2_built_info.argtypes = [vp, vp]
    lib.h2_built_times.argtypes = [vp, vp]
    lib.h2_built_read.argtypes = [vp, i32, vp, i64]
    lib.h2_built_destroy.argtypes = [vp]
    lib.h2_create_built.argtypes = [vp, i32, i32, i32, ctypes.POINTER(vp)]
    lib.h2_last_error.restype = ctypes.c_char_p
    for name in ("h2_matvec_f32", "h2_create_built", "h2_build", "h2_built_info", "h2_built_times", "h2_built_read", "h2_built_destroy", "h2_compress_create", "h2_compress_run", "h2_compress_result", "h2_compress_read",
                 "h2_compress_profile", "h2_compress_profile_read", "h2_compress_info", "h2_compress_destroy", "h2_create", "h2_create_kernel_coupling", "h2_create_generated", "h2_matvec", "h2_matvec_host", "h2_check", "h2_debug_withhold_copy", "h2_info", "h2_profile",
                 "h2_profile_read", "h2_matvec_static", "h2_matvec_static_check", "h2_destroy", "h2_batch_create", "h2_batch_matvec",
                 "h2_batch_check", "h2_batch_info", "h2_batch_profile", "h2_batch_profile_read", "h2_batch_destroy",
                 "h2_tune", "h2_batch_tune"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()


def _check(status: int):
    if status != H2_OK:
        raise H2Error(status, _lib.h2_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())  # torch tensor


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class H2Matrix:
    """An H^2 matrix resident on the current CUDA device (h2_create / h2_destroy)."""

    def __init__(self, *, n, depth, rank, leaf_offset, U, E, S_rowptr, S_colidx, S_val, D_rowptr, D_colidx, D_val,
                 V=None, F=None, storage="fp64", check_cover=False, bases_fp32=False, coupling_kernel=None,
                 points=None):
        """coupling_kernel: None (S_val stored), or dict(kernel="exp"|"matern32", ell, cheb) with cheb the
        (n_nodes, dim, p) Chebyshev nodes of every node: the coupling blocks are then evaluated from the
        kernel at the interpolation points in every product (h2_create_kernel_coupling), S_val unused.
        points: with coupling_kernel, the (n, dim) points in cluster order: the dense blocks are then
        generated on the device from the kernel (h2_create_generated), D_val unused."""
        sym = V is None and F is None
        keep = dict(leaf_offset=np.ascontiguousarray(leaf_offset, dtype=np.int64),
                    U=np.ascontiguousarray(U, dtype=np.float64), E=np.ascontiguousarray(E, dtype=np.float64),
                    V=None if sym else np.ascontiguousarray(V, dtype=np.float64),
                    F=None if sym else np.ascontiguousarray(F, dtype=np.float64),
                    S_rowptr=np.ascontiguousarray(S_rowptr, dtype=np.int32),
                    S_colidx=np.ascontiguousarray(S_colidx, dtype=np.int32),
                    S_val=None if coupling_kernel is not None else np.ascontiguousarray(S_val, dtype=np.float64),
                    D_rowptr=np.ascontiguousarray(D_rowptr, dtype=np.int32),
                    D_colidx=np.ascontiguousarray(D_colidx, dtype=np.int32),
                    D_val=None if points is not None else np.ascontiguousarray(D_val, dtype=np.float64))
        d = h2_desc(n=int(n), depth=int(depth), rank=int(rank), symmetric=1 if sym else 0, storage=STORAGE[storage],
                    check_cover=1 if check_cover else 0, bases_fp32=1 if bases_fp32 else 0,
                    **{key: _ptr(val) for key, val in keep.items()})
        self._h = ctypes.c_void_p()
        if coupling_kernel is None:
            _check(_lib.h2_create(ctypes.byref(d), ctypes.byref(self._h)))
        else:
            cheb = np.ascontiguousarray(coupling_kernel["cheb"], dtype=np.float64)
            kc = h2_coupling_kernel(kernel=KERNELS[coupling_kernel["kernel"]], dim=int(cheb.shape[1]),
                                    p=int(cheb.shape[2]), reserved=0, ell=float(coupling_kernel["ell"]), cheb=_ptr(cheb))
            if points is None:
                _check(_lib.h2_create_kernel_coupling(ctypes.byref(d), ctypes.byref(kc), ctypes.byref(self._h)))
            else:
                pts = np.ascontiguousarray(points, dtype=np.float64)
                _check(_lib.h2_create_generated(ctypes.byref(d), ctypes.byref(kc), _ptr(pts), ctypes.byref(self._h)))
        self.n = int(n)

    @classmethod
    def from_generator(cls, A, storage="fp64", check_cover=False, bases_fp32=False, coupling="stored",
                       dense="stored") -> "H2Matrix":
        """From an object with the generator's arrays (h2gen.H2Matrix). coupling="kernel" evaluates the
        coupling blocks from the generator's kernel at its interpolation points in every product;
        dense="generated" (with coupling="kernel") generates the dense blocks on the device from the
        generator's points."""
        ck = None
        if coupling == "kernel":
            ck = dict(kernel=A.kernel, ell=A.ell, cheb=A.chebyshev_nodes())
        elif coupling != "stored":
            raise ValueError(f"coupling={coupling!r}: 'stored' or 'kernel'")
        if dense not in ("stored", "generated") or (dense == "generated" and ck is None):
            raise ValueError(f"dense={dense!r}: 'stored', or 'generated' with coupling='kernel'")
        return cls(n=A.n, depth=A.q, rank=A.k, leaf_offset=A.leaf_offset, U=A.U, E=A.E, S_rowptr=A.S_rowptr,
                   S_colidx=A.S_colidx, S_val=A.S_val, D_rowptr=A.D_rowptr, D_colidx=A.D_colidx, D_val=A.D_val,
                   storage=storage, check_cover=check_cover, bases_fp32=bases_fp32, coupling_kernel=ck,
                   points=A.points if dense == "generated" else None)

    def matvec(self, x, y=None, stream=None):
        """y = A^H x on the device. x, y: torch float64 CUDA tensors, shape (n,) or (n, nv) column-major."""
        import torch
        assert x.is_cuda and x.dtype == torch.float64
        vec = x.dim() == 1
        X = x.unsqueeze(1) if vec else x
        if X.stride(0) != 1:
            X = X.t().contiguous().t()
        nv = X.shape[1]
        if y is None:
            Y = torch.empty((nv, self.n), dtype=torch.float64, device=x.device).t()
        else:
            Y = y.unsqueeze(1) if y.dim() == 1 else y
            assert Y.stride(0) == 1 and Y.dtype == torch.float64
        ldx = X.stride(1) if nv > 1 else self.n
        ldy = Y.stride(1) if nv > 1 else self.n
        _check(_lib.h2_matvec(self._h, nv, _ptr(X), ldx, _ptr(Y), ldy, _stream_ptr(stream)))
        return Y[:, 0] if (vec and y is None) else (y if y is not None else Y)

    def matvec_f32(self, x, y=None, stream=None):
        """y = A^H x with FP32 vectors (h2_matvec_f32; scaled storage forms). x, y: torch float32 CUDA
        tensors, shape (n,) or (n, nv) column-major."""
        import torch
        assert x.is_cuda and x.dtype == torch.float32
        vec = x.dim() == 1
        X = x.unsqueeze(1) if vec else x
        if X.stride(0) != 1:
            X = X.t().contiguous().t()
        nv = X.shape[1]
        if y is None:
            Y = torch.empty((nv, self.n), dtype=torch.float32, device=x.device).t()
        else:
            Y = y.unsqueeze(1) if y.dim() == 1 else y
            assert Y.stride(0) == 1 and Y.dtype == torch.float32
        ldx = X.stride(1) if nv > 1 else self.n
        ldy = Y.stride(1) if nv > 1 else self.n
        _check(_lib.h2_matvec_f32(self._h, nv, _ptr(X), ldx, _ptr(Y), ldy, _stream_ptr(stream)))
        return Y[:, 0] if (vec and y is None) else (y if y is not None else Y)

    def matvec_host(self, x: np.ndarray, y: np.ndarray | None = None, stream=None) -> np.ndarray:
        """y = A^H x with host (numpy) buffers; copies are part of the call."""
        vec = x.ndim == 1
        X = np.asfortranarray(x[:, None] if vec else x, dtype=np.float64)
        nv = X.shape[1]
        Y = np.empty((self.n, nv), order="F") if y is None else y
        _check(_lib.h2_matvec_host(self._h, nv, _ptr(X), self.n, _ptr(Y), self.n, _stream_ptr(stream)))
        return Y[:, 0] if (vec and y is None) else Y

    def tune(self, x, y, stream=None) -> dict:
        """Choose the launch parameters by timing products with x, y (h2_tune); y holds A^H x on return."""
        import torch
        X = x.unsqueeze(1) if x.dim() == 1 else x
        Y = y.unsqueeze(1) if y.dim() == 1 else y
        assert X.stride(0) == 1 and Y.stride(0) == 1 and X.dtype == torch.float64 and Y.dtype == torch.float64
        nv = X.shape[1]
        ch = np.zeros(3, dtype=np.int32)
        _check(_lib.h2_tune(self._h, nv, _ptr(X), X.stride(1) if nv > 1 else self.n, _ptr(Y),
                            Y.stride(1) if nv > 1 else self.n, _stream_ptr(stream), _ptr(ch)))
        return {"consumer_warps": int(ch[0]), "chunk_blocks": int(ch[1]), "tree_leaves": int(ch[2])}

    def info(self) -> dict:
        a = np.zeros(8, dtype=np.int64)
        _check(_lib.h2_info(self._h, _ptr(a)))
        keys = ["paper_bytes", "device_bytes", "nS", "nD", "q", "k", "m_max", "n"]
        return {key: int(v) for key, v in zip(keys, a)}

    def check(self, stream=None):
        """Wait for the stream and raise H2Error(H2_ERR_TIMEOUT) if a bounded device wait ran out (h2_check)."""
        _check(_lib.h2_check(self._h, _stream_ptr(stream)))

    def debug_withhold_copy(self, item: int, wait_budget_cycles: int = 0):
        """Test hook: make the next product's dense kernel withhold one copy (h2_debug_withhold_copy)."""
        _check(_lib.h2_debug_withhold_copy(self._h, int(item), int(wait_budget_cycles)))

    def profile(self, enable: bool = True):
        """Record per-phase CUDA events in every product while enabled (h2_profile)."""
        _check(_lib.h2_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> tuple[dict, int]:
        """Summed milliseconds per phase since the last read, and the kernel launch count."""
        ms = np.zeros(len(PHASES), dtype=np.float64)
        n = np.zeros(1, dtype=np.int64)
        _check(_lib.h2_profile_read(self._h, _ptr(ms), _ptr(n)))
        return dict(zip(PHASES, ms.tolist())), int(n[0])

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.h2_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class H2Batch:
    """Independent precision-form matrices multiplied together, one launch per phase
    (h2_batch_create / h2_batch_matvec). Keeps its member H2Matrix objects alive."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (ctypes.c_void_p * len(self.mats))(*[m._h.value for m in self.mats])
        self._b = ctypes.c_void_p()
        _check(_lib.h2_batch_create(arr, len(self.mats), ctypes.byref(self._b)))

    def prepare(self, xs, ys):
        """Argument arrays of h2_batch_matvec for lists of (n_i, nv_i) column-major torch tensors
        (None or nv_i = 0 skips a matrix)."""
        count = len(self.mats)
        assert len(xs) == count and len(ys) == count
        nv = np.zeros(count, dtype=np.int32)
        ldx = np.zeros(count, dtype=np.int64)
        ldy = np.zeros(count, dtype=np.int64)
        xp = (ctypes.c_void_p * count)()
        yp = (ctypes.c_void_p * count)()
        for i, (m, x, y) in enumerate(zip(self.mats, xs, ys)):
            if x is None or (x.dim() == 2 and x.shape[1] == 0):
                continue
            X = x.unsqueeze(1) if x.dim() == 1 else x
            Y = y.unsqueeze(1) if y.dim() == 1 else y
            assert X.stride(0) == 1 and Y.stride(0) == 1 and X.shape == Y.shape and X.shape[0] == m.n
            nv[i] = X.shape[1]
            ldx[i] = X.stride(1) if X.shape[1] > 1 else m.n
            ldy[i] = Y.stride(1) if Y.shape[1] > 1 else m.n
            xp[i] = X.data_ptr()
            yp[i] = Y.data_ptr()
        return (nv, xp, ldx, yp, ldy)

    def matvec_prepared(self, args, stream=None):
        nv, xp, ldx, yp, ldy = args
        _check(_lib.h2_batch_matvec(self._b, _ptr(nv), xp, _ptr(ldx), yp, _ptr(ldy), _stream_ptr(stream)))

    def matvec(self, xs, ys=None, stream=None):
        """ys[i] = A_i xs[i]; xs: list of float64 CUDA tensors (n_i,) or (n_i, nv_i) column-major."""
        import torch
        if ys is None:
            ys = []
            for m, x in zip(self.mats, xs):
                if x is None:
                    ys.append(None)
                elif x.dim() == 1:
                    ys.append(torch.empty(m.n, dtype=torch.float64, device=x.device))
                else:
                    ys.append(torch.empty((x.shape[1], m.n), dtype=torch.float64, device=x.device).t())
        self.matvec_prepared(self.prepare(xs, ys), stream)
        return ys

    def check(self, stream=None):
        _check(_lib.h2_batch_check(self._b, _stream_ptr(stream)))

    def tune(self, xs, ys, stream=None) -> dict:
        """Choose the batch's launch parameters by timing batched products (h2_batch_tune)."""
        nv, xp, ldx, yp, ldy = self.prepare(xs, ys)
        ch = np.zeros(3, dtype=np.int32)
        _check(_lib.h2_batch_tune(self._b, _ptr(nv), xp, _ptr(ldx), yp, _ptr(ldy), _stream_ptr(stream), _ptr(ch)))
        return {"consumer_warps": int(ch[0]), "chunk_blocks": int(ch[1]), "tree_leaves": int(ch[2])}

    def profile(self, enable: bool = True):
        """Record per-phase CUDA events in every batched product while enabled (h2_batch_profile)."""
        _check(_lib.h2_batch_profile(self._b, 1 if enable else 0))

    def profile_read(self) -> tuple[dict, int]:
        """Summed milliseconds per phase since the last read, and the kernel launch count."""
        ms = np.zeros(len(PHASES), dtype=np.float64)
        n = np.zeros(1, dtype=np.int64)
        _check(_lib.h2_batch_profile_read(self._b, _ptr(ms), _ptr(n)))
        return dict(zip(PHASES, ms.tolist())), int(n[0])

    def info(self) -> dict:
        a = np.zeros(6, dtype=np.int64)
        _check(_lib.h2_batch_info(self._b, _ptr(a)))
        keys = ["members", "coupling_rows", "tree_jobs", "dense_items", "device_bytes", "launches_per_pass"]
        return {key: int(v) for key, v in zip(keys, a)}

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            _lib.h2_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Compressor:
    """Algebraic compression of an FP64 H^2 matrix on the current CUDA device
    (h2_compress_create / h2_compress_run / h2_compress_read / h2_compress_destroy)."""

    def __init__(self, *, n, depth, rank, leaf_offset, U, E, S_rowptr, S_colidx, S_val, D_rowptr, D_colidx,
                 V=None, F=None):
        sym = V is None and F is None
        keep = dict(leaf_offset=np.ascontiguousarray(leaf_offset, dtype=np.int64),
                    U=np.ascontiguousarray(U, dtype=np.float64), E=np.ascontiguousarray(E, dtype=np.float64),
                    V=None if sym else np.ascontiguousarray(V, dtype=np.float64),
                    F=None if sym else np.ascontiguousarray(F, dtype=np.float64),
                    S_rowptr=np.ascontiguousarray(S_rowptr, dtype=np.int32),
                    S_colidx=np.ascontiguousarray(S_colidx, dtype=np.int32),
                    S_val=np.ascontiguousarray(S_val, dtype=np.float64),
                    D_rowptr=np.ascontiguousarray(D_rowptr, dtype=np.int32),
                    D_colidx=np.ascontiguousarray(D_colidx, dtype=np.int32))
        d = h2_desc(n=int(n), depth=int(depth), rank=int(rank), symmetric=1 if sym else 0, storage=STORAGE["fp64"],
                    check_cover=0, bases_fp32=0, D_val=None, **{key: _ptr(val) for key, val in keep.items()})
        self._c = ctypes.c_void_p()
        _check(_lib.h2_compress_create(ctypes.byref(d), ctypes.byref(self._c)))
        self.n, self.q, self.k, self.sym = int(n), int(depth), int(rank), sym
        self.nS = int(keep["S_colidx"].size)

    @classmethod
    def from_generator(cls, A, V=None, F=None) -> "Compressor":
        return cls(n=A.n, depth=A.q, rank=A.k, leaf_offset=A.leaf_offset, U=A.U, E=A.E, S_rowptr=A.S_rowptr,
                   S_colidx=A.S_colidx, S_val=A.S_val, D_rowptr=A.D_rowptr, D_colidx=A.D_colidx, V=V, F=F)

    def run(self, eps: float, stream=None):
        """eps < 0: orthogonalize and project only; 0 <= eps < 1: the whole compression (asynchronous)."""
        _check(_lib.h2_compress_run(self._c, float(eps), _stream_ptr(stream)))

    def result(self, stream=None) -> tuple[int, list, list]:
        """(uniform rank, row-tree level ranks, column-tree level ranks); waits for the stream."""
        k = np.zeros(1, dtype=np.int32)
        ru = np.zeros(self.q + 1, dtype=np.int32)
        rv = np.zeros(self.q + 1, dtype=np.int32)
        _check(_lib.h2_compress_result(self._c, _ptr(k), _ptr(ru), _ptr(rv), _stream_ptr(stream)))
        return int(k[0]), ru.tolist(), rv.tolist()

    def read(self, what: str, stream=None) -> np.ndarray:
        """One result array (see COMPRESS_ARRAYS) as a flat numpy array."""
        K = self.result(stream)[0]
        nodes = (2 << self.q) - 1
        size = {"U": self.n * K, "V": self.n * K, "E": (nodes - 1) * K * K, "F": (nodes - 1) * K * K,
                "S": self.nS * K * K, "T_ortho_U": nodes * self.k ** 2, "T_ortho_V": nodes * self.k ** 2,
                "R_U": nodes * self.k ** 2, "R_V": nodes * self.k ** 2, "sigma_U": nodes * self.k,
                "sigma_V": nodes * self.k}[what]
        out = np.empty(size, dtype=np.float64)
        _check(_lib.h2_compress_read(self._c, COMPRESS_ARRAYS[what], _ptr(out), size, _stream_ptr(stream)))
        return out

    def profile(self, enable: bool = True):
        _check(_lib.h2_compress_profile(self._c, 1 if enable else 0))

    def profile_read(self) -> tuple[dict, int]:
        ms = np.zeros(len(COMPRESS_PHASES), dtype=np.float64)
        n = np.zeros(1, dtype=np.int64)
        _check(_lib.h2_compress_profile_read(self._c, _ptr(ms), _ptr(n)))
        return dict(zip(COMPRESS_PHASES, ms.tolist())), int(n[0])

    def info(self) -> dict:
        a = np.zeros(6, dtype=np.int64)
        _check(_lib.h2_compress_info(self._c, _ptr(a)))
        keys = ["max_sweeps", "total_sweeps", "device_bytes", "nS", "q", "k"]
        return {key: int(v) for key, v in zip(keys, a)}

    def close(self):
        if getattr(self, "_c", None) is not None and self._c.value:
            _lib.h2_compress_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BUILT_ARRAYS = {"perm": (0, np.int64), "leaf_offset": (1, np.int64), "points": (2, np.float64), "cheb": (3, np.float64),
                "S_rowptr": (4, np.int32), "S_colidx": (5, np.int32), "D_rowptr": (6, np.int32),
                "D_colidx": (7, np.int32), "D_valoff": (8, np.int64), "U": (9, np.float64), "E": (10, np.float64),
                "S_val": (11, np.float64), "D_val": (12, np.float64)}
BUILD_VALUES = {"U": 1, "E": 2, "S": 4, "D": 8}


class Built:
    """A covariance H^2 matrix constructed on the current CUDA device (h2_build): cluster tree, boxes,
    Chebyshev nodes, block structure and, as asked, FP64 values (U, E, S, D)."""

    def __init__(self, points, *, m, p, eta, kernel="exp", ell=0.1, values=("U", "E", "S", "D")):
        pts = np.ascontiguousarray(points, dtype=np.float64)
        n, dim = pts.shape
        d = h2_build_desc(n=n, dim=dim, m=int(m), p=int(p), kernel=KERNELS[kernel], eta=float(eta), ell=float(ell),
                          values=sum(BUILD_VALUES[v] for v in values), reserved=0)
        self._b = ctypes.c_void_p()
        _check(_lib.h2_build(ctypes.byref(d), _ptr(pts), ctypes.byref(self._b)))
        self.n, self.dim, self.p = n, dim, int(p)
        a = np.zeros(8, dtype=np.int64)
        _check(_lib.h2_built_info(self._b, _ptr(a)))
        self.q, self.k, self.nS, self.nD, self.nDval, self.n_nodes, self.leaves, self.device_bytes = (int(v) for v in a)

    def times(self) -> dict:
        ms = np.zeros(3, dtype=np.float64)
        _check(_lib.h2_built_times(self._b, _ptr(ms)))
        return {"tree_ms": float(ms[0]), "blocks_ms": float(ms[1]), "values_ms": float(ms[2])}

    def read(self, what: str) -> np.ndarray:
        code, dt = BUILT_ARRAYS[what]
        kk = self.k * self.k
        size = {"perm": self.n, "leaf_offset": self.leaves + 1, "points": self.n * self.dim,
                "cheb": self.n_nodes * self.dim * self.p, "S_rowptr": self.n_nodes + 1, "S_colidx": self.nS,
                "D_rowptr": self.leaves + 1, "D_colidx": self.nD, "D_valoff": self.nD + 1, "U": self.n * self.k,
                "E": (self.n_nodes - 1) * kk, "S_val": self.nS * kk, "D_val": self.nDval}[what]
        out = np.empty(size, dtype=dt)
        _check(_lib.h2_built_read(self._b, code, _ptr(out), size))
        return out

    def matrix(self, storage="fp64", bases_fp32=False, coupling="stored", dense="stored") -> "H2Matrix":
        """A product handle of this matrix (h2_create_built); coupling="kernel" evaluates the coupling
        blocks in every product, dense="generated" (with it) generates the dense blocks on the device."""
        flags = (1 if coupling == "kernel" else 0) | (2 if dense == "generated" else 0)
        M = H2Matrix.__new__(H2Matrix)
        M._h = ctypes.c_void_p()
        _check(_lib.h2_create_built(self._b, STORAGE[storage], 1 if bases_fp32 else 0, flags, ctypes.byref(M._h)))
        M.n = self.n
        return M

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            _lib.h2_built_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def matvec_static(n, depth, rank, leaf_offset, U, E, S_rowptr, S_colidx, S_val, D_rowptr, D_colidx, D_val, x, y,
                  V=None, F=None, stream=None, n_dense_blocks=None):
    """y = A^H x through h2_matvec_static, which allocates nothing.

    For callers that may not allocate device memory: every array is a torch
    CUDA tensor the caller already owns (int64 leaf_offset, int32 index arrays,
    float64 values); x and y are (n, nv) column-major float64 CUDA tensors.
    The library's only working memory is a static 16 MiB device array.
    n_dense_blocks defaults to D_colidx.numel(). A malformed description is
    reported by matvec_static_check(), not by this call.
    """
    sym = V is None and F is None
    d = h2_desc(n=int(n), depth=int(depth), rank=int(rank), symmetric=1 if sym else 0, storage=STORAGE["fp64"],
                check_cover=0, leaf_offset=_ptr(leaf_offset), U=_ptr(U), V=_ptr(V), E=_ptr(E), F=_ptr(F),
                S_rowptr=_ptr(S_rowptr), S_colidx=_ptr(S_colidx), S_val=_ptr(S_val), D_rowptr=_ptr(D_rowptr),
                D_colidx=_ptr(D_colidx), D_val=_ptr(D_val))
    X = x.unsqueeze(1) if x.dim() == 1 else x
    Y = y.unsqueeze(1) if y.dim() == 1 else y
    assert X.stride(0) == 1 and Y.stride(0) == 1
    nv = X.shape[1]
    ldx = X.stride(1) if nv > 1 else int(n)
    ldy = Y.stride(1) if nv > 1 else int(n)
    nd = int(D_colidx.numel()) if n_dense_blocks is None else int(n_dense_blocks)
    _check(_lib.h2_matvec_static(ctypes.byref(d), nd, nv, _ptr(X), ldx, _ptr(Y), ldy, _stream_ptr(stream)))
    return y


def matvec_static_check(stream=None):
    """Raise H2Error (H2_ERR_INVALID) if a static product since the last check found a malformed
    description; synchronizes the stream and clears the error."""
    _check(_lib.h2_matvec_static_check(_stream_ptr(stream)))
