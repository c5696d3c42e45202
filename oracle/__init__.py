"""ORACLE for the H^2 matrix-vector product (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never does, and this
package never imports the library.

Two independent forms of y = A^H x:
  * ``matvec``  -- O-tree: plain FP64 C traversal, one step per equation of the
    paper (Eq. 2 upsweep, Eq. 3 coupling, Eq. 5 downsweep, Eq. 4 expansion, the
    dense near-field blocks of Sec. 2.2); see ``h2_oracle.c``.
  * ``dense.assemble`` -- O-dense: the n x n matrix assembled block by block from
    the same representation (nested bases expanded with Eq. 1), for n <= 8192.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h2_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MUTATIONS = {
    "F_transposed": 1, "E_transposed": 2, "no_downsweep": 3, "S_transposed": 4, "no_dense": 5,
    "one_child": 6, "D_transposed": 7, "downsweep_sign": 8, "coupling_row_x": 9, "V_rowmajor": 10,
    "skip_top_level": 11,
}


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2 -fopenmp, no floating-point contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_matvec.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      i32, vp, i64, vp, i64, vp, i32]
        lib.oracle_matvec.restype = i32
        lib.oracle_threads.restype = i32
        lib.oracle_set_threads.argtypes = [i32]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_load().oracle_threads())


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def matvec(A, x: np.ndarray, *, U=None, V=None, E=None, F=None, S_val=None, D_val=None,
           leaf_mask: np.ndarray | None = None, mutate: str | int = 0) -> np.ndarray:
    """y = A^H x in FP64 (O-tree).

    A: an object with the generator's structure arrays (n, q, k, leaf_offset,
    S_rowptr, S_colidx, D_rowptr, D_colidx, D_valoff) and, unless overridden by
    keyword, the value arrays U, E (V == U, F == E), S_val, D_val.
    x: n (or n x nv) FP64. leaf_mask: optional bool per leaf; unmarked rows of y are NaN.
    """
    U = A.U if U is None else U
    V = U if V is None else V
    E = A.E if E is None else E
    F = E if F is None else F
    S_val = A.S_val if S_val is None else S_val
    D_val = A.D_val if D_val is None else D_val
    vec = x.ndim == 1
    X = np.asfortranarray(x[:, None] if vec else x, dtype=np.float64)
    nv = X.shape[1]
    Y = np.full((A.n, nv), np.nan, order="F") if leaf_mask is not None else np.empty((A.n, nv), order="F")
    mask = None
    if leaf_mask is not None:
        mask = np.ascontiguousarray(leaf_mask, dtype=np.uint8)
        assert mask.size == A.leaf_offset.size - 1
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (U, V, E, F, S_val, D_val)]
    mut = MUTATIONS[mutate] if isinstance(mutate, str) else int(mutate)
    rc = _load().oracle_matvec(A.n, A.q, A.k, _p(A.leaf_offset), *[_p(a) for a in arrs[:4]],
                               _p(A.S_rowptr), _p(A.S_colidx), _p(arrs[4]), _p(A.D_rowptr), _p(A.D_colidx),
                               _p(A.D_valoff), _p(arrs[5]), nv, _p(X), A.n, _p(Y), A.n, _p(mask), mut)
    if rc != 0:
        raise MemoryError("oracle_matvec: allocation failed")
    return Y[:, 0] if vec else Y


def rel_l2(y: np.ndarray, y_ref: np.ndarray) -> float:
    """Relative l2 error; for several columns the maximum over columns."""
    y = np.asarray(y, dtype=np.float64)
    y_ref = np.asarray(y_ref, dtype=np.float64)
    if y.ndim == 1:
        return float(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref))
    num = np.linalg.norm(y - y_ref, axis=0)
    den = np.linalg.norm(y_ref, axis=0)
    return float(np.max(num / den))
