"""Seeded synthetic H^2 covariance matrices (inputs for the oracle, the tests and the bench).

The construction follows the paper's experiments (Sec. 4.6): points in the unit
square/cube, a KD cluster tree, Chebyshev interpolation bases and transfer
matrices, a dual traversal producing the coupling quadtree (kernel evaluated at
interpolation points) and the dense leaf blocks (kernel evaluated at points).
The heavy lifting is in ``h2gen.c``; this module compiles it on demand and wraps
it with ctypes. It contains none of the matrix-vector product's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h2gen.c")
_LIB = os.path.join(_HERE, "libh2gen.so")
_lib = None

KERNELS = {"exp": 0, "matern32": 1, "poly": 2, "const": 3}


def build(force: bool = False) -> str:
    """Compile libh2gen.so next to its source (gcc, OpenMP, no fp contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.h2gen_build.argtypes = [i32, i64, i32, i32, dbl, i32, dbl, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        lib.h2gen_build.restype = i32
        lib.h2gen_info.argtypes = [vp, vp]
        lib.h2gen_fill_structure.argtypes = [vp] + [vp] * 8
        lib.h2gen_fill_values.argtypes = [vp] * 5
        lib.h2gen_fill_cheb.argtypes = [vp, vp]
        lib.h2gen_free.argtypes = [vp]
        lib.h2gen_normal.argtypes = [ctypes.c_uint64, i64, vp]
        lib.h2gen_uniform.argtypes = [ctypes.c_uint64, i64, vp]
        lib.h2gen_exact_matvec_rows.argtypes = [vp, vp, i64, i32, vp, i64, vp]
        lib.h2gen_kernel_matrix.argtypes = [vp, vp, i64, vp, i64, vp]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def normal(seed: int, shape) -> np.ndarray:
    """N(0,1) samples (xoshiro256** + Box-Muller), filled in C order."""
    out = np.empty(shape, dtype=np.float64)
    _load().h2gen_normal(ctypes.c_uint64(seed), out.size, _p(out))
    return out


def uniform(seed: int, shape) -> np.ndarray:
    """U[0,1) samples (xoshiro256**), filled in C order."""
    out = np.empty(shape, dtype=np.float64)
    _load().h2gen_uniform(ctypes.c_uint64(seed), out.size, _p(out))
    return out


def vectors(seed: int, n: int, nv: int, dist: str = "normal") -> np.ndarray:
    """n x nv test vectors, column-major (Fortran order), x ~ N(0,1) or U[0,1)."""
    flat = normal(seed, n * nv) if dist == "normal" else uniform(seed, n * nv)
    return flat.reshape(nv, n).T  # column v = flat[v*n:(v+1)*n]; result is F-contiguous


@dataclass
class H2Matrix:
    """An H^2 matrix in the library's input format (see h2gen.c for the layout)."""
    dim: int
    n: int
    m: int
    p: int
    k: int
    q: int
    eta: float
    kernel: str
    ell: float
    seed: int
    points: np.ndarray          # n x dim, cluster order
    perm: np.ndarray            # cluster position -> original index
    leaf_offset: np.ndarray     # int64 [2^q + 1]
    S_rowptr: np.ndarray        # int32 [2^(q+1)]  (all nodes, heap order)
    S_colidx: np.ndarray        # int32 [nS] heap index of column node
    D_rowptr: np.ndarray        # int32 [2^q + 1]
    D_colidx: np.ndarray        # int32 [nD] leaf index
    D_valoff: np.ndarray        # int64 [nD + 1]
    U: np.ndarray = field(repr=False, default=None)      # sum size_i*k
    E: np.ndarray = field(repr=False, default=None)      # (n_nodes-1)*k*k
    S_val: np.ndarray = field(repr=False, default=None)  # nS*k*k
    D_val: np.ndarray = field(repr=False, default=None)  # D_valoff[-1]
    _h: ctypes.c_void_p = field(repr=False, default=None)

    @property
    def n_nodes(self) -> int:
        return (2 << self.q) - 1

    @property
    def leaves(self) -> int:
        return 1 << self.q

    @property
    def nS(self) -> int:
        return int(self.S_colidx.size)

    @property
    def nD(self) -> int:
        return int(self.D_colidx.size)

    @property
    def V(self) -> np.ndarray:  # symmetric construction: V == U
        return self.U

    @property
    def F(self) -> np.ndarray:  # symmetric construction: F == E
        return self.E

    def leaf_size(self, i: int) -> int:
        return int(self.leaf_offset[i + 1] - self.leaf_offset[i])

    def exact_matvec_rows(self, rows: np.ndarray, x: np.ndarray) -> np.ndarray:
        """Rows (cluster order) of K x with the exact kernel matrix K (not the H^2 form)."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        x = np.asfortranarray(x, dtype=np.float64)
        if x.ndim == 1:
            x = x[:, None]
        out = np.empty((rows.size, x.shape[1]), dtype=np.float64, order="F")
        _load().h2gen_exact_matvec_rows(self._h, _p(rows), rows.size, x.shape[1], _p(x), x.shape[0], _p(out))
        return out

    def dense_kernel_matrix(self) -> np.ndarray:
        """The exact n x n kernel matrix in cluster order (small n only)."""
        assert self.n <= 8192
        idx = np.arange(self.n, dtype=np.int64)
        out = np.empty((self.n, self.n), order="F")
        _load().h2gen_kernel_matrix(self._h, _p(idx), self.n, _p(idx), self.n, _p(out))
        return out

    def chebyshev_nodes(self) -> np.ndarray:
        """(n_nodes, dim, p) first-kind Chebyshev nodes of every node's box per dimension; the
        node's interpolation points are their tensor grid (dimension 0 slowest)."""
        out = np.empty((self.n_nodes, self.dim, self.p), dtype=np.float64)
        _load().h2gen_fill_cheb(self._h, _p(out))
        return out

    def free(self):
        if self._h is not None:
            _load().h2gen_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def generate(dim: int = 2, n: int = 4096, m: int = 32, p: int = 4, eta: float = 0.9, kernel: str = "exp",
             ell: float = 0.1, seed: int = 0, points: np.ndarray | None = None, values: bool = True,
             coupling_values: bool = True, dense_values: bool = True) -> H2Matrix:
    """Build a synthetic H^2 covariance matrix.

    points: optional n x dim array (original order) replacing the seeded uniform points.
    values: fill U, E, S and D (False gives only the structure).
    coupling_values: with values, also fill S (False leaves S_val None: for a handle that
    evaluates its coupling blocks from the kernel).
    dense_values: with values, also fill D (False leaves D_val None: for a handle whose dense
    blocks are generated on the device from the points).
    """
    lib = _load()
    h = ctypes.c_void_p()
    pts_in = None
    if points is not None:
        pts_in = np.ascontiguousarray(points, dtype=np.float64)
        assert pts_in.shape == (n, dim)
    rc = lib.h2gen_build(dim, n, m, p, float(eta), KERNELS[kernel], float(ell), ctypes.c_uint64(seed),
                         _p(pts_in) if pts_in is not None else None, ctypes.byref(h))
    if rc != 0:
        raise RuntimeError(f"h2gen_build failed with code {rc}")
    info = np.zeros(8, dtype=np.int64)
    lib.h2gen_info(h, _p(info))
    q, k, nS, nD, nDval, n_nodes, leaves = (int(v) for v in info[:7])
    A = H2Matrix(dim=dim, n=n, m=m, p=p, k=k, q=q, eta=eta, kernel=kernel, ell=ell, seed=seed,
                 points=np.empty((n, dim)), perm=np.empty(n, dtype=np.int64),
                 leaf_offset=np.empty(leaves + 1, dtype=np.int64),
                 S_rowptr=np.empty(n_nodes + 1, dtype=np.int32), S_colidx=np.empty(nS, dtype=np.int32),
                 D_rowptr=np.empty(leaves + 1, dtype=np.int32), D_colidx=np.empty(nD, dtype=np.int32),
                 D_valoff=np.empty(nD + 1, dtype=np.int64), _h=h)
    lib.h2gen_fill_structure(h, _p(A.points), _p(A.perm), _p(A.leaf_offset), _p(A.S_rowptr), _p(A.S_colidx),
                             _p(A.D_rowptr), _p(A.D_colidx), _p(A.D_valoff))
    if values:
        A.U = np.empty(n * k)
        A.E = np.empty(max(n_nodes - 1, 0) * k * k)
        A.S_val = np.empty(nS * k * k) if coupling_values else None
        A.D_val = np.empty(nDval) if dense_values else None
        lib.h2gen_fill_values(h, _p(A.U), _p(A.E), _p(A.S_val) if coupling_values else None,
                              _p(A.D_val) if dense_values else None)
    return A


# The workloads measured and tested (sizes and parameters of the covariance
# matrices in the paper's experiments, Sec. 4.6, with uniform random points).
CONFIGS = {
    # 2D, n=4096, exp(-r/0.1), m=32, 4x4 Chebyshev (k=16), eta=0.9
    "2d_n4096": dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=1),
    # 2D, n=2^20, exp(-r/0.1), m=64, k=16, eta=0.9
    "2d_n1M": dict(dim=2, n=1 << 20, m=64, p=4, eta=0.9, kernel="exp", ell=0.1, seed=2),
    # 2D, n=2^18 (a few GB, still far larger than L2): the profiling case
    "2d_n256k": dict(dim=2, n=1 << 18, m=64, p=4, eta=0.9, kernel="exp", ell=0.1, seed=4),
    # 3D, n=2^20, exp(-r/0.2), m=64, 4x4x4 Chebyshev (k=64), eta=0.9
    "3d_n1M": dict(dim=3, n=1 << 20, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=3),
    # the same 3D workload at n=2^19 (its FP64 arrays, about 91 GB, fit the host memory of one GPU node)
    "3d_n512k": dict(dim=3, n=1 << 19, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=3),
    # the same 3D workload at n=2^16 (1.6 GB of 16-bit coupling codes, far larger than L2): the 3D profiling case
    "3d_n64k": dict(dim=3, n=1 << 16, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=6),
    # 3D, n=2^22, Matern-3/2 length 0.1, m=64, k=64, eta=0.7
    "3d_n4M": dict(dim=3, n=1 << 22, m=64, p=4, eta=0.7, kernel="matern32", ell=0.1, seed=5),
}


def batch_workload(count: int = 256, lo: float = 12.0, hi: float = 17.0, seed: int = 40, nvs=(1, 4, 16)):
    """The batched workload: `count` independent 2D exponential-covariance matrices (length 0.1,
    leaf m=32, 4x4 Chebyshev rank k=16, eta=0.9), n_i = floor(2^u) with u ~ U(lo, hi)
    (log-uniform sizes) and nv_i drawn uniformly from `nvs`. Returns (generate kwargs, nv) pairs;
    matrix i uses seed 1000 * seed + i + 1."""
    u = uniform(seed, (count, 2))
    out = []
    for i in range(count):
        n = int(np.floor(2.0 ** (lo + (hi - lo) * u[i, 0])))
        nv = int(nvs[min(int(u[i, 1] * len(nvs)), len(nvs) - 1)])
        out.append((dict(dim=2, n=n, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=1000 * seed + i + 1), nv))
    return out
