"""ORACLE (test infrastructure only): coupling blocks as the kernel at the interpolation points.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
this module; it shares nothing with the CUDA library.

The paper builds its matrices ab initio (Sec. 4.6, the experiments' setup): cluster bases by
Chebyshev interpolation, and every coupling block by evaluating the covariance kernel at the
interpolation points of its row and column clusters,

    S_ij[nu, mu] = K(xi_i^nu, xi_j^mu),

where the points of a cluster are the tensor grid of the first-kind Chebyshev nodes of its box
(index nu with dimension 0 slowest). K is the isotropic exponential kernel exp(-r / ell) of the
paper's experiments, or the Matern-3/2 kernel (1 + s) exp(-s), s = sqrt(3) r / ell. Plain FP64,
one block at a time, straight from that definition.
"""
from __future__ import annotations

import math

import numpy as np

KINDS = ("exp", "matern32")


def kernel_value(kind: str, r, ell: float):
    """K(r) for distance(s) r >= 0."""
    r = np.asarray(r, dtype=np.float64)
    if kind == "exp":
        return np.exp(-r / ell)
    if kind == "matern32":
        s = math.sqrt(3.0) * r / ell
        return (1.0 + s) * np.exp(-s)
    raise ValueError(f"kernel {kind!r} is not one of {KINDS}")


def tensor_digits(dim: int, p: int) -> np.ndarray:
    """(k, dim) digits of the tensor index: point nu has digit (nu // p^(dim-1-d)) % p in
    dimension d (dimension 0 slowest)."""
    nu = np.arange(p ** dim)
    return np.stack([(nu // p ** (dim - 1 - d)) % p for d in range(dim)], axis=1)


def tensor_points(cheb_node: np.ndarray) -> np.ndarray:
    """The k = p^dim interpolation points of one cluster, (k, dim), from its (dim, p) Chebyshev
    nodes per dimension."""
    dim, p = cheb_node.shape
    a = tensor_digits(dim, p)
    return np.stack([cheb_node[d, a[:, d]] for d in range(dim)], axis=1)


def coupling_blocks(cheb: np.ndarray, kind: str, ell: float, S_rowptr: np.ndarray, S_colidx: np.ndarray) -> np.ndarray:
    """All coupling blocks of the block-sparse rows (S_rowptr over all nodes in heap order,
    S_colidx the column node): block b is k x k column-major at b*k*k, entry (nu, mu) at
    nu + k*mu. cheb is (n_nodes, dim, p). One block row at a time."""
    n_nodes, dim, p = cheb.shape
    k = p ** dim
    a = tensor_digits(dim, p)
    pts = np.stack([cheb[:, d, a[:, d]] for d in range(dim)], axis=2)   # (n_nodes, k, dim)
    out = np.empty(int(S_rowptr[-1]) * k * k)
    for i in range(n_nodes):
        b0, b1 = int(S_rowptr[i]), int(S_rowptr[i + 1])
        if b1 == b0:
            continue
        J = np.asarray(S_colidx[b0:b1], dtype=np.int64)
        diff = pts[i][None, :, None, :] - pts[J][:, None, :, :]          # (block, nu, mu, dim)
        r = np.sqrt(np.sum(diff * diff, axis=3))
        out[b0 * k * k:b1 * k * k] = kernel_value(kind, r, ell).transpose(0, 2, 1).ravel()  # nu fastest
    return out
