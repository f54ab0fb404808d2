"""Plain FP64 tensor algebra used by the nnCANDELINC oracle.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module. The CUDA library never
calls it and shares no code with it.

Every routine follows a definition of the paper (arXiv 1909.07570) and is
written for a reader to check by eye, not for speed. Arrays are numpy float64
in C order; the first index of a d-way tensor is mode 1 of the paper.
"""
from __future__ import annotations

import numpy as np


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def mode_product(X, A, n):
    """The n-mode product X x_n A (Appendix A, Def. of n-mode multiplication).

    (X x_n A)[.., i, ..] = sum_l X[.., l, ..] * A[i, l], where the summed index
    sits at position ``n`` (0-based) and A has shape (M, N_n).
    """
    X = _f64(X)
    A = _f64(A)
    if A.ndim != 2 or A.shape[1] != X.shape[n]:
        raise ValueError(f"mode_product: A {A.shape} does not match mode {n} of X {X.shape}")
    Y = np.tensordot(A, X, axes=([1], [n]))  # the new mode comes first
    return np.moveaxis(Y, 0, n)


def unfold(X, n):
    """The mode-n unfolding (Appendix A, Def. of unfolding).

    The mode-n fibres become the columns of an N_n x prod(other N) matrix. The
    column order is the one of Sec. 3.1, m(j, k) = j + N_2 (k - 1) for mode 1:
    the first remaining index varies fastest.
    """
    X = _f64(X)
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def fold(M, n, shape):
    """Inverse of :func:`unfold`: put the columns of M back as mode-n fibres."""
    M = _f64(M)
    rest = [s for i, s in enumerate(shape) if i != n]
    T = np.reshape(M, [shape[n]] + rest, order="F")
    return np.moveaxis(T, 0, n)


def khatri_rao(mats):
    """Column-wise Kronecker product whose row index matches :func:`unfold`.

    For matrices [B_1, ..., B_p] (each with r columns) row
    i_1 + N_1 i_2 + N_1 N_2 i_3 + ... holds prod_t B_t[i_t, q]: the first
    matrix's index varies fastest, like the first remaining mode of an unfolding.
    """
    mats = [_f64(B) for B in mats]
    r = mats[0].shape[1]
    K = mats[0]
    for B in mats[1:]:
        if B.shape[1] != r:
            raise ValueError("khatri_rao: column counts differ")
        K = (B[:, None, :] * K[None, :, :]).reshape(-1, r)
    return K


def superdiagonal(r, d):
    """The d-way r x ... x r identity tensor I (Sec. 2, Eq. CPD:matrix-format)."""
    D = np.zeros((r,) * d)
    for q in range(r):
        D[(q,) * d] = 1.0
    return D


def tucker_reconstruct(G, F):
    """X_hat = G x_1 F^(1) x_2 F^(2) ... (Eq. TD:matrix-format)."""
    X = _f64(G)
    for n, Fn in enumerate(F):
        X = mode_product(X, Fn, n)
    return X


def cp_reconstruct(A):
    """X_hat = I x_1 A^(1) x_2 A^(2) ... (Eq. CPD:matrix-format with D = I)."""
    r = _f64(A[0]).shape[1]
    return tucker_reconstruct(superdiagonal(r, len(A)), A)


def frobenius(X):
    """||X||_F, the square root of the sum of squares (Sec. 4.1)."""
    X = _f64(X)
    return float(np.sqrt(np.sum(X * X)))
