"""FP64 CPU oracle of the nnCANDELINC hot path (Alg. 1 of arXiv 1909.07570).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module; the CUDA library shares no
code with it and never calls it.

What it computes, in the paper's notation (X is d-way, N_1 x ... x N_d):

* nnTD of X with multirank m (Alg. 1, first step; model Eq. TD:matrix-format,
  nonnegative Tucker of Sec. 3),
* nnCPD of the core G with rank r (Alg. 1, second step; model Eq. npd),
* the lift A^(i) = F^(i) B^(i) (the substitution in the proof of Lemma
  "rank and min exists", Sec. 2.1), whose model I x_i A^(i) is the
  nnCANDELINC objective of Eq. nnCANDELINC (Sec. 4),
* the relative reconstruction error of Sec. 4.1,
* the gradient of the lifted loss 1/2 ||X - I x_i F^(i) B^(i)||_F^2 and a
  block projected-gradient fit of it (the differentiation form),
* Alg. 2: nnCPD of X followed by an NMF of every CP factor.

The paper names the problem and the packages it called, not their update
rules. The rules here are the multiplicative updates (MU) obtained by splitting
each block gradient of f = 1/2 ||X - X_hat||^2 into its positive part (the
denominator) and its negative part (the numerator); the gradients follow from
the unfolding identity Eq. unfolding:property. The order within one sweep is
Gauss-Seidel: F^(1), ..., F^(d), then G (nnTD); B^(1), ..., B^(d) (nnCPD).
Every denominator is guarded by max(., eps) and every update is projected with
max(., 0); the projection is a no-op in exact arithmetic.
"""
from __future__ import annotations

import itertools

import numpy as np

from .tensor_algebra import (
    cp_reconstruct,
    frobenius,
    khatri_rao,
    mode_product,
    tucker_reconstruct,
    unfold,
)

DEFAULT_EPS = 1e-12


def _f64(a):
    return np.array(a, dtype=np.float64, copy=True)


# ---------------------------------------------------------------------------
# nnTD (Alg. 1, step 1)
# ---------------------------------------------------------------------------

def ntd_factor_terms(X, F, G, n):
    """Numerator and denominator of the F^(n) update.

    With X_hat = G x_k F^(k), Eq. unfolding:property gives
    unfold_n(X_hat) = F^(n) unfold_n(G x_{k!=n} F^(k)), so the gradient of
    f wrt F^(n) is Den - Num with
      Num = unfold_n(X x_{k!=n} F^(k)T) unfold_n(G)^T              (N_n x m_n)
      Den = F^(n) unfold_n(G x_{k!=n} F^(k)T F^(k)) unfold_n(G)^T   (N_n x m_n)
    """
    d = X.ndim
    Z = X
    W = G
    for k in range(d):
        if k == n:
            continue
        Z = mode_product(Z, F[k].T, k)
        W = mode_product(W, F[k].T @ F[k], k)
    Gn = unfold(G, n)
    num = unfold(Z, n) @ Gn.T
    den = F[n] @ (unfold(W, n) @ Gn.T)
    return num, den


def ntd_core_terms(X, F, G):
    """Numerator and denominator of the core update.

    The gradient of f wrt G is Den - Num with
      Num = M = X x_1 F^(1)T x_2 ... x_d F^(d)T
      Den = G x_1 F^(1)T F^(1) x_2 ... x_d F^(d)T F^(d)
    """
    M = X
    D = G
    for k in range(X.ndim):
        M = mode_product(M, F[k].T, k)
        D = mode_product(D, F[k].T @ F[k], k)
    return M, D


def mu_step(theta, num, den, eps):
    """theta <- max(theta * num / max(den, eps), 0), elementwise."""
    return np.maximum(theta * num / np.maximum(den, eps), 0.0)


def residual_sq_identity(x_norm_sq, M, G, F):
    """||X - G x_k F^(k)||^2 = ||X||^2 - 2<M, G> + <G, G x_k F^(k)T F^(k)>.

    M = X x_k F^(k)T. This expands the squared Frobenius norm of Sec. 4.1 and
    needs only core-sized arrays once M is known.
    """
    D = G
    for k in range(G.ndim):
        D = mode_product(D, F[k].T @ F[k], k)
    return x_norm_sq - 2.0 * float(np.sum(M * G)) + float(np.sum(G * D))


def ntd_sweep(X, F, G, eps=DEFAULT_EPS):
    """One Gauss-Seidel MU sweep: F^(1), ..., F^(d), then G.

    Returns (F, G, M) where M = X x_k F^(k)T was the core numerator; M is
    reused by the caller for the residual identity.
    """
    F = [_f64(Fn) for Fn in F]
    G = _f64(G)
    for n in range(X.ndim):
        num, den = ntd_factor_terms(X, F, G, n)
        F[n] = mu_step(F[n], num, den, eps)
    M, D = ntd_core_terms(X, F, G)
    G = mu_step(G, M, D, eps)
    return F, G, M


def ntd_fit(X, F0, G0, iters, eps=DEFAULT_EPS):
    """nnTD by ``iters`` MU sweeps from the given initial factors and core.

    Returns (F, G, trace): trace[t] is the relative error after sweep t,
    evaluated with :func:`residual_sq_identity`.
    """
    X = _f64(X)
    F = [_f64(Fn) for Fn in F0]
    G = _f64(G0)
    x2 = float(np.sum(X * X))
    trace = []
    for _ in range(iters):
        F, G, M = ntd_sweep(X, F, G, eps)
        r2 = residual_sq_identity(x2, M, G, F)
        trace.append(np.sqrt(max(r2, 0.0) / x2))
    return F, G, np.array(trace)


def rel_err_tucker(X, G, F):
    """Relative reconstruction error ||X - G x_k F^(k)||_F / ||X||_F (Sec. 4.1)."""
    X = _f64(X)
    return frobenius(X - tucker_reconstruct(G, F)) / frobenius(X)


# ---------------------------------------------------------------------------
# nnCPD of the core (Alg. 1, step 2)
# ---------------------------------------------------------------------------

def nncp_terms(G, B, n):
    """Numerator and denominator of the B^(n) update for 1/2 ||G - I x_k B^(k)||^2.

    unfold_n(I x_k B^(k)) = B^(n) KR_{k!=n}(B^(k))^T (Eq. unfolding:property
    with a superdiagonal core), so the gradient is Den - Num with
      Num = unfold_n(G) KR_{k!=n}(B^(k))
      Den = B^(n) (Hadamard product over k!=n of B^(k)T B^(k))
    """
    others = [k for k in range(G.ndim) if k != n]
    num = unfold(G, n) @ khatri_rao([B[k] for k in others])
    V = np.ones((B[n].shape[1],) * 2)
    for k in others:
        V = V * (B[k].T @ B[k])
    den = B[n] @ V
    return num, den


def nncp_sweep(G, B, eps=DEFAULT_EPS):
    """One Gauss-Seidel MU sweep over B^(1), ..., B^(d)."""
    B = [_f64(Bn) for Bn in B]
    for n in range(G.ndim):
        num, den = nncp_terms(G, B, n)
        B[n] = mu_step(B[n], num, den, eps)
    return B


def nncp_fit(G, B0, iters, eps=DEFAULT_EPS):
    """nnCPD of G by ``iters`` MU sweeps. Returns (B, trace of relative errors)."""
    G = _f64(G)
    B = [_f64(Bn) for Bn in B0]
    g = frobenius(G)
    trace = []
    for _ in range(iters):
        B = nncp_sweep(G, B, eps)
        trace.append(frobenius(G - cp_reconstruct(B)) / g)
    return B, np.array(trace)


def rel_err_cp(X, A):
    """Relative error ||X - I x_k A^(k)||_F / ||X||_F of a CP model (Sec. 4.1)."""
    X = _f64(X)
    return frobenius(X - cp_reconstruct(A)) / frobenius(X)


# ---------------------------------------------------------------------------
# Lift, scoring and the gradient of the lifted loss
# ---------------------------------------------------------------------------

def lift(F, B):
    """A^(i) = F^(i) B^(i): the CPD of the core substituted into the Tucker
    model (proof of Lemma "rank and min exists", Sec. 2.1)."""
    return [_f64(Fn) @ _f64(Bn) for Fn, Bn in zip(F, B)]


def congruence_matrix(A, A_hat):
    """cong(q, q') = prod_i cos(a^(i)_q, a_hat^(i)_q') (Sec. 4.1)."""
    r = A[0].shape[1]
    C = np.ones((r, A_hat[0].shape[1]))
    for An, Bn in zip(A, A_hat):
        An = _f64(An)
        Bn = _f64(Bn)
        na = np.linalg.norm(An, axis=0)
        nb = np.linalg.norm(Bn, axis=0)
        C = C * ((An.T @ Bn) / np.outer(na, nb))
    return C


def mean_congruence(A, A_hat):
    """Mean congruence after the permutation of A_hat's components that
    maximises it (Sec. 4.1). Exhaustive search over permutations: fine for the
    r <= 8 of the tests."""
    C = congruence_matrix(A, A_hat)
    r = C.shape[0]
    best = -np.inf
    for perm in itertools.permutations(range(r)):
        best = max(best, float(np.mean(C[np.arange(r), perm])))
    return best


def lifted_loss(X, F, B):
    """L = 1/2 ||X - I x_i F^(i) B^(i)||_F^2, the objective of Eq. nnCANDELINC."""
    R = _f64(X) - cp_reconstruct(lift(F, B))
    return 0.5 * float(np.sum(R * R))


def lifted_loss_grad(X, F, B):
    """Gradients of :func:`lifted_loss` wrt every F^(n) and B^(n).

    With A^(k) = F^(k) B^(k) and unfold_n(I x_k A^(k)) = A^(n) KR_{k!=n}(A^(k))^T,
      dL/dA^(n) = A^(n) V_n - unfold_n(X) KR_{k!=n}(A^(k)),
      V_n = Hadamard product over k!=n of A^(k)T A^(k),
    and by the chain rule dL/dF^(n) = dL/dA^(n) B^(n)T, dL/dB^(n) = F^(n)T dL/dA^(n).
    """
    X = _f64(X)
    A = lift(F, B)
    r = A[0].shape[1]
    gF, gB = [], []
    for n in range(X.ndim):
        others = [k for k in range(X.ndim) if k != n]
        V = np.ones((r, r))
        for k in others:
            V = V * (A[k].T @ A[k])
        gA = A[n] @ V - unfold(X, n) @ khatri_rao([A[k] for k in others])
        gF.append(gA @ _f64(B[n]).T)
        gB.append(_f64(F[n]).T @ gA)
    return gF, gB


# ---------------------------------------------------------------------------
# Projected-gradient fit of the lifted loss (differentiation form)
# ---------------------------------------------------------------------------
# The paper minimises Eq. nnCANDELINC through its two-stage Alg. 1 and gives no
# first-order method on the lifted loss itself. The reading used here (a
# builder's choice): block-coordinate projected gradient over the blocks
# F^(1), B^(1), F^(2), B^(2), ..., each step of length 1 / L_block, with
# L_block the largest eigenvalue of the block's Hessian estimated by
# POWER_ITERS power iterations. With the other blocks fixed each block problem
# is a convex quadratic, so a step of length in (0, 2 / lambda_max) never
# increases the loss.

POWER_ITERS = 30


def power_iteration_lmax(H, iters=POWER_ITERS):
    """Largest eigenvalue of a symmetric PSD matrix H: ``iters`` power
    iterations from the normalised all-ones vector, then the Rayleigh quotient
    of the last iterate. Returns 0 if H maps the iterate to zero."""
    H = _f64(H)
    n = H.shape[0]
    v = np.ones(n) / np.sqrt(n)
    for _ in range(iters):
        w = H @ v
        nrm = float(np.sqrt(np.sum(w * w)))
        if nrm == 0.0:
            return 0.0
        v = w / nrm
    return float(v @ (H @ v))


def lifted_block_terms(X, A, n):
    """(MT, V) of mode n at the lifted point A^(k) = F^(k) B^(k):
      MT = unfold_n(X) KR_{k!=n}(A^(k)),   V = Hadamard_{k!=n} A^(k)T A^(k),
    so that dL/dA^(n) = A^(n) V - MT (see :func:`lifted_loss_grad`)."""
    others = [k for k in range(X.ndim) if k != n]
    r = A[0].shape[1]
    V = np.ones((r, r))
    for k in others:
        V = V * (A[k].T @ A[k])
    MT = unfold(_f64(X), n) @ khatri_rao([A[k] for k in others])
    return MT, V


def lifted_pg_step(X, F, B):
    """One block-coordinate projected-gradient step on the lifted loss.

    For n = 1..d: with MT, V of mode n (unchanged by this mode's blocks),
      F^(n) <- max(F^(n) - (A V - MT) B^(n)T / L_F, 0),  L_F = lmax(B^(n) V B^(n)T),
      B^(n) <- max(B^(n) - F^(n)T (A V - MT) / L_B, 0),  L_B = lmax(F^(n)T F^(n)) lmax(V),
    where A = F^(n) B^(n) is re-formed after the F^(n) update. A block whose
    L is 0 is left unchanged.
    """
    F = [_f64(Fn) for Fn in F]
    B = [_f64(Bn) for Bn in B]
    A = lift(F, B)
    for n in range(X.ndim):
        MT, V = lifted_block_terms(X, A, n)
        LF = power_iteration_lmax(B[n] @ V @ B[n].T)
        if LF > 0.0:
            gA = F[n] @ B[n] @ V - MT
            F[n] = np.maximum(F[n] - (gA @ B[n].T) / LF, 0.0)
        LB = power_iteration_lmax(F[n].T @ F[n]) * power_iteration_lmax(V)
        if LB > 0.0:
            gA = F[n] @ B[n] @ V - MT
            B[n] = np.maximum(B[n] - (F[n].T @ gA) / LB, 0.0)
        A[n] = F[n] @ B[n]
    return F, B


def lifted_pg_fit(X, F0, B0, steps):
    """``steps`` projected-gradient steps (:func:`lifted_pg_step`). Returns
    (F, B, trace) with trace[t] the lifted loss after step t."""
    F = [_f64(Fn) for Fn in F0]
    B = [_f64(Bn) for Bn in B0]
    trace = []
    for _ in range(steps):
        F, B = lifted_pg_step(X, F, B)
        trace.append(lifted_loss(X, F, B))
    return F, B, np.array(trace)


# ---------------------------------------------------------------------------
# Alg. 2: nnCPD of X, then an NMF of every CP factor
# ---------------------------------------------------------------------------
# Alg. 2 (Sec. 4.1) computes A^(i) <- nnCPD(X, r) and then
# F^(i), B^(i) <- NMF(A^(i), m_i). The nnCPD is :func:`nncp_fit` applied to X
# itself. The NMF, like every other update rule here, is the MU split of its
# gradient (Lee-Seung): for 1/2 ||A - F B||^2,
#   F <- max(F .* (A B^T) / max(F B B^T, eps), 0),
#   B <- max(B .* (F^T A) / max(F^T F B, eps), 0),   F first, then B.

def nmf_terms(A, F, B):
    """((num_F, den_F), (num_B, den_B)) of the NMF A ~ F B at (F, B); the
    gradients are den - num."""
    A, F, B = _f64(A), _f64(F), _f64(B)
    return (A @ B.T, F @ (B @ B.T)), (F.T @ A, (F.T @ F) @ B)


def nmf_fit(A, F0, B0, iters, eps=DEFAULT_EPS):
    """NMF of A (N x r) with rank m by ``iters`` MU iterations (F, then B).
    Returns (F, B, trace) with trace[t] = ||A - F B||_F / ||A||_F after t."""
    A = _f64(A)
    F, B = _f64(F0), _f64(B0)
    a = frobenius(A)
    trace = []
    for _ in range(iters):
        (nf, df), _ = nmf_terms(A, F, B)
        F = mu_step(F, nf, df, eps)
        _, (nb, db) = nmf_terms(A, F, B)
        B = mu_step(B, nb, db, eps)
        trace.append(frobenius(A - F @ B) / a)
    return F, B, np.array(trace)


def alg2_fit(X, A0, F0, B0, cp_iters, nmf_iters, eps=DEFAULT_EPS):
    """Alg. 2: A = nnCPD(X, r) from A0, then (F^(i), B^(i)) = NMF(A^(i), m_i)
    from (F0, B0). Returns (A, F, B, cp_trace, nmf_traces)."""
    A, cp_trace = nncp_fit(X, A0, cp_iters, eps)
    F, B, nmf_traces = [], [], []
    for n in range(len(A)):
        Fn, Bn, tr = nmf_fit(A[n], F0[n], B0[n], nmf_iters, eps)
        F.append(Fn)
        B.append(Bn)
        nmf_traces.append(tr)
    return A, F, B, cp_trace, nmf_traces
