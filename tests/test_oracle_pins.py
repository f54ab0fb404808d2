"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the worked
examples printed in the paper (tests/golden/), brute-force sums written from
the definitions, central finite differences of the objective, exact fixed
points built as in Thm. "canonical preserve rank", and invariants (monotone
objective, nonnegativity, column span). A dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle as orc
from _golden import load
from paper_1909_07570_gb300 import inputs

RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------------------
# n-mode product, unfolding, Khatri-Rao: brute force from the definitions
# ---------------------------------------------------------------------------

def _mode_product_loops(X, A, n):
    """Appendix A, Def. of n-mode multiplication, summed index by index."""
    out_shape = list(X.shape)
    out_shape[n] = A.shape[0]
    Y = np.zeros(out_shape)
    for idx in itertools.product(*[range(s) for s in out_shape]):
        s = 0.0
        for l in range(X.shape[n]):
            src = list(idx)
            src[n] = l
            s += X[tuple(src)] * A[idx[n], l]
        Y[idx] = s
    return Y


@pytest.mark.parametrize("shape", [(3, 4, 2), (2, 3, 4, 2)])
def test_mode_product_matches_definition(shape):
    X = RNG.standard_normal(shape)
    for n in range(len(shape)):
        A = RNG.standard_normal((3, shape[n]))
        np.testing.assert_allclose(orc.mode_product(X, A, n), _mode_product_loops(X, A, n),
                                   rtol=0, atol=1e-12)


def test_mode_products_commute_and_distribute():
    # Appendix A: (X x_i A) x_j B = (X x_j B) x_i A for i != j, and X x_i (AB) = (X x_i B) x_i A.
    X = RNG.standard_normal((3, 4, 5))
    A = RNG.standard_normal((2, 3))
    B = RNG.standard_normal((6, 4))
    np.testing.assert_allclose(orc.mode_product(orc.mode_product(X, A, 0), B, 1),
                               orc.mode_product(orc.mode_product(X, B, 1), A, 0), atol=1e-12)
    C = RNG.standard_normal((2, 7))
    D = RNG.standard_normal((7, 5))
    np.testing.assert_allclose(orc.mode_product(X, C @ D, 2),
                               orc.mode_product(orc.mode_product(X, D, 2), C, 2), atol=1e-12)


def test_unfold_column_order():
    # Sec. 3.1: column m(j, k) = j + N_2 (k - 1) of unfold_1 holds the fibre X[:, j, k];
    # likewise for modes 2 and 3 the first remaining index varies fastest.
    N1, N2, N3 = 3, 4, 5
    X = RNG.standard_normal((N1, N2, N3))
    U1, U2, U3 = (orc.unfold(X, n) for n in range(3))
    for i, j, k in itertools.product(range(N1), range(N2), range(N3)):
        assert U1[i, j + N2 * k] == X[i, j, k]
        assert U2[j, i + N1 * k] == X[i, j, k]
        assert U3[k, i + N1 * j] == X[i, j, k]
    for n in range(3):
        np.testing.assert_array_equal(orc.fold(orc.unfold(X, n), n, X.shape), X)


def test_khatri_rao_matches_unfolding_identity():
    # Eq. unfolding:property with a superdiagonal core: unfold_n(I x_k A^(k)) = A^(n) KR^T,
    # checked against a CP tensor summed term by term (Eq. pd).
    dims, r = (3, 4, 2, 3), 2
    A = [RNG.random((n, r)) for n in dims]
    X = np.zeros(dims)
    for q in range(r):
        for idx in itertools.product(*[range(s) for s in dims]):
            X[idx] += np.prod([A[t][idx[t], q] for t in range(len(dims))])
    np.testing.assert_allclose(orc.cp_reconstruct(A), X, atol=1e-13)
    for n in range(len(dims)):
        others = [k for k in range(len(dims)) if k != n]
        np.testing.assert_allclose(orc.unfold(X, n), A[n] @ orc.khatri_rao([A[k] for k in others]).T,
                                   atol=1e-13)


# ---------------------------------------------------------------------------
# Worked examples printed in the paper (exact integer arithmetic)
# ---------------------------------------------------------------------------

def test_example_not_in_cones():
    g = load("ex_not_in_cones.txt")
    X = orc.fold(g["unfold1_X"], 0, g["shape"]["X"])
    np.testing.assert_array_equal(orc.unfold(X, 1), g["unfold2_X"])
    np.testing.assert_array_equal(orc.unfold(X, 2), g["unfold3_X"])
    G = orc.fold(g["unfold1_G"], 0, g["shape"]["G"])
    np.testing.assert_array_equal(orc.tucker_reconstruct(G, [g["W1"], g["W2"], g["W3"]]), X)
    assert G.min() < 0  # the printed core has a negative entry: X is not in C1 x C2 x C3


def test_example_equal():
    g = load("ex_equal.txt")
    X = orc.cp_reconstruct([g["A1"], g["A2"], g["A3"]])
    np.testing.assert_array_equal(orc.unfold(X, 0), g["unfold1_X"])
    np.testing.assert_array_equal(g["F1"] @ g["unfold1_G"], g["unfold1_X"])
    G = orc.fold(g["unfold1_G"], 0, g["shape"]["G"])
    np.testing.assert_array_equal(orc.tucker_reconstruct(G, [g["F1"], np.eye(4), np.eye(4)]), X)
    ranks = [np.linalg.matrix_rank(orc.unfold(X, n)) for n in range(3)]
    assert ranks == list(g["unfold_ranks"].astype(int))


def test_example_cones_dne():
    g = load("ex_cones_dne.txt")
    X = orc.fold(g["unfold1_X"], 0, g["shape"]["X"])
    np.testing.assert_array_equal(orc.unfold(X, 1), g["unfold2_X"])
    np.testing.assert_array_equal(orc.unfold(X, 2), g["unfold3_X"])
    np.testing.assert_array_equal(g["W2"] @ g["H2"], g["unfold2_X"])
    np.testing.assert_array_equal(g["W"] @ g["unfold1_H"], g["unfold1_X"])
    H = orc.fold(g["unfold1_H"], 0, g["shape"]["H"])
    np.testing.assert_array_equal(orc.mode_product(H, g["W"], 0), X)
    np.testing.assert_array_equal(orc.unfold(H, 1), g["unfold2_H"])


def test_example_rank_one_with_rank_two_core():
    # Sec. 2.1: the 2x2x2 all-ones tensor equals a rank-2 core times the all-ones matrix in mode 1.
    G = orc.fold(np.array([[1.0, 0, 1, 0], [0, 1, 0, 1]]), 0, (2, 2, 2))
    np.testing.assert_array_equal(orc.mode_product(G, np.ones((2, 2)), 0), np.ones((2, 2, 2)))


def test_example_rank_of_V():
    # Appendix B, Example mrank_mrank+: rank(V) = 3 since v1 + v4 = v2 + v3.
    V = np.array([[1.0, 1, 0, 0], [1, 0, 1, 0], [0, 1, 0, 1], [0, 0, 1, 1]])
    assert np.linalg.matrix_rank(V) == 3
    np.testing.assert_array_equal(V[:, 0] + V[:, 3], V[:, 1] + V[:, 2])


# ---------------------------------------------------------------------------
# Multiplicative updates: gradients by central differences
# ---------------------------------------------------------------------------

def _tucker_loss(X, F, G):
    R = X - orc.tucker_reconstruct(G, F)
    return 0.5 * np.sum(R * R)


def _fd_grad(fun, P, h=1e-5):
    g = np.zeros_like(P)
    for idx in np.ndindex(P.shape):
        old = P[idx]
        P[idx] = old + h
        fp = fun()
        P[idx] = old - h
        fm = fun()
        P[idx] = old
        g[idx] = (fp - fm) / (2 * h)
    return g


@pytest.mark.parametrize("dims,m", [((4, 3, 5), (2, 3, 2)), ((3, 4, 2, 3), (2, 2, 2, 3))])
def test_ntd_terms_are_the_gradient(dims, m):
    X = RNG.random(dims)
    F = [RNG.random((n, k)) for n, k in zip(dims, m)]
    G = RNG.random(m)
    for n in range(len(dims)):
        num, den = orc.ntd_factor_terms(X, F, G, n)
        fd = _fd_grad(lambda: _tucker_loss(X, F, G), F[n])
        np.testing.assert_allclose(den - num, fd, rtol=1e-7, atol=1e-7)
        assert (num >= 0).all() and (den >= 0).all()
    M, D = orc.ntd_core_terms(X, F, G)
    fd = _fd_grad(lambda: _tucker_loss(X, F, G), G)
    np.testing.assert_allclose(D - M, fd, rtol=1e-7, atol=1e-7)


def test_nncp_terms_are_the_gradient():
    m, r = (3, 4, 2), 3
    G = RNG.random(m)
    B = [RNG.random((k, r)) for k in m]

    def loss():
        R = G - orc.cp_reconstruct(B)
        return 0.5 * np.sum(R * R)

    for n in range(3):
        num, den = orc.nncp_terms(G, B, n)
        np.testing.assert_allclose(den - num, _fd_grad(loss, B[n]), rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("dims,m,r", [((4, 3, 5), (2, 3, 2), 2), ((3, 3, 2, 4), (2, 2, 2, 3), 3)])
def test_lifted_loss_gradient(dims, m, r):
    X = RNG.random(dims)
    F = [RNG.random((n, k)) for n, k in zip(dims, m)]
    B = [RNG.random((k, r)) for k in m]
    gF, gB = orc.lifted_loss_grad(X, F, B)
    for n in range(len(dims)):
        np.testing.assert_allclose(gF[n], _fd_grad(lambda: orc.lifted_loss(X, F, B), F[n]),
                                   rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(gB[n], _fd_grad(lambda: orc.lifted_loss(X, F, B), B[n]),
                                   rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------------------
# Fixed points (Thm. "canonical preserve rank"), residual identity, invariants
# ---------------------------------------------------------------------------

def _canonical_solution(dims, kappa, r, seed):
    rng = np.random.default_rng(seed)
    W = [rng.random((n, k)) + 0.1 for n, k in zip(dims, kappa)]
    H = [rng.random((k, r)) + 0.1 for k in kappa]
    G = orc.cp_reconstruct(H)          # G = D x_i H^(i)
    X = orc.tucker_reconstruct(G, W)   # X = G x_i W^(i) = D x_i W^(i) H^(i)
    return X, W, H, G


def test_exact_canonical_tucker_is_a_fixed_point():
    X, W, H, G = _canonical_solution((9, 8, 7), (3, 4, 5), 5, 7)
    F1, G1, _ = orc.ntd_sweep(X, W, G)
    for a, b in zip(F1, W):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    np.testing.assert_allclose(G1, G, rtol=1e-12)
    B1 = orc.nncp_sweep(G, H)
    for a, b in zip(B1, H):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    A = orc.lift(W, H)
    assert orc.rel_err_cp(X, A) < 1e-14


def test_residual_identity_matches_brute_force():
    X, _, F0, G0, _ = inputs.small_problem((7, 6, 5), 3, (3, 3, 2), 3, seed=3)
    F, G, _ = orc.ntd_sweep(X, F0, G0)
    M, _ = orc.ntd_core_terms(X, F, G)
    x2 = np.sum(X * X)
    r2 = orc.residual_sq_identity(x2, M, G, F)
    brute = np.sum((X - orc.tucker_reconstruct(G, F)) ** 2)
    np.testing.assert_allclose(r2, brute, rtol=1e-10)


def test_ntd_fit_trace_is_the_relative_error_and_monotone():
    X, _, F0, G0, _ = inputs.small_problem((10, 9, 8), 3, (4, 4, 3), 3, seed=11, noise=0.05)
    F, G, trace = orc.ntd_fit(X, F0, G0, 60)
    np.testing.assert_allclose(trace[-1], orc.rel_err_tucker(X, G, F), rtol=1e-9)
    assert np.all(np.diff(trace) <= 1e-12 * trace[:-1])
    assert all((f >= 0).all() for f in F) and (G >= 0).all()


def test_nncp_fit_monotone_and_nonnegative():
    G = np.random.default_rng(5).random((4, 5, 3))
    B0 = inputs.initial_cp((4, 5, 3), 3, 9)
    B, trace = orc.nncp_fit(G, B0, 80)
    assert np.all(np.diff(trace) <= 1e-12 * trace[:-1])
    assert all((b >= 0).all() for b in B)


def test_lift_substitution_and_column_span():
    # Proof of Lemma "rank and min exists": (I x_i B^(i)) x_i F^(i) = I x_i (F^(i) B^(i)),
    # and by Prop. tdspaces every lifted factor lies in col(F^(i)).
    dims, m, r = (6, 5, 7), (3, 2, 4), 3
    F = [RNG.random((n, k)) for n, k in zip(dims, m)]
    B = [RNG.random((k, r)) for k in m]
    A = orc.lift(F, B)
    np.testing.assert_allclose(orc.tucker_reconstruct(orc.cp_reconstruct(B), F),
                               orc.cp_reconstruct(A), rtol=1e-12)
    for Fn, An in zip(F, A):
        P = Fn @ np.linalg.pinv(Fn)
        assert np.linalg.norm(An - P @ An) <= 1e-12 * np.linalg.norm(An)


def test_congruence_is_permutation_invariant():
    A = [RNG.random((n, 4)) for n in (5, 6, 7)]
    perm = [2, 0, 3, 1]
    A_hat = [a[:, perm] * 3.0 for a in A]
    assert orc.mean_congruence(A, A_hat) == pytest.approx(1.0, abs=1e-12)
    C = orc.congruence_matrix(A, A)
    for q in range(4):
        for p in range(4):
            expect = np.prod([A[i][:, q] @ A[i][:, p] / np.linalg.norm(A[i][:, q]) /
                              np.linalg.norm(A[i][:, p]) for i in range(3)])
            assert C[q, p] == pytest.approx(expect, rel=1e-12)


def test_congruence_closed_forms_and_best_assignment():
    # Columns orthonormal in every mode: a factor set's congruence with itself
    # is the identity. Rotating component q0 by theta within the plane of two
    # unit vectors (in each of the three modes) gives cong(q0, q0) = cos^3
    # theta, so the best mean is (r - 1 + cos^3 theta) / r (Sec. 4.1).
    r, theta, q0 = 5, 0.7, 2
    A = [np.linalg.qr(RNG.standard_normal((n, r + 1)))[0] for n in (8, 9, 10)]
    A_hat = [a[:, :r].copy() for a in A]
    for a_hat, a in zip(A_hat, A):
        a_hat[:, q0] = np.cos(theta) * a[:, q0] + np.sin(theta) * a[:, r]
    A = [a[:, :r] for a in A]
    np.testing.assert_allclose(orc.congruence_matrix(A, A), np.eye(r), atol=1e-12)
    C = orc.congruence_matrix(A, A_hat)
    assert C[q0, q0] == pytest.approx(np.cos(theta) ** 3, rel=1e-12)
    assert orc.mean_congruence(A, A_hat) == pytest.approx((r - 1 + np.cos(theta) ** 3) / r,
                                                          rel=1e-12)
    # The exhaustive search over permutations agrees with a linear assignment
    # solver on random nonnegative factors (the best permutation is unique).
    scipy_opt = pytest.importorskip("scipy.optimize")
    for seed in range(3):
        rng = np.random.default_rng(900 + seed)
        A = [rng.random((n, 7)) for n in (6, 7, 8)]
        A_hat = [rng.random((n, 7)) for n in (6, 7, 8)]
        C = orc.congruence_matrix(A, A_hat)
        rows, cols = scipy_opt.linear_sum_assignment(-C)
        assert orc.mean_congruence(A, A_hat) == pytest.approx(float(C[rows, cols].mean()),
                                                              rel=1e-12)


def test_recovery_of_a_planted_canonical_tucker():
    # Sec. 4.3 in miniature: noise-free planted rank-3 data, multirank above the
    # canonical one. A quality check of the whole Alg. 1 (MU is a local method),
    # not a tolerance gate.
    X, A, F0, G0, B0 = inputs.small_problem((12, 11, 10), 3, (4, 4, 4), 3, seed=21, noise=0.0)
    F, G, trace = orc.ntd_fit(X, F0, G0, 1000)
    assert trace[-1] < 1e-2
    B, cp_trace = orc.nncp_fit(G, B0, 300)
    assert cp_trace[-1] < cp_trace[0]
    A_hat = orc.lift(F, B)
    assert orc.rel_err_cp(X, A_hat) < 0.15
    assert orc.mean_congruence(A, A_hat) > 0.8


# ---------------------------------------------------------------------------
# Differentiation form: block projected gradient on the lifted loss
# ---------------------------------------------------------------------------

def test_power_iteration_lmax_against_eigendecomposition():
    # Closed form: a diagonal matrix; a rank-one matrix u u^T has lmax = |u|^2.
    assert orc.power_iteration_lmax(np.diag([1.0, 4.0, 2.5])) == pytest.approx(4.0, rel=1e-9)
    u = RNG.random(7)
    assert orc.power_iteration_lmax(np.outer(u, u)) == pytest.approx(u @ u, rel=1e-12)
    assert orc.power_iteration_lmax(np.zeros((3, 3))) == 0.0
    for n in (3, 12, 24):
        Q = RNG.random((40, n))
        H = Q.T @ Q  # nonnegative Gram: a dominant Perron eigenvalue
        assert orc.power_iteration_lmax(H) == pytest.approx(np.linalg.eigvalsh(H)[-1], rel=1e-10)


@pytest.mark.parametrize("dims,m,r", [((4, 3, 5), (2, 3, 2), 2), ((3, 3, 2, 4), (2, 2, 2, 3), 3)])
def test_lifted_block_terms_are_the_gradient_in_A(dims, m, r):
    # dL/dA^(n) = A^(n) V - MT, with L = 1/2 ||X - I x_k A^(k)||^2 by differences.
    X = RNG.random(dims)
    A = [RNG.random((n, r)) for n in dims]

    def loss():
        R = X - orc.cp_reconstruct(A)
        return 0.5 * np.sum(R * R)

    for n in range(len(dims)):
        MT, V = orc.lifted_block_terms(X, A, n)
        np.testing.assert_allclose(A[n] @ V - MT, _fd_grad(loss, A[n]), rtol=1e-6, atol=1e-7)


def test_lifted_pg_exact_lift_is_a_fixed_point():
    # X = I x_i F^(i) B^(i) exactly: every block gradient vanishes, so a step
    # changes nothing and the loss stays 0.
    dims, m, r = (6, 5, 7), (3, 4, 3), 3
    rng = np.random.default_rng(77)
    F = [rng.random((n, k)) + 0.1 for n, k in zip(dims, m)]
    B = [rng.random((k, r)) + 0.1 for k in m]
    X = orc.cp_reconstruct(orc.lift(F, B))
    F1, B1 = orc.lifted_pg_step(X, F, B)
    for a, b in zip(F1 + B1, F + B):
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13)
    assert orc.lifted_loss(X, F1, B1) < 1e-20 * np.sum(X * X)


@pytest.mark.parametrize("dims,m,r", [((9, 8, 7), (3, 4, 5), 4), ((6, 5, 4, 5), (3, 3, 2, 3), 3)])
def test_lifted_pg_monotone_and_nonnegative(dims, m, r):
    X, _, _, _, _ = inputs.small_problem(dims, 3, m, r, seed=31)
    rng = np.random.default_rng(5)
    F0 = [1.0 - rng.random((n, k)) for n, k in zip(dims, m)]
    B0 = [1.0 - rng.random((k, r)) for k in m]
    F, B, tr = orc.lifted_pg_fit(X, F0, B0, 40)
    l0 = orc.lifted_loss(X, F0, B0)
    assert tr[0] <= l0 * (1 + 1e-12)
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])
    assert tr[-1] < 0.5 * l0
    assert all((a >= 0).all() for a in F + B)


# ---------------------------------------------------------------------------
# Alg. 2: NMF of the CP factors
# ---------------------------------------------------------------------------

def test_nmf_terms_are_the_gradient():
    A = RNG.random((7, 4))
    F = RNG.random((7, 3))
    B = RNG.random((3, 4))

    def loss():
        R = A - F @ B
        return 0.5 * np.sum(R * R)

    (nf, df), (nb, db) = orc.nmf_terms(A, F, B)
    np.testing.assert_allclose(df - nf, _fd_grad(loss, F), rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(db - nb, _fd_grad(loss, B), rtol=1e-7, atol=1e-8)


def test_nmf_exact_factorisation_is_a_fixed_point_and_fit_is_monotone():
    rng = np.random.default_rng(91)
    F = rng.random((9, 3)) + 0.1
    B = rng.random((3, 5)) + 0.1
    F1, B1, tr = orc.nmf_fit(F @ B, F, B, 3)
    np.testing.assert_allclose(F1, F, rtol=1e-12)
    np.testing.assert_allclose(B1, B, rtol=1e-12)
    assert tr.max() < 1e-13
    A = rng.random((30, 6))
    F2, B2, tr = orc.nmf_fit(A, 1 - rng.random((30, 4)), 1 - rng.random((4, 6)), 60)
    assert np.all(np.diff(tr) <= 1e-12) and tr[-1] < tr[0]
    assert (F2 >= 0).all() and (B2 >= 0).all()


def test_alg2_on_a_planted_canonical_tensor():
    # X = I x_i W^(i) H^(i) with W^(i) H^(i) of rank r: Alg. 2's nnCPD fits X
    # and each NMF of a CP factor reaches a small residual (a quality check of
    # the composition; the pieces are pinned above).
    dims, kappa, r = (10, 9, 8), (3, 3, 3), 3
    rng = np.random.default_rng(123)
    W = [rng.random((n, k)) + 0.1 for n, k in zip(dims, kappa)]
    H = [rng.random((k, r)) + 0.1 for k in kappa]
    X = orc.cp_reconstruct(orc.lift(W, H))
    A0 = [1 - rng.random((n, r)) for n in dims]
    F0 = [1 - rng.random((n, k)) for n, k in zip(dims, kappa)]
    B0 = [1 - rng.random((k, r)) for k in kappa]
    A, F, B, cpt, nmft = orc.alg2_fit(X, A0, F0, B0, 300, 300)
    assert cpt[-1] < 0.05 and np.all(np.diff(cpt) <= 1e-12)
    assert all(t[-1] < 0.05 for t in nmft)
    assert orc.rel_err_cp(X, orc.lift(F, B)) < 0.1


def test_kruskal_rank_on_known_matrices():
    # Kruskal rank: the largest k with every k columns independent.
    assert inputs.kruskal_rank(np.eye(5)) == 5
    A = np.eye(4)[:, [0, 1, 2, 2]]               # a repeated column
    assert inputs.kruskal_rank(A) == 1
    B = np.c_[np.eye(3), np.zeros(3)]            # a zero column
    assert inputs.kruskal_rank(B) == 0
    C = np.array([[1.0, 0, 1], [0, 1, 1]])       # any 2 independent, 3 columns in R^2
    assert inputs.kruskal_rank(C) == 2


def test_paper_batch_problems_follow_the_recipe():
    # The Sec. 4.3 batch generator: rank-deficient planted factors F B with
    # kappa = (3, 4, 5), Kruskal ranks adding up to at least 2r + 2, X their
    # CP tensor, positive starts; the same seed gives the same batch.
    p = inputs.paper_batch_problems(3, N=12, seed=5)
    q = inputs.paper_batch_problems(3, N=12, seed=5)
    for a, b in zip(p, q):
        np.testing.assert_array_equal(a["X"], b["X"])
    for t in p:
        A = t["A_true"]
        assert [np.linalg.matrix_rank(a) for a in A] == [3, 4, 5]
        assert sum(inputs.kruskal_rank(a) for a in A) >= 2 * 5 + 2
        np.testing.assert_allclose(t["X"], np.einsum("iq,jq,kq->ijk", *A), rtol=1e-12)
        assert t["m"] == (3, 4, 5) and t["r"] == 5
        for key in ("F", "B", "A", "F2", "B2"):
            assert all((x > 0).all() for x in t[key])
        assert (t["G"] > 0).all() and t["G"].shape == (3, 4, 5)


# 4-way counterparts of the pins above (the d = 4 nnTD and residual on the GPU
# are checked against these oracle functions).

def test_exact_canonical_tucker_is_a_fixed_point_4way():
    X, W, H, G = _canonical_solution((7, 6, 5, 4), (3, 2, 4, 2), 4, 13)
    F1, G1, _ = orc.ntd_sweep(X, W, G)
    for a, b in zip(F1, W):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    np.testing.assert_allclose(G1, G, rtol=1e-12)
    assert orc.rel_err_cp(X, orc.lift(W, H)) < 1e-14
    assert orc.rel_err_tucker(X, G, W) < 1e-14


def test_residual_identity_matches_brute_force_4way():
    X, _, F0, G0, _ = inputs.small_problem((6, 5, 4, 7), 3, (3, 2, 2, 3), 3, seed=4)
    F, G, _ = orc.ntd_sweep(X, F0, G0)
    M, _ = orc.ntd_core_terms(X, F, G)
    r2 = orc.residual_sq_identity(np.sum(X * X), M, G, F)
    brute = np.sum((X - orc.tucker_reconstruct(G, F)) ** 2)
    np.testing.assert_allclose(r2, brute, rtol=1e-10)


def test_ntd_fit_trace_monotone_4way():
    X, _, F0, G0, _ = inputs.small_problem((8, 7, 6, 5), 3, (3, 3, 2, 2), 3, seed=12, noise=0.05)
    F, G, trace = orc.ntd_fit(X, F0, G0, 40)
    np.testing.assert_allclose(trace[-1], orc.rel_err_tucker(X, G, F), rtol=1e-9)
    assert np.all(np.diff(trace) <= 1e-12 * trace[:-1])
    assert all((f >= 0).all() for f in F) and (G >= 0).all()
