"""Differentiation form on the GPU against the oracle: the adjoint of the
lifted loss (candelinc_lifted_grad), its torch.autograd wrapper, and the block
projected-gradient fit (candelinc_pg_fit).

Tolerances: FP64 1e-9 relative. FP32: a gradient entry is the difference of
A V B^T and MT B^T, so its error is FP32 rounding (with TF32x3 passes about
2^-17 of each contraction term) of those terms: 1e-5 of their magnitude; the
loss to 1e-5 of the magnitude of its terms (1/2 ||X||^2, <X, X_hat> and
1/2 ||X_hat||^2, the FP64 sums of FP32 products); fitted relative errors
sqrt(2 L)/||X|| to 1e-5 of max(1, value) as in the nnTD parity.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import autograd as nag
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu

SHAPES = [((37, 29, 24), (5, 6, 7), 4),      # TF32x3 passes (N3 % 4 == 0)
          ((23, 17, 30), (4, 3, 5), 3),      # N3 % 4 != 0: SIMT passes
          ((12, 10, 9, 16), (3, 4, 2, 5), 3),
          ((9, 14, 11, 8), (6, 2, 5, 3), 5),
          # TF32x3 passes over X viewed as N1 x N2 N3 x N4 with N2 N3 a
          # multiple of the 128-row tile, and ragged ranks
          ((6, 5, 128, 12), (3, 4, 5, 6), 3),
          ((4, 3, 256, 8), (3, 2, 24, 4), 2)]


def _problem(dims, m, r, seed):
    X, _, F0, _, B0 = inputs.small_problem(dims, 3, m, r, seed=seed)
    return X, F0, B0


def _dev(arrs, dt):
    return [torch.tensor(a, dtype=dt, device="cuda") for a in arrs]


def _term_scale(X, F, B, n):
    A = orc.lift(F, B)
    MT, V = orc.lifted_block_terms(X, A, n)
    return max(np.abs(A[n] @ V @ B[n].T).max(), np.abs(MT @ B[n].T).max(),
               np.abs(F[n].T @ (A[n] @ V)).max(), np.abs(F[n].T @ MT).max())


@pytest.mark.parametrize("dims,m,r", SHAPES)
def test_lifted_grad_fp64_matches_oracle(dims, m, r):
    X, F0, B0 = _problem(dims, m, r, 41)
    gFo, gBo = orc.lifted_loss_grad(X, F0, B0)
    Lo = orc.lifted_loss(X, F0, B0)
    Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    loss, gF, gB = native.candelinc_lifted_grad(Xd, _dev(F0, torch.float64), _dev(B0, torch.float64))
    assert loss == pytest.approx(Lo, rel=1e-9)
    for n in range(len(dims)):
        np.testing.assert_allclose(gF[n].cpu().numpy(), gFo[n], rtol=1e-9,
                                   atol=1e-12 * np.abs(gFo[n]).max())
        np.testing.assert_allclose(gB[n].cpu().numpy(), gBo[n], rtol=1e-9,
                                   atol=1e-12 * np.abs(gBo[n]).max())
    loss_only, none_f, none_b = native.candelinc_lifted_grad(
        Xd, _dev(F0, torch.float64), _dev(B0, torch.float64), grads=False)
    assert none_f is None and none_b is None
    assert loss_only == pytest.approx(Lo, rel=1e-9)


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
@pytest.mark.parametrize("dims,m,r", SHAPES)
def test_lifted_grad_fp32_matches_oracle(dims, m, r, precision):
    X, F0, B0 = _problem(dims, m, r, 43)
    X32 = X.astype(np.float32).astype(np.float64)
    F32 = [f.astype(np.float32).astype(np.float64) for f in F0]
    B32 = [b.astype(np.float32).astype(np.float64) for b in B0]
    gFo, gBo = orc.lifted_loss_grad(X32, F32, B32)
    Lo = orc.lifted_loss(X32, F32, B32)
    loss, gF, gB = native.candelinc_lifted_grad(
        torch.tensor(X32, dtype=torch.float32, device="cuda"), _dev(F32, torch.float32),
        _dev(B32, torch.float32), precision=precision)
    Xh = orc.cp_reconstruct(orc.lift(F32, B32))
    terms = 0.5 * np.sum(X32 * X32) + abs(np.sum(X32 * Xh)) + 0.5 * np.sum(Xh * Xh)
    assert abs(loss - Lo) <= 1e-5 * terms
    for n in range(len(dims)):
        sc = _term_scale(X32, F32, B32, n)
        assert np.abs(gF[n].double().cpu().numpy() - gFo[n]).max() <= 1e-5 * sc
        assert np.abs(gB[n].double().cpu().numpy() - gBo[n]).max() <= 1e-5 * sc


def test_autograd_function_fp64_against_central_differences():
    dims, m, r = (8, 7, 6, 4), (3, 2, 3, 2), 2
    X, F0, B0 = _problem(dims, m, r, 47)
    Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    F = [t.requires_grad_() for t in _dev(F0, torch.float64)]
    B = [t.requires_grad_() for t in _dev(B0, torch.float64)]
    L = nag.lifted_loss(Xd, F, B)
    (2.0 * L).backward()
    gFo, gBo = orc.lifted_loss_grad(X, F0, B0)
    for n in range(4):
        np.testing.assert_allclose(F[n].grad.cpu().numpy(), 2.0 * gFo[n], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(B[n].grad.cpu().numpy(), 2.0 * gBo[n], rtol=1e-9, atol=1e-12)
    # Central differences (h = 1e-3) of the library's own loss on sampled entries.
    rng = np.random.default_rng(3)
    h = 1e-3
    with torch.no_grad():
        for P, G in [(F[0], F[0].grad), (B[2], B[2].grad), (F[3], F[3].grad)]:
            for _ in range(4):
                idx = tuple(int(rng.integers(s)) for s in P.shape)
                old = P[idx].item()
                P[idx] = old + h
                lp = nag.lifted_loss(Xd, F, B).item()
                P[idx] = old - h
                lm = nag.lifted_loss(Xd, F, B).item()
                P[idx] = old
                assert (lp - lm) / (2 * h) * 2.0 == pytest.approx(G[idx].item(), rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("dims,m,r", SHAPES)
def test_pg_fit_fp64_matches_oracle(dims, m, r):
    X, F0, B0 = _problem(dims, m, r, 53)
    Fo, Bo, tro = orc.lifted_pg_fit(X, F0, B0, 6)
    F = _dev(F0, torch.float64)
    B = _dev(B0, torch.float64)
    loss, tr = native.candelinc_pg_fit(torch.tensor(X, dtype=torch.float64, device="cuda"), F, B, 6)
    np.testing.assert_allclose(tr.cpu().numpy(), tro, rtol=1e-9)
    assert loss == pytest.approx(tro[-1], rel=1e-9)
    for a, b in zip(F + B, Fo + Bo):
        np.testing.assert_allclose(a.cpu().numpy(), b, rtol=1e-8, atol=1e-11 * np.abs(b).max())


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
@pytest.mark.parametrize("dims,m,r", [((40, 36, 32), (6, 5, 7), 4),
                                      ((6, 5, 128, 12), (3, 4, 5, 6), 3)])
def test_pg_fit_fp32_trace_matches_oracle_and_descends(precision, dims, m, r):
    X, F0, B0 = _problem(dims, m, r, 59)
    X32 = X.astype(np.float32).astype(np.float64)
    F32 = [f.astype(np.float32).astype(np.float64) for f in F0]
    B32 = [b.astype(np.float32).astype(np.float64) for b in B0]
    _, _, tro = orc.lifted_pg_fit(X32, F32, B32, 30)
    F = _dev(F32, torch.float32)
    B = _dev(B32, torch.float32)
    _, tr = native.candelinc_pg_fit(torch.tensor(X32, dtype=torch.float32, device="cuda"), F, B, 30,
                                    precision=precision)
    tr = tr.cpu().numpy()
    xn = np.sqrt(np.sum(X32 * X32))
    rel, relo = np.sqrt(2 * np.maximum(tr, 0)) / xn, np.sqrt(2 * tro) / xn
    assert np.all(np.abs(rel - relo) <= 1e-5 * np.maximum(1.0, relo))
    assert np.all(np.diff(tr) <= 1e-6 * tr[:-1])
    assert all((f >= 0).all() for f in F + B)


def test_pg_fit_full_size_cp12_128x128x128x64():
    # The 4-way workload at full size in the launch configuration the benchmark
    # would use; the oracle runs the same two steps in FP64.
    w = inputs.WORKLOADS["cp12_128x128x128x64_m24_fp32"]
    X, _, F0, _, B0 = inputs.make_problem(w)
    X32 = X.astype(np.float32)
    F32 = [f.astype(np.float32) for f in F0]
    B32 = [b.astype(np.float32) for b in B0]
    F = _dev(F32, torch.float32)
    B = _dev(B32, torch.float32)
    _, tr = native.candelinc_pg_fit(torch.tensor(X32, device="cuda"), F, B, 2)
    X64 = X32.astype(np.float64)
    _, _, tro = orc.lifted_pg_fit(X64, [f.astype(np.float64) for f in F32],
                                  [b.astype(np.float64) for b in B32], 2)
    xn = np.sqrt(np.sum(X64 * X64))
    rel, relo = np.sqrt(2 * np.maximum(tr.cpu().numpy(), 0)) / xn, np.sqrt(2 * tro) / xn
    assert np.all(np.abs(rel - relo) <= 1e-5 * np.maximum(1.0, relo))


def test_lifted_entries_reject_bad_input():
    X = torch.rand(5, 6, 7, device="cuda")
    F = [torch.rand(n, 2, device="cuda") for n in (5, 6, 7)]
    B = [torch.rand(2, 3, device="cuda") for _ in range(3)]
    with pytest.raises(native.NncError) as ei:
        native.candelinc_lifted_grad(X, F, B, precision="bf16")
    assert ei.value.status == -6
    with pytest.raises(native.NncError):
        native.candelinc_pg_fit(X, F, B, -1)
    Xbad = X.clone()
    Xbad[0, 0, 0] = float("nan")
    with pytest.raises(native.NncError) as ei:
        native.candelinc_lifted_grad(Xbad, F, B)
    assert ei.value.status == -3
    loss, tr = native.candelinc_pg_fit(X, F, B, 0)
    assert np.isnan(loss) and tr.numel() == 0
