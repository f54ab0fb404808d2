"""Alg. 2 on the GPU against the oracle: nnCPD of X (nncp_tensor_fit), the MU
NMF of a CP factor (nmf_fit) and the composition (candelinc_alg2).

Tolerances: FP64 1e-9 relative on the traces and 1e-8 on the factors (MU
sweeps amplify rounding mildly). FP32 relative errors within 1e-5 of the
oracle: the final error and the exact trace checkpoints come from an explicit
FP64 pass over X. The identity trace (no checkpoints) is compared within 1e-5
plus the cancellation of the residual identity: ||X - X_hat||^2 = ||X||^2 -
2 <MT, A> + sum(V .* A^T A) with FP32-accurate terms (relative error eps,
about 2e-6 for the TF32x3 passes) has an absolute error of eps ||X||^2, so the
relative error rel = ||X - X_hat|| / ||X|| is off by up to eps / (2 rel).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu


def _dev(arrs, dt):
    return [torch.tensor(a, dtype=dt, device="cuda") for a in arrs]


def _init(dims, r, seed):
    rng = np.random.default_rng(seed)
    return [1.0 - rng.random((n, r)) for n in dims]


@pytest.mark.parametrize("dims,r", [((30, 25, 28), 4), ((23, 17, 30), 5), ((12, 10, 9, 16), 3)])
def test_nncp_tensor_fit_fp64_matches_oracle(dims, r):
    X, _, _, _, _ = inputs.small_problem(dims, r, (2,) * len(dims), 2, seed=61)
    A0 = _init(dims, r, 62)
    Ao, tro = orc.nncp_fit(X, A0, 8)
    A = _dev(A0, torch.float64)
    err, tr = native.nncp_tensor_fit(torch.tensor(X, device="cuda"), A, 8)
    np.testing.assert_allclose(tr.cpu().numpy(), tro, rtol=1e-9)
    assert err == pytest.approx(tro[-1], rel=1e-9)
    for a, b in zip(A, Ao):
        np.testing.assert_allclose(a.cpu().numpy(), b, rtol=1e-8, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
@pytest.mark.parametrize("dims,r", [((48, 40, 36), 6), ((12, 10, 9, 16), 3), ((4, 3, 128, 8), 3)])
def test_nncp_tensor_fit_fp32_trace_matches_oracle(dims, r, precision):
    # With exact checkpoints at every sweep the trace is the explicit FP64
    # residual of each iterate: within the plain FP32 bound of the oracle, as
    # is the final error (always explicit). The identity trace (no
    # checkpoints) carries the identity's cancellation, eps / (2 rel).
    X, _, _, _, _ = inputs.small_problem(dims, r, (2,) * len(dims), 2, seed=63)
    X32 = X.astype(np.float32).astype(np.float64)
    A0 = [a.astype(np.float32).astype(np.float64) for a in _init(dims, r, 64)]
    _, tro = orc.nncp_fit(X32, A0, 40)
    Xd = torch.tensor(X32, dtype=torch.float32, device="cuda")
    A = _dev(A0, torch.float32)
    err, tr = native.nncp_tensor_fit(Xd, A, 40, precision=precision, exact_every=1)
    assert np.abs(tr.cpu().numpy() - tro).max() <= 1e-5
    assert abs(err - tro[-1]) <= 1e-5
    assert all((a >= 0).all() for a in A)
    A = _dev(A0, torch.float32)
    err2, tr2 = native.nncp_tensor_fit(Xd, A, 40, precision=precision)
    assert err2 == err  # the same iterates, the same explicit final pass
    assert np.all(np.abs(tr2.cpu().numpy() - tro) <= 1e-5 + 2e-6 / (2 * tro))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 1e-5)])
def test_nmf_fit_matches_oracle(dtype, tol):
    rng = np.random.default_rng(65)
    A = rng.random((200, 12))
    F0, B0 = 1 - rng.random((200, 5)), 1 - rng.random((5, 12))
    if dtype == torch.float32:
        A, F0, B0 = (x.astype(np.float32).astype(np.float64) for x in (A, F0, B0))
    Fo, Bo, tro = orc.nmf_fit(A, F0, B0, 50)
    F, B = torch.tensor(F0, dtype=dtype, device="cuda"), torch.tensor(B0, dtype=dtype, device="cuda")
    err, tr = native.nmf_fit(torch.tensor(A, dtype=dtype, device="cuda"), F, B, 50)
    assert np.abs(tr.cpu().numpy() - tro).max() <= tol * max(1.0, tro.max())
    if dtype == torch.float64:
        np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(B.cpu().numpy(), Bo, rtol=1e-8, atol=1e-12)


def test_alg2_end_to_end_fp64_matches_oracle():
    dims, m, r = (20, 18, 16), (3, 4, 3), 3
    X, _, _, _, _ = inputs.small_problem(dims, 3, m, r, seed=67)
    rng = np.random.default_rng(68)
    A0 = [1 - rng.random((n, r)) for n in dims]
    F0 = [1 - rng.random((n, k)) for n, k in zip(dims, m)]
    B0 = [1 - rng.random((k, r)) for k in m]
    Ao, Fo, Bo, cpt, nmft = orc.alg2_fit(X, A0, F0, B0, 30, 40)
    A, F, B = _dev(A0, torch.float64), _dev(F0, torch.float64), _dev(B0, torch.float64)
    cp_err, nmf_errs = native.candelinc_alg2(torch.tensor(X, device="cuda"), A, F, B, 30, 40)
    assert cp_err == pytest.approx(cpt[-1], rel=1e-9)
    np.testing.assert_allclose(nmf_errs, [t[-1] for t in nmft], rtol=1e-8)
    for a, b in zip(A + F + B, Ao + Fo + Bo):
        np.testing.assert_allclose(a.cpu().numpy(), b, rtol=1e-7, atol=1e-11 * np.abs(b).max())


def test_alg2_entries_reject_bad_input():
    X = torch.rand(6, 5, 4, device="cuda")
    A = [torch.rand(n, 3, device="cuda") for n in (6, 5, 4)]
    with pytest.raises(native.NncError) as ei:
        native.nncp_tensor_fit(X, A, 3, precision="bf16")
    assert ei.value.status == -6
    with pytest.raises(native.NncError):
        native.nncp_tensor_fit(X, A, -1)
    err, tr = native.nncp_tensor_fit(X, A, 0)
    assert np.isnan(err) and tr.numel() == 0
