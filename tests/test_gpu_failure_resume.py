"""Failure detection without a GPU fault, and resuming a fit from saved factors.

* The tensor-core pass kernel bounds every mbarrier wait; the self-test runs
  that wait on a barrier nothing arrives on, with a limit of about a
  millisecond, and must get NNC_ERR_TIMEOUT back with the context intact.
* A fit of 2k sweeps and a fit of k sweeps resumed from its own output for k
  more agree (the MU state is just the factors and the core).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu


def _dev(arrs, dtype):
    return [torch.tensor(a, dtype=dtype, device="cuda") for a in arrs]


def test_bounded_wait_gives_up_and_the_context_survives():
    assert native.nnc_wait_selftest(2_000_000) == -7
    assert native.nnc_wait_selftest(0) == -7
    # The context is still usable: a fit right after matches the oracle.
    X, _, F0, G0, _ = inputs.small_problem((12, 10, 8), 2, (3, 3, 3), 2, seed=3)
    F = _dev(F0, torch.float64)
    G = torch.tensor(G0, device="cuda")
    err, _ = native.ntd_fit(torch.tensor(X, device="cuda"), F, G, 5)
    Fo, Go, _ = orc.ntd_fit(X, F0, G0, 5)
    assert err == pytest.approx(orc.rel_err_tucker(X, Go, Fo), rel=1e-9)


@pytest.mark.parametrize("dtype,precision", [(torch.float64, "fp64"), (torch.float32, "fp32")])
def test_resumed_fit_matches_a_straight_fit(dtype, precision):
    X, _, F0, G0, _ = inputs.small_problem((40, 128, 36), 4, (5, 6, 7), 3, seed=17)
    Xd = torch.tensor(X, dtype=dtype, device="cuda")
    F1, G1 = _dev(F0, dtype), torch.tensor(G0, dtype=dtype, device="cuda")
    _, tr1 = native.ntd_fit(Xd, F1, G1, 40, precision=precision)
    F2, G2 = _dev(F0, dtype), torch.tensor(G0, dtype=dtype, device="cuda")
    _, tra = native.ntd_fit(Xd, F2, G2, 20, precision=precision)
    _, trb = native.ntd_fit(Xd, F2, G2, 20, precision=precision)  # resumed from F2, G2
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    for a, b in zip(F1 + [G1], F2 + [G2]):
        np.testing.assert_allclose(b.double().cpu().numpy(), a.double().cpu().numpy(),
                                   rtol=tol, atol=tol * float(a.abs().max()))
    tr = np.concatenate([tra.cpu().numpy(), trb.cpu().numpy()])
    np.testing.assert_allclose(tr, tr1.cpu().numpy(), rtol=tol, atol=tol)


def test_exact_checkpoints_are_exact_and_change_nothing_else():
    # exact_every = 5 over 23 sweeps: entries 4, 9, 14, 19 and 22 (the last)
    # come from an explicit FP64 pass and match the oracle far inside the FP32
    # bound; the fit itself is the same bits as without checkpoints.
    X, _, F0, G0, _ = inputs.small_problem((40, 128, 36), 4, (5, 6, 7), 3, seed=19, noise=0.0)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    X32 = X.astype(np.float32).astype(np.float64)
    Fo, Go, tro = orc.ntd_fit(X32, F0, G0, 23)
    runs = []
    for every in (0, 5):
        F = _dev(F0, torch.float32)
        G = torch.tensor(G0, dtype=torch.float32, device="cuda")
        _, tr = native.ntd_fit(Xd, F, G, 23, precision="fp32", exact_every=every)
        runs.append((F, G, tr.cpu().numpy()))
    (F0d, G0d, tr0), (F5, G5, tr5) = runs
    for a, b in zip(F0d + [G0d], F5 + [G5]):
        assert torch.equal(a, b)
    ck = [4, 9, 14, 19, 22]
    rest = [t for t in range(23) if t not in ck]
    np.testing.assert_array_equal(tr5[rest], tr0[rest])
    # The last checkpoint is the explicit residual of the final model.
    rn, xn = native.recon_residual(Xd, F5, G5)
    assert tr5[22] == pytest.approx(rn / xn, rel=1e-12)
    assert np.abs(tr5[ck] - tro[ck]).max() <= 1e-6
    assert np.abs(tr0 - tro).max() <= 1e-5


def test_refinement_trigger_switches_early_and_stays_within_bf16_bound():
    X, _, F0, G0, _ = inputs.small_problem((64, 128, 48), 4, (6, 6, 6), 3, seed=29, noise=0.01)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    X32 = X.astype(np.float32).astype(np.float64)
    _, _, tro = orc.ntd_fit(X32, F0, G0, 120)
    out = {}
    for tol in (0.0, 0.5):
        F = _dev(F0, torch.float32)
        G = torch.tensor(G0, dtype=torch.float32, device="cuda")
        err, tr = native.ntd_fit(Xd, F, G, 120, precision="bf16", refine_iters=10,
                                 exact_every=10, refine_tol=tol)
        out[tol] = (native.nnc_last_refine_sweep(), err, tr.cpu().numpy())
    assert out[0.0][0] == 110
    sweep, err, tr = out[0.5]
    assert sweep % 10 == 0 and 20 <= sweep <= 110
    # The entries that measure the iterate itself: the exact checkpoints (an
    # explicit FP64 pass) and the FP32 refinement sweeps' identity. The BF16
    # sweeps' identity entries carry the BF16 error of their terms, about
    # 2^-9 / (2 rel), and are not compared.
    ck = np.arange(9, 120, 10)
    assert np.abs(tr[ck] - tro[ck]).max() <= 1e-3
    assert np.abs(tr[sweep:] - tro[sweep:]).max() <= 1e-3
    assert abs(err - tro[-1]) <= 1e-3
